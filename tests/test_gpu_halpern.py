"""Reflected Halpern form of the iteration (option halpern) against the
oracle's Halpern variant: the same bars as the parity tests (1e-10 after 100
iterations, identical decision traces, converged objectives within 1e-7 of
the closed-form optimum)."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, TINY_PLAIN, assert_iterates_close, compare_traces, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _pair(lp, rho=1.0, engine=None, **opts):
    oopt = O.Options(halpern=True, halpern_reflect=rho, **opts)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, halpern=1, halpern_reflect=rho,
                   **(engine or {}), **copts)
    return orc, sol


@pytest.mark.parametrize("rho", [0.0, 0.5, 1.0])
def test_fixed_step_100_iterations(tiny_lp, rho):
    orc, sol = _pair(tiny_lp, rho, **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)


def test_restarted_100_iterations(tiny_lp):
    orc, sol = _pair(tiny_lp)
    orc.run(100)
    sol.iterate(100)
    assert [r["kind"] for r in sol.trace()] == [r.kind for r in orc.trace]
    assert all(r["candidate"] == P.PDHG_RESTART_TO_CURRENT for r in sol.trace())
    assert_iterates_close(sol, orc, 1e-10)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)


def test_restarted_trace(tiny_lp):
    orc, sol = _pair(tiny_lp)
    orc.run(3000, 1e-10)
    sol.iterate(3000, 1e-10)
    tr = sol.trace()
    assert len(tr) == len(orc.trace) >= 10
    agreed = compare_traces(tr, orc.trace)
    assert agreed >= 10
    for g, o in zip(tr[:agreed], orc.trace[:agreed]):
        assert g["omega"] == pytest.approx(o.omega, rel=1e-6)


def test_converges_to_known_optimum(tiny_lp):
    orc, sol = _pair(tiny_lp)
    st, done = sol.iterate(200000, 1e-8)
    assert st == P.PDHG_OK
    k = sol.kkt()
    assert k["rel_kkt"] <= 1e-8
    assert k["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=1e-7)
    assert orc.run(200000, 1e-8)
    assert done == orc.k
    x, _, _ = sol.solution()
    assert rel_err(x, tiny_lp.x_star) <= 1e-6


def test_graph_replay_matches_direct_launches(tiny_lp):
    sols = []
    for g in (0, 1):
        _, s = _pair(tiny_lp, engine=dict(use_graphs=g))
        s.iterate(1000)
        sols.append(s.solution())
    for a, b in zip(*sols):
        np.testing.assert_array_equal(a, b)


def test_fp32_close_to_fp64_oracle(tiny_lp):
    orc, _ = _pair(tiny_lp, **TINY_PLAIN)
    orc.run(100)
    with P.Solver.from_lp(tiny_lp, precision=P.PDHG_FP32, halpern=1, pock_chambolle=0, restarts=0,
                          primal_weight=0) as sol:
        sol.iterate(100)
        x, y, _ = sol.solution()
    xo, yo, _ = orc.solution()
    assert rel_err(x, xo) < 1e-4 and rel_err(y, yo) < 1e-4
    assert rel_err(x, xo) > 0


def test_fp32_panels_match_direct_fp32(tiny_lp):
    runs = []
    for opts in (dict(primal_panels=1, panel_rows=32), dict(primal_panels=0)):
        with P.Solver.from_lp(tiny_lp, precision=P.PDHG_FP32, halpern=1, **opts) as sol:
            sol.iterate(640)
            runs.append(sol.solution())
    for a, b in zip(*runs):
        assert rel_err(a, b) <= 1e-4


@pytest.mark.parametrize("panels", [0, 1])
def test_mixed_reaches_tolerance_and_optimum(tiny_lp, panels):
    lp = tiny_lp
    # an explicit switch: the refined FP32 phase (the default) to 1e-5, then FP64
    with P.Solver.from_lp(lp, precision=P.PDHG_MIXED, halpern=1, primal_panels=panels, panel_rows=48,
                          polish_switch=1e-5) as sol:
        st, done = sol.iterate(200000, 1e-8)
        info = sol.info()
        k = sol.kkt()
    assert st == P.PDHG_OK and k["rel_kkt"] <= 1e-8
    assert info["precision_now"] == P.PDHG_FP64 and 0 < info["polish_started_at"] <= done
    assert k["primal_obj"] == pytest.approx(lp.f_star, rel=1e-7)


def test_option_checks(tiny_lp):
    for bad in (dict(persistent=1), dict(halpern_reflect=1.5), dict(record_for_backward=1, restarts=0,
                                                                      primal_weight=0)):
        with pytest.raises(P.PDHGError) as ei:
            P.Solver.from_lp(tiny_lp, halpern=1, **bad)
        assert ei.value.status == P.PDHG_ERR_INVALID, bad
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny_lp, tiny_lp], halpern=1, persistent=1)


def test_batch_matches_single_lp_engine():
    from paper_2510_24429_b300 import lpgen

    sizes = [200, 17, 1000, 333, 50]
    lps = [lpgen.generate(m, max(1, int(round(2.5 * m))), 500 + i, nnz_per_col=min(5, m), support=0.3)
           for i, m in enumerate(sizes)]
    lps.append(lpgen.tiny_lp(0))
    tol = 1e-6
    with P.BatchSolver(lps, halpern=1) as bs:
        st, _ = bs.iterate(100000, tol)
        info = bs.info()
        sols = [bs.solution(i) for i in range(len(lps))]
    assert st == P.PDHG_OK and info["converged"].all()
    for i, lp in enumerate(lps):
        with P.Solver.from_lp(lp, halpern=1) as s:
            st1, k1 = s.iterate(100000, tol)
        assert st1 == P.PDHG_OK
        assert abs(int(info["iterations"][i]) - k1) <= 2 * 64, (i, info["iterations"][i], k1)
        x = sols[i][0]
        assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=10 * tol, abs=10 * tol), i
