"""The single-block solve loop (option persistent): one launch runs the
iterations, the evaluations, the restart decisions and the termination test of
a small LP, with its vectors in shared memory.

Its half-steps sum every row in the multi-launch engine's order, so plain runs
(no evaluations) are bit-identical to that engine; with evaluations only the
grouping of the evaluation sums differs (rounding-level agreement, decisions
identical up to near-ties). Against the oracle it is held to the parity
tests' bars: 1e-10 after 100 iterations, identical decision traces, converged
objectives within 1e-7 of the closed-form optimum."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, TINY_PLAIN, assert_iterates_close, compare_traces, max_rel_err, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _solvers(lp, persistent, **opts):
    """(oracle, solver with the given persistent flag) on the same LP and options."""
    oopt = O.Options(**opts)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    return orc, P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, persistent=persistent, **copts)


def test_plain_run_bit_identical_to_multi_launch_engine(tiny_lp):
    _, sp = _solvers(tiny_lp, 1, **TINY_PLAIN)
    _, sm = _solvers(tiny_lp, 0, **TINY_PLAIN)
    assert sp.iterate(1000) == sm.iterate(1000) == (P.PDHG_OK, 1000)
    for a, b in zip(sp.solution(), sm.solution()):
        np.testing.assert_array_equal(a, b)
    assert sp.info()["kernel_launches"] == 1


def test_plain_100_iterations_match_oracle(tiny_lp):
    orc, sol = _solvers(tiny_lp, 1, **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)


def test_restarted_100_iterations_match_oracle(tiny_lp):
    orc, sol = _solvers(tiny_lp, 1)
    orc.run(100)
    sol.iterate(100)
    assert [r["kind"] for r in sol.trace()] == [r.kind for r in orc.trace] != [0]
    assert_iterates_close(sol, orc, 1e-10)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_AVERAGE)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)


def test_restarted_trace_matches_oracle(tiny_lp):
    orc, sol = _solvers(tiny_lp, 1)
    orc.run(3000, 1e-10)
    sol.iterate(3000, 1e-10)
    tr = sol.trace()
    assert len(tr) == len(orc.trace) >= 20
    agreed = compare_traces(tr, orc.trace)
    assert agreed >= 20
    for g, o in zip(tr[:agreed], orc.trace[:agreed]):
        assert g["omega"] == pytest.approx(o.omega, rel=1e-6)
        assert g["rel_kkt"] == pytest.approx(o.rel_kkt, rel=1e-5)
    if agreed == len(tr):
        assert_iterates_close(sol, orc, 1e-6)


def test_converges_to_known_optimum_like_multi_launch(tiny_lp):
    orc, sp = _solvers(tiny_lp, 1)
    _, sm = _solvers(tiny_lp, 0)
    st, done = sp.iterate(200000, 1e-8)
    st_m, done_m = sm.iterate(200000, 1e-8)
    assert st == st_m == P.PDHG_OK
    assert abs(done - done_m) <= 2 * 64
    assert orc.run(200000, 1e-8)
    k = sp.kkt()
    assert k["rel_kkt"] <= 1e-8
    assert k["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=1e-7)
    assert k["primal_obj"] == pytest.approx(float(tiny_lp.c @ orc.solution()[0]), rel=1e-7)
    x, _, _ = sp.solution()
    assert rel_err(x, tiny_lp.x_star) <= 1e-6
    assert sp.info()["kernel_launches"] <= 2


def test_algorithm1_snapshots(tiny_lp):
    """The launch returns at each scheduled snapshot; the host takes it and
    launches again."""
    orc, sol = _solvers(tiny_lp, 1, eps_cross=1e-2, eps_factor=0.1)
    assert orc.run(200000, 1e-7)
    sol.iterate(200000, 1e-7)
    cnt, _ = sol.snapshot_poll()
    assert cnt == len(orc.snapshots) >= 4
    snap = sol.snapshot()
    ref = orc.snapshots[-1]
    assert snap["iteration"] == ref["iteration"]
    for key in ("x", "y", "z"):
        assert max_rel_err(snap[key], ref[key]) <= 1e-8, key


def test_resume_in_chunks(tiny_lp):
    orc, sol = _solvers(tiny_lp, 1)
    orc.run(1000)
    for chunk in (1, 63, 200, 736):
        sol.iterate(chunk)
    assert sol.info()["iterations"] == 1000
    if compare_traces(sol.trace(), orc.trace) == len(orc.trace):
        assert_iterates_close(sol, orc, 1e-6)


def _small_lps():
    sizes = [200, 17, 1000, 333, 50, 1, 120]
    lps = [lpgen.generate(m, max(1, int(round(2.5 * m))), 300 + i, nnz_per_col=min(5, m), support=0.3)
           for i, m in enumerate(sizes)]
    lps.append(lpgen.tiny_lp(0))
    return lps


def test_batch_one_block_per_instance():
    lps = _small_lps()
    tol = 1e-7
    with P.BatchSolver(lps, persistent=1) as bp:
        st, done = bp.iterate(100000, tol)
        info = bp.info()
        sols = [bp.solution(i) for i in range(len(lps))]
    assert st == P.PDHG_OK and info["converged"].all() and (info["rel_kkt"] <= tol).all()
    assert done == info["iterations"].max()
    with P.BatchSolver(lps) as bm:
        bm.iterate(100000, tol)
        info_m = bm.info()
    for i, lp in enumerate(lps):
        assert abs(int(info["iterations"][i]) - int(info_m["iterations"][i])) <= 2 * 64, i
        x, _, _ = sols[i]
        assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=10 * tol, abs=10 * tol), i


def test_options_checked():
    big = lpgen.generate(2000, 5000, 1, nnz_per_col=3)
    with pytest.raises(P.PDHGError) as ei:
        P.Solver.from_lp(big, persistent=1)
    assert ei.value.status == P.PDHG_ERR_INVALID and "shared memory" in str(ei.value)
    tiny = lpgen.tiny_lp(0)
    for bad in (dict(precision=P.PDHG_FP32), dict(kernel_timing=1), dict(record_for_backward=1, restarts=0,
                                                                           primal_weight=0)):
        with pytest.raises(P.PDHGError) as ei:
            P.Solver.from_lp(tiny, persistent=1, **bad)
        assert ei.value.status == P.PDHG_ERR_INVALID, bad
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny, big], persistent=1)
