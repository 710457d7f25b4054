"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: FP64 iterates after 100 iterations agree to 1e-10 relative error;
converged objectives to 1e-7 relative (also against the generator's closed-form
optimum f*). Restart decisions (iteration, kind, candidate) must be identical.
"""
import math

import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import (LONG_RUN_ITERATES, LONG_RUN_OMEGA, LONG_RUN_RELKKT, TINY_PLAIN, assert_iterates_close,
                               compare_at, compare_traces, max_rel_err, pair, rel_err)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.mark.parametrize("opts", [TINY_PLAIN, {}])
def test_setup_matches_oracle(tiny_lp, opts):
    orc, sol = pair(tiny_lp, **opts)
    info = sol.info()
    assert info["norm_estimate"] == pytest.approx(orc.norm_est, rel=1e-12)
    assert info["eta"] == pytest.approx(orc.eta, rel=1e-12)
    assert info["omega"] == pytest.approx(orc.omega, rel=1e-12)
    assert info["tau"] == pytest.approx(orc.tau, rel=1e-12)
    # the starting point is the restart reference; KKT of x = 0, y = 0
    k = sol.kkt()
    ko = O.kkt(orc.A, orc.b, orc.c, *orc.solution()[:2])
    for key in ("rp_norm2", "rd_norm2", "rel_kkt"):
        assert k[key] == pytest.approx(ko[key], rel=1e-12)


def test_plain_pdhg_100_iterations(tiny_lp):
    orc, sol = pair(tiny_lp, **TINY_PLAIN)
    orc.run(100)
    st, done = sol.iterate(100)
    assert st == P.PDHG_OK and done == 100
    assert_iterates_close(sol, orc, 1e-10)


def test_plain_pdhg_20k_iterations(tiny_lp):
    """The tiny configuration as specified: Ruiz, fixed step, 20k iterations."""
    orc, sol = pair(tiny_lp, **TINY_PLAIN)
    orc.run(20000)
    sol.iterate(20000)
    assert_iterates_close(sol, orc, 1e-9)
    x, _, _ = sol.solution()
    assert float(tiny_lp.c @ x) == pytest.approx(float(tiny_lp.c @ orc.solution()[0]), rel=1e-10)


def test_restarted_pdhg_100_iterations(tiny_lp):
    """Default options (Ruiz + Pock-Chambolle, restarts, primal weight): the
    first evaluation restarts and updates omega, and iterates still agree to
    1e-10 after 100 iterations."""
    orc, sol = pair(tiny_lp)
    orc.run(100)
    sol.iterate(100)
    assert [r["kind"] for r in sol.trace()] == [r.kind for r in orc.trace] != [0]
    assert_iterates_close(sol, orc, 1e-10)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_AVERAGE)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)


def test_restarted_trace_and_iterates(tiny_lp):
    """Decisions must be identical over a long restarted run, and omega,
    rel. KKT and the iterates stay within 100x (or more) of the spread that a
    change of summation order alone causes (measured on the oracle:
    tests/test_oracle_rounding_spread.py). If a near-tie splits the traces,
    the iterates are compared at the last evaluation both runs agreed on."""
    orc, sol = pair(tiny_lp)
    orc.run(3000, 1e-10)
    sol.iterate(3000, 1e-10)
    tr = sol.trace()
    assert len(tr) == len(orc.trace) >= 20
    agreed = compare_traces(tr, orc.trace)
    assert agreed >= 20
    for g, o in zip(tr[:agreed], orc.trace[:agreed]):
        assert g["omega"] == pytest.approx(o.omega, rel=LONG_RUN_OMEGA)
        assert g["rel_kkt"] == pytest.approx(o.rel_kkt, **LONG_RUN_RELKKT)
    assert sum(1 for r in tr[:agreed] if r["kind"]) >= 3
    if agreed == len(tr):
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES)
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES, P.PDHG_AVERAGE)
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES, P.PDHG_LAST_RESTART)
    else:
        compare_at(tiny_lp, tr[agreed - 1]["iteration"], 1e-10)


def test_converged_objective(tiny_lp):
    orc, sol = pair(tiny_lp)
    assert orc.run(200000, 1e-8)
    st, done = sol.iterate(200000, 1e-8)
    assert st == P.PDHG_OK and sol.info()["converged"] == 1
    assert done == orc.k
    k = sol.kkt()
    assert k["rel_kkt"] <= 1e-8
    assert k["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=1e-7)
    assert k["primal_obj"] == pytest.approx(float(tiny_lp.c @ orc.solution()[0]), rel=1e-7)
    x, _, _ = sol.solution()
    assert rel_err(x, tiny_lp.x_star) <= 1e-6


def test_kkt_of_each_point_matches_oracle(tiny_lp):
    orc, sol = pair(tiny_lp)
    orc.run(500)
    sol.iterate(500)
    points = {P.PDHG_CURRENT: (orc.x, orc.y), P.PDHG_AVERAGE: (orc.x_avg, orc.y_avg),
              P.PDHG_LAST_RESTART: (orc.x_r, orc.y_r)}
    for which, (xh, yh) in points.items():
        k = sol.kkt(which)
        ko = orc.kkt_of(xh, yh)
        for key, v in ko.items():
            assert k[key] == pytest.approx(v, rel=1e-8, abs=1e-12), (which, key)
        assert k["iteration"] == 500


def test_algorithm1_snapshot_schedule(tiny_lp):
    orc, sol = pair(tiny_lp, eps_cross=1e-2, eps_factor=0.1)
    assert orc.run(200000, 1e-7)
    sol.iterate(200000, 1e-7)
    cnt, _ = sol.snapshot_poll()
    assert cnt == len(orc.snapshots) >= 4
    snap = sol.snapshot()
    ref = orc.snapshots[-1]
    assert snap["iteration"] == ref["iteration"]
    assert snap["rel_kkt"] == pytest.approx(ref["rel_kkt"], rel=1e-6)
    for key in ("x", "y", "z"):
        assert max_rel_err(snap[key], ref[key]) <= 1e-8, key


def test_periodic_snapshots(tiny_lp):
    orc, sol = pair(tiny_lp, snapshot_every=1000)
    orc.run(3008)
    sol.iterate(3008)
    cnt, _ = sol.snapshot_poll()
    assert cnt == len(orc.snapshots) == 3
    snap = sol.snapshot()
    assert snap["iteration"] == orc.snapshots[-1]["iteration"] == 3008
    assert max_rel_err(snap["x"], orc.snapshots[-1]["x"]) <= 1e-8


def test_snapshot_before_any_is_state_error(tiny_lp):
    _, sol = pair(tiny_lp, **TINY_PLAIN)
    with pytest.raises(P.PDHGError) as ei:
        sol.snapshot()
    assert ei.value.status == P.PDHG_ERR_STATE


def test_warm_start_at_optimum_is_fixed_point(tiny_lp):
    lp = tiny_lp
    _, sol = pair(lp, x0=lp.x_star, y0=lp.y_star, **TINY_PLAIN)
    assert sol.kkt()["rel_kkt"] < 1e-14
    sol.iterate(64)
    x, y, z = sol.solution()
    assert rel_err(x, lp.x_star) < 1e-13 and rel_err(y, lp.y_star) < 1e-12


def test_resume_equals_single_call(tiny_lp):
    orc, sol = pair(tiny_lp)
    orc.run(1000)
    for chunk in (1, 63, 200, 736):
        sol.iterate(chunk)
    assert sol.info()["iterations"] == 1000
    tr = sol.trace()
    agreed = compare_traces(tr, orc.trace)
    if agreed == len(orc.trace):
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES)
    else:
        assert agreed > 0
        compare_at(tiny_lp, tr[agreed - 1]["iteration"], 0.0)


# ---------------------------------------------------------------------------
# edge shapes
# ---------------------------------------------------------------------------

def _lp_from_dense(A, x_star, y_star, z_star, name):
    m, n = A.shape
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(m + 1, np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return lpgen.LP(m, n, row_ptr, cols.astype(np.int32), A[rows, cols], A @ x_star, A.T @ y_star + z_star,
                    x_star, y_star, z_star, name)


def _edge_lps():
    base = lpgen.tiny_lp(3)
    A = base.dense()
    out = []
    # an empty column (free of constraints, c_j > 0) and an empty row (b_i = 0)
    A2 = np.zeros((A.shape[0] + 1, A.shape[1] + 1))
    A2[:-1, :-1] = A
    out.append(_lp_from_dense(A2, np.append(base.x_star, 0.0), np.append(base.y_star, 0.0),
                              np.append(base.z_star, 1.5), "empty-row-col"))
    # m = 1
    one = lpgen.generate(1, 7, 11, nnz_per_col=1, support=1)
    out.append(one)
    # n = 1
    col = lpgen.generate(5, 1, 12, nnz_per_col=5, support=1)
    out.append(col)
    # one dense row of 10000 nnz plus sparse rows
    n = 10000
    u = lpgen.rand_uniform(7, 99, np.arange(3 * n, dtype=np.uint64)).reshape(3, n)
    A3 = np.zeros((3, n))
    A3[0] = 0.1 + 0.9 * u[0]
    mask = u[1] < 0.001
    A3[1, mask] = -(0.1 + 0.9 * u[2, mask])
    A3[2, ::997] = 1.0
    xs = np.zeros(n)
    xs[[0, 5, 997 * 3]] = [1.0, 0.5, 2.0]
    zs = np.where(xs > 0, 0.0, 1.0)
    out.append(_lp_from_dense(A3, xs, np.array([0.3, -0.7, 1.1]), zs, "long-row"))
    # several tiles plus a ragged tail
    out.append(lpgen.generate(3001, 7919, 5, nnz_per_col=5, support=0.3))
    return out


@pytest.mark.parametrize("lp", _edge_lps(), ids=lambda lp: f"{lp.m}x{lp.n}")
def test_edge_shapes(lp):
    orc, sol = pair(lp, **TINY_PLAIN)
    orc.run(100)
    sol.iterate(100)
    assert_iterates_close(sol, orc, 1e-10)
    # restarted, stopped at 1e-9 before rounding noise can decide a restart
    orc, sol = pair(lp)
    orc.run(640, 1e-9)
    sol.iterate(640, 1e-9)
    tr = sol.trace()
    agreed = compare_traces(tr, orc.trace)
    if agreed == len(orc.trace):
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES)
    elif agreed > 0:
        compare_at(lp, tr[agreed - 1]["iteration"], 1e-9)


# ---------------------------------------------------------------------------
# the large workload, in the configuration the benchmark runs
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def large_lp():
    return lpgen.large_lp(0)


def test_large_fixed_point_and_kkt(large_lp):
    """At m=1e6, n=3e6, nnz~3e7: the generator's optimum is a fixed point of the
    GPU iteration, and its KKT measures vanish."""
    lp = large_lp
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, x0=lp.x_star, y0=lp.y_star)
    k = sol.kkt()
    assert k["rel_kkt"] < 1e-13
    assert k["primal_obj"] == pytest.approx(lp.f_star, rel=1e-13)
    sol.iterate(128)
    x, y, _ = sol.solution()
    assert rel_err(x, lp.x_star) < 1e-12 and rel_err(y, lp.y_star) < 1e-11
    sol.close()


def test_large_setup_and_first_iterations_match_oracle(large_lp):
    """Full-size setup (scaling, power iteration, omega0) and two iterations."""
    lp = large_lp
    orc, sol = pair(lp, restarts=False)
    info = sol.info()
    assert info["norm_estimate"] == pytest.approx(orc.norm_est, rel=1e-10)
    assert info["omega"] == pytest.approx(orc.omega, rel=1e-10)
    orc.run(2)
    sol.iterate(2)
    assert_iterates_close(sol, orc, 1e-10)
    sol.close()


@pytest.mark.parametrize("hot", [64, 500])
def test_dual_step_with_shared_memory_hot_columns(tiny_lp, hot):
    """The persistent dual step that stages xbar[0, hot) in shared memory gives
    the same iterates (hot = 64: part staged, part gathered from global
    memory; hot = 500: all of xbar staged)."""
    orc, _ = pair(tiny_lp, **TINY_PLAIN)
    orc.run(100)
    sol = P.Solver.from_lp(tiny_lp, pock_chambolle=0, restarts=0, primal_weight=0, dual_hot_cols=hot)
    sol.iterate(100)
    assert_iterates_close(sol, orc, 1e-10)
    lp = lpgen.generate(3001, 7919, 5, nnz_per_col=5, support=0.3)
    orc, _ = pair(lp)
    orc.run(640, 1e-9)
    sol = P.Solver.from_lp(lp, dual_hot_cols=hot * 4)
    sol.iterate(640, 1e-9)
    if compare_traces(sol.trace(), orc.trace) == len(orc.trace):
        assert_iterates_close(sol, orc, 1e-7)


def test_cuda_graph_replay_equals_direct_launches(tiny_lp):
    """Evaluation blocks replayed from a captured CUDA graph give bit-identical
    results to the same launches issued one by one."""
    out = {}
    for g in (0, 1):
        with P.Solver.from_lp(tiny_lp, use_graphs=g) as sol:
            sol.iterate(1000)
            sol.iterate(37)  # an unaligned remainder, then aligned blocks again
            sol.iterate(200)
            out[g] = (sol.solution(), [(r["iteration"], r["kind"], r["omega"]) for r in sol.trace()])
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a, b)
    assert out[0][1] == out[1][1]
    lps = [lpgen.generate(m, int(2.5 * m), 7 + m, nnz_per_col=5, support=0.3) for m in (40, 300, 90)]
    sols = {}
    for g in (0, 1):
        with P.BatchSolver(lps, use_graphs=g) as bs:
            bs.iterate(640, 1e-7)
            sols[g] = [bs.solution(i) for i in range(len(lps))], bs.info()["iterations"]
    np.testing.assert_array_equal(sols[0][1], sols[1][1])
    for s0, s1 in zip(sols[0][0], sols[1][0]):
        for a, b in zip(s0, s1):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("alpha", [0.0, 0.5, 2.0])
def test_pock_chambolle_alphas_match_oracle(tiny_lp, alpha):
    """Pock-Chambolle with alpha != 1 (the default): setup and 100 plain
    iterations against the oracle."""
    orc, sol = pair(tiny_lp, pc_alpha=alpha, restarts=False, primal_weight=False)
    info = sol.info()
    assert info["norm_estimate"] == pytest.approx(orc.norm_est, rel=1e-12)
    orc.run(100)
    sol.iterate(100)
    assert_iterates_close(sol, orc, 1e-10)
    sol.close()
