"""Parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times (the panel-tiled primal half-step of large
LPs, CUDA-graph replay):

* the m=1e6, n=3e6, nnz=3e7 LP in the benchmark's own configuration (restarts,
  primal weight, evaluations every 64 iterations, snapshots): 192 FP64
  iterations against the oracle - three evaluations, two restarts with primal
  weight updates, every decision equal, the current, average and last-restart
  points at 1e-10 and the snapshot at 1e-8; the reflected Halpern form in FP64
  after 100 iterations against the oracle's Halpern variant (1e-10); the FP32
  engine after 100 iterations against the FP64 oracle (FP32 rounding, error
  printed, bound 1e-4);
* the adjoint LP (m=1e5, n=3e5, 6 entries per column): the reverse pass through
  500 unrolled FP64 iterations (the configured K, checkpoints every 50, so ten
  recomputed segments) against the oracle's reverse pass (1e-9);
* the 256-LP batch (m log-uniform in [1e3, 1e5]) solved to 1e-6: every
  instance checked against properties that hold at any size - its solution's
  residuals and gap recomputed on the host with scipy meet the tolerance, and
  its objective is close to the generator's known optimum.

The large-LP oracle takes about a minute to set up (scaling and 100 power
iterations over 3e7 entries in scipy); it is built once for the module."""
import copy
import dataclasses

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, assert_iterates_close, compare_traces, max_rel_err, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.fixture(scope="module")
def large():
    lp = lpgen.large_lp(0)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(restarts=False))
    return lp, orc


def _fresh(orc, **changes):
    """A copy of the oracle at its starting point with changed options (the
    scaled matrices are shared; nothing below modifies them)."""
    o = copy.copy(orc)
    o.opt = dataclasses.replace(orc.opt, **changes)
    for k in ("x", "y", "x_sum", "y_sum", "x_r", "y_r"):
        setattr(o, k, getattr(orc, k).copy())
    o.trace, o.snapshots, o.polish_log = [], [], []
    o.next_snapshot, o.eps_target = o.opt.snapshot_every, o.opt.eps_cross  # the schedule of the new options
    return o


def _solver(lp, orc, **engine):
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(orc.opt, k)) for k in SHARED)}
    return P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, **copts, **engine)


def test_large_restarted_fp64_matches_oracle(large):
    """The benchmark's configuration at full size: restarts and primal weight
    on, evaluations every 64 iterations, a periodic snapshot, panel-tiled
    primal half-step, CUDA-graph replay. 192 iterations: the evaluations at 64
    and 128 restart (the artificial rule: t >= 0.36 k) and update omega, the
    one at 192 decides on the decay rules. Every decision and omega must be
    equal, the three points agree at 1e-10 and the snapshot taken at iteration
    128 at 1e-8."""
    lp, orc0 = large
    orc = _fresh(orc0, restarts=True, snapshot_every=128)
    orc.run(192)
    with _solver(lp, orc) as sol:
        info = sol.info()
        assert info["norm_estimate"] == pytest.approx(orc.norm_est, rel=1e-10)
        st, done = sol.iterate(192)
        assert done == 192
        tr = sol.trace()
        assert len(tr) == len(orc.trace) == 3
        assert compare_traces(tr, orc.trace) == 3, (tr, orc.trace)
        for g, o in zip(tr, orc.trace):
            assert g["omega"] == pytest.approx(o.omega, rel=1e-10)
            assert g["rel_kkt"] == pytest.approx(o.rel_kkt, rel=1e-9)
        assert [r["kind"] for r in tr[:2]] != [0, 0] and sol.info()["restarts"] >= 2
        errs = {}
        for which, name in ((P.PDHG_CURRENT, "current"), (P.PDHG_AVERAGE, "average"),
                            (P.PDHG_LAST_RESTART, "last restart")):
            assert_iterates_close(sol, orc, 1e-10, which)
            x, y, _ = sol.solution(which)
            xo, yo, _ = (orc.solution() if which == P.PDHG_CURRENT else
                         orc.unscale(orc.x_avg, orc.y_avg) if which == P.PDHG_AVERAGE else
                         orc.unscale(orc.x_r, orc.y_r))
            errs[name] = (rel_err(x, xo), rel_err(y, yo))
        print("large LP, restarted FP64 vs oracle after 192 iterations (x, y):",
              {k: f"{a:.1e} {b:.1e}" for k, (a, b) in errs.items()})
        cnt, _ = sol.snapshot_poll()
        assert cnt == len(orc.snapshots) == 1
        snap = sol.snapshot()
        ref = orc.snapshots[-1]
        assert snap["iteration"] == ref["iteration"] == 128
        for key in ("x", "y", "z"):
            assert max_rel_err(snap[key], ref[key]) <= 1e-8, key


def test_large_halpern_fp64_100_iterations(large):
    lp, orc0 = large
    orc = _fresh(orc0, halpern=True)
    orc.run(100)
    with _solver(lp, orc, halpern=1) as sol:
        sol.iterate(100)
        assert_iterates_close(sol, orc, 1e-10)
        x, y, _ = sol.solution()
    xo, yo, _ = orc.solution()
    print(f"large LP, Halpern FP64 vs oracle after 100 iterations: x {rel_err(x, xo):.1e}, y {rel_err(y, yo):.1e}")


def test_large_fixed_point_scheme_matches_oracle(large):
    """The cuPDLP+ restart scheme (restart_scheme = 1, reflected Halpern, PID
    primal weight) at full size: 192 iterations, three evaluations (two
    artificial restarts to T(z) with PID steps), decisions equal, iterates at
    1e-10."""
    lp, orc0 = large
    orc = _fresh(orc0, restarts=True, halpern=True, restart_scheme=1)
    orc.r_restart = orc.r_prev = orc.fixed_point_measure(orc.x, orc.y)[0]
    orc.pid_integral, orc.pid_prev = 0.0, 0.0
    orc.run(192)
    with _solver(lp, orc, halpern=1, restart_scheme=1) as sol:
        sol.iterate(192)
        tr = sol.trace()
        assert compare_traces(tr, orc.trace) == 3
        assert sum(1 for r in tr if r["kind"] == P.PDHG_RESTART_TO_PDHG_STEP) >= 2
        for g, o in zip(tr, orc.trace):
            assert g["omega"] == pytest.approx(o.omega, rel=1e-10)
        assert_iterates_close(sol, orc, 1e-10)
        assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)


def test_large_fp32_100_iterations_close_to_fp64_oracle(large):
    """FP32 half-steps against the FP64 oracle: the error is FP32 rounding
    (unit roundoff 6e-8) carried through 100 iterations; it is printed and
    bounded by 1e-4."""
    lp, orc0 = large
    orc = _fresh(orc0)
    orc.run(100)
    with _solver(lp, orc, precision=P.PDHG_FP32) as sol:
        assert sol.info()["precision_now"] == P.PDHG_FP32
        sol.iterate(100)
        x, y, _ = sol.solution()
    xo, yo, _ = orc.solution()
    ex, ey = rel_err(x, xo), rel_err(y, yo)
    print(f"large LP, FP32 vs FP64 oracle after 100 iterations: x {ex:.2e}, y {ey:.2e}")
    assert 0 < max(ex, ey) and ex < 1e-4 and ey < 1e-4


def test_adjoint_lp_reverse_pass_matches_oracle():
    lp = lpgen.adjoint_lp(0)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                   O.Options(restarts=False, primal_weight=False))
    K = 500
    rng = np.random.default_rng(3)
    gx, gy = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    gc_o, gb_o = O.unrolled_adjoint(orc, K, gx, gy)
    with P.Solver.from_lp(lp, restarts=0, primal_weight=0, record_for_backward=1, checkpoint_every=50) as sol:
        sol.iterate(K)
        gc, gb = sol.backward(gx, gy)
    assert rel_err(gc, gc_o) <= 1e-9 and rel_err(gb, gb_o) <= 1e-9


def test_batch_of_256_lps_to_1e6():
    sizes = lpgen.batch_sizes(0, 256)
    lps = [lpgen.batch_lp(0, i, m) for i, m in enumerate(sizes)]
    tol = 1e-6
    with P.BatchSolver(lps) as bs:
        st, _ = bs.iterate(200_000, tol)
        info = bs.info()
        assert st == P.PDHG_OK and bool(np.all(info["converged"]))
        worst_obj = 0.0
        for i, lp in enumerate(lps):
            x, y, _ = bs.solution(i)
            A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
            rp = np.linalg.norm(lp.b - A @ x) / (1 + np.linalg.norm(lp.b))
            rd = np.linalg.norm(np.maximum(0.0, A.T @ y - lp.c)) / (1 + np.linalg.norm(lp.c))
            cx, by = float(lp.c @ x), float(lp.b @ y)
            rg = abs(cx - by) / (1 + abs(cx) + abs(by))
            assert max(rp, rd, rg) <= tol * (1 + 1e-6), (i, rp, rd, rg)
            assert float(x.min()) >= 0.0
            worst_obj = max(worst_obj, abs(cx - lp.f_star) / (1 + abs(lp.f_star)))
    print(f"256 LPs to {tol:g}: worst objective error vs the known optimum {worst_obj:.2e}")
    assert worst_obj <= 1e-4
