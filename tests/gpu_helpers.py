"""Shared helpers of the GPU parity tests: build the oracle and the CUDA solver
on the same seeded LP with the same options, and compare results."""
import numpy as np

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import pdhg as P

# option names shared by the oracle's Options and the C ABI's pdhg_options
SHARED = ("ruiz_iters", "pock_chambolle", "pc_alpha", "power_iters", "step_factor", "restarts", "primal_weight",
          "eval_every", "beta_suff", "beta_nec", "beta_art", "theta", "eps_cross", "eps_factor", "snapshot_every")

TINY_PLAIN = dict(pock_chambolle=False, restarts=False, primal_weight=False)  # Ruiz only, fixed step, omega = 1


def pair(lp, x0=None, y0=None, **opts):
    """(oracle, solver) on the same LP and options."""
    oopt = O.Options(**opts)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt, x0=x0, y0=y0)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, x0=x0, y0=y0, **copts)
    return orc, sol


def rel_err(a, b):
    """Relative error ||a - b|| / ||b|| (absolute when b is zero)."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def max_rel_err(a, b):
    """Largest elementwise error relative to the largest magnitude of b."""
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = float(np.max(np.abs(b))) if b.size else 1.0
    return float(np.max(np.abs(a - b)) / (scale if scale > 0 else 1.0)) if b.size else 0.0


def assert_iterates_close(sol, orc, tol, which=P.PDHG_CURRENT):
    x, y, z = sol.solution(which)
    if which == P.PDHG_CURRENT:
        xo, yo, zo = orc.solution()
    elif which == P.PDHG_AVERAGE:
        xo, yo, zo = orc.unscale(orc.x_avg, orc.y_avg)
    else:
        xo, yo, zo = orc.unscale(orc.x_r, orc.y_r)
    # z = max(0, c - A^T y) is a difference of terms of the size of c, so its
    # error is measured against max(||z||, ||c||) (z itself is ~0 at an optimum).
    c_norm = float(np.linalg.norm(orc.c))
    for name, a, b, floor in (("x", x, xo, 0.0), ("y", y, yo, 0.0), ("z", z, zo, c_norm)):
        nb = max(float(np.linalg.norm(b)), floor)
        e1 = float(np.linalg.norm(np.asarray(a) - b)) / (nb if nb > 0 else 1.0)
        mb = max(float(np.max(np.abs(b))) if b.size else 0.0, floor / max(1.0, np.sqrt(b.size)))
        e2 = float(np.max(np.abs(np.asarray(a) - b))) / (mb if mb > 0 else 1.0) if b.size else 0.0
        assert e1 <= tol and e2 <= tol, f"{name}: rel {e1:.3e} max-rel {e2:.3e} > {tol:.1e}"


def compare_traces(gpu_trace, orc_trace, near_tie=1e-6):
    """Decisions (iteration, kind, candidate) must agree. A differing decision
    is accepted only where the oracle's decision margin is at rounding level
    (a near-tie that a different summation order can flip) or the method has
    already converged to rounding noise (rel. KKT <= 1e-12); the trajectories
    may part after it, so comparison stops there. Returns the number of
    evaluations compared."""
    assert len(gpu_trace) == len(orc_trace)
    for i, (g, o) in enumerate(zip(gpu_trace, orc_trace)):
        if (g["iteration"], g["kind"], g["candidate"]) != (o.iteration, o.kind, o.candidate):
            assert g["iteration"] == o.iteration
            # a near-tie, or KKT errors already at the FP64 noise floor
            assert o.margin <= near_tie or o.rel_kkt <= 1e-12, (i, g, o)
            return i
    return len(orc_trace)


# Long restarted runs: two FP64 runs that differ only in summation order and
# in eta by a few ulps stay within 1.3e-14 (iterates), 2.7e-8 (omega) and
# 8e-16 (rel. KKT, absolute) of each other over a whole solve
# (tests/test_oracle_rounding_spread.py); the GPU tests allow 100x or more.
LONG_RUN_ITERATES = 1e-10
LONG_RUN_OMEGA = 1e-6
LONG_RUN_RELKKT = dict(rel=1e-6, abs=1e-13)


def compare_at(lp, k, tol, rtol=LONG_RUN_ITERATES, **opts):
    """Run a fresh (oracle, solver) pair on lp with opts for exactly k
    iterations (tolerance tol) and compare the current, average and
    last-restart points at rtol. Both sides are deterministic, so this
    reproduces the state of a longer run at its evaluation k: the check made
    at the last evaluation on which two longer runs still agreed."""
    import pytest

    orc, sol = pair(lp, **opts)
    orc.run(k, tol)
    st, done = sol.iterate(k, tol)
    assert done == orc.k == k, (done, orc.k, k)
    assert len(sol.trace()) == len(orc.trace)
    for g, o in zip(sol.trace(), orc.trace):
        assert (g["iteration"], g["kind"], g["candidate"]) == (o.iteration, o.kind, o.candidate)
        assert g["omega"] == pytest.approx(o.omega, rel=LONG_RUN_OMEGA)
    assert_iterates_close(sol, orc, rtol)
    assert_iterates_close(sol, orc, rtol, P.PDHG_AVERAGE)
    assert_iterates_close(sol, orc, rtol, P.PDHG_LAST_RESTART)
    sol.close()
