"""The fixed-point residual restart scheme with the PID primal weight
(restart_scheme = 1, the cuPDLP+ line the paper's solver follows, Section
4.1; readings) on the GPU, against the oracle's pinned version of the scheme:
iterates after 100 iterations at 1e-10, decision traces and primal weights
over whole restarted solves (with the long-run tolerances measured in
tests/test_oracle_rounding_spread.py), the panel-tiled large-LP layout, the
FP32 and mixed forms against the known optimum, and the option checks."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import (LONG_RUN_ITERATES, LONG_RUN_OMEGA, SHARED, assert_iterates_close, compare_traces)

pytestmark = pytest.mark.gpu

FP = dict(halpern=True, restart_scheme=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _pair(lp, engine=None, **opts):
    oopt = O.Options(**FP, **opts)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, halpern=1, restart_scheme=1,
                   pid_kp=oopt.pid_kp, pid_ki=oopt.pid_ki, pid_kd=oopt.pid_kd, **(engine or {}), **copts)
    return orc, sol


def test_100_iterations_match_oracle(tiny_lp):
    orc, sol = _pair(tiny_lp)
    orc.run(100)
    sol.iterate(100)
    tr = sol.trace()
    assert [(r["iteration"], r["kind"]) for r in tr] == [(r.iteration, r.kind) for r in orc.trace]
    assert tr[0]["kind"] == P.PDHG_RESTART_TO_PDHG_STEP  # the first evaluation restarts (t >= 0.36 k)
    assert tr[0]["omega"] == pytest.approx(orc.trace[0].omega, rel=1e-12)
    assert_iterates_close(sol, orc, 1e-10)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)


@pytest.mark.parametrize("gains", [(0.99, 0.01, 0.0), (0.5, 0.0, 0.0), (0.3, 0.2, 0.1)])
def test_restarted_solve_traces_match_oracle(tiny_lp, gains):
    kp, ki, kd = gains
    orc, sol = _pair(tiny_lp, pid_kp=kp, pid_ki=ki, pid_kd=kd)
    assert orc.run(200_000, 1e-10)
    st, done = sol.iterate(200_000, 1e-10)
    assert st == P.PDHG_OK
    tr = sol.trace()
    agreed = compare_traces(tr, orc.trace)
    assert agreed >= 10 and sum(1 for r in tr[:agreed] if r["kind"] == P.PDHG_RESTART_TO_PDHG_STEP) >= 3
    for g, o in zip(tr[:agreed], orc.trace[:agreed]):
        assert g["omega"] == pytest.approx(o.omega, rel=LONG_RUN_OMEGA)
    if agreed == len(tr):
        assert done == orc.k
        assert_iterates_close(sol, orc, LONG_RUN_ITERATES)
    x, _, _ = sol.solution()
    assert float(tiny_lp.c @ x) == pytest.approx(tiny_lp.f_star, rel=1e-7)


def test_panel_layout_matches_oracle():
    """A Zipf-shaped LP with the long columns in panels and the one-entry
    columns numbered by row, as the large LP runs."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3)
    orc, sol = _pair(lp, engine=dict(primal_panels=1, panel_rows=256, long_row_min=32))
    orc.run(128)
    sol.iterate(128)
    assert compare_traces(sol.trace(), orc.trace) == 2
    assert_iterates_close(sol, orc, 1e-10)
    orc.run(1500 - 128, 1e-8)
    sol.iterate(1500 - 128, 1e-8)
    assert compare_traces(sol.trace(), orc.trace) >= 10


@pytest.mark.parametrize("prec", [P.PDHG_FP32, P.PDHG_MIXED])
def test_fp32_and_mixed_reach_the_optimum(tiny_lp, prec):
    tol = 1e-4 if prec == P.PDHG_FP32 else 1e-8  # FP32 alone: as far as FP32 rounding lets the tiny LP go
    with P.Solver.from_lp(tiny_lp, precision=prec, halpern=1, restart_scheme=1) as sol:
        st, done = sol.iterate(200_000, tol)
        assert st == P.PDHG_OK
        k = sol.kkt()
    assert k["rel_kkt"] <= tol
    assert k["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=30 * tol)


def test_option_checks(tiny_lp):
    for bad in (dict(restart_scheme=1), dict(restart_scheme=2, halpern=1),
                dict(restart_scheme=1, halpern=1, feas_polish=1), dict(restart_scheme=1, halpern=1, pid_kp=np.inf)):
        with pytest.raises(P.PDHGError) as ei:
            P.Solver.from_lp(tiny_lp, **bad)
        assert ei.value.status == P.PDHG_ERR_INVALID, bad
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny_lp, tiny_lp], halpern=1, restart_scheme=1)
