"""The method's degenerate cases on the GPU against the oracle: LPs without an
optimum (primal infeasible, dual infeasible) run without faults or NaNs,
report NOT_CONVERGED, follow the oracle's diverging iterates, and their
iterate differences give the same infeasibility certificates; a zero-cost LP
and a zero right-hand side converge like the oracle."""
import numpy as np
import pytest

from paper_2510_24429_b300 import pdhg as P
from tests import degenerate_lps as D
from tests.gpu_helpers import TINY_PLAIN, assert_iterates_close, compare_traces, pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.mark.parametrize("make", [D.infeasible_2x2, D.unbounded_1x2, D.infeasible_tiny], ids=lambda f: f.__name__)
def test_plain_iterates_follow_the_oracle(make):
    lp = make()
    orc, sol = pair(lp, **TINY_PLAIN)
    with sol:
        orc.run(2000)
        assert sol.iterate(2000) == (P.PDHG_OK, 2000)
        assert_iterates_close(sol, orc, 1e-9)


def test_infeasible_lp_reports_not_converged_and_a_certificate():
    lp = D.infeasible_tiny()
    orc, sol = pair(lp)
    with sol:
        orc.run(2048, 1e-8)
        st, done = sol.iterate(2048, 1e-8)
        assert st == P.PDHG_ERR_NOT_CONVERGED and done == 2048
        assert compare_traces(sol.trace(), orc.trace) >= 10
        k = sol.kkt()
        assert all(np.isfinite(v) for v in k.values()) and k["rel_p"] > 1e-3
        _, y0, _ = sol.solution()
        sol.iterate(256)
        _, y1, _ = sol.solution()
    d = (y1 - y0) / np.linalg.norm(y1 - y0)
    assert float(lp.b @ d) > 0.5 and float(np.max(lp.dense.T @ d)) <= 1e-9


def test_unbounded_lp_runs_without_faults():
    """With restarts the primal weight collapses on this LP (the oracle's does
    too), so trajectories are too sensitive to compare point by point; x grows
    without bound along the ray (1, 1)/sqrt(2) and stays finite: NOT_CONVERGED."""
    lp = D.unbounded_1x2()
    with P.Solver.from_lp(lp) as sol:
        st, _ = sol.iterate(20000, 1e-8)
        assert st == P.PDHG_ERR_NOT_CONVERGED
        x0, y0, _ = sol.solution()
        sol.iterate(256)
        x1, y1, z1 = sol.solution()
        assert all(np.all(np.isfinite(a)) for a in (x1, y1, z1)) and np.linalg.norm(x1) > 1e6
    d = (x1 - x0) / np.linalg.norm(x1 - x0)
    np.testing.assert_allclose(d, np.array([1.0, 1.0]) / np.sqrt(2.0), atol=1e-6)


@pytest.mark.parametrize("make", [D.zero_objective_tiny, D.zero_rhs_tiny], ids=lambda f: f.__name__)
def test_degenerate_optima_converge_like_the_oracle(make):
    lp = make()
    orc, sol = pair(lp)
    with sol:
        assert orc.run(200000, 1e-9)
        st, done = sol.iterate(200000, 1e-9)
        assert st == P.PDHG_OK and abs(done - orc.k) <= 2 * 64
        k = sol.kkt()
        assert k["rel_kkt"] <= 1e-9
        if make is D.zero_rhs_tiny:
            assert np.linalg.norm(sol.solution()[0]) <= 1e-8


@pytest.mark.parametrize("engine", [dict(), dict(use_graphs=0), dict(persistent=1)], ids=["graphs", "direct", "loop"])
def test_overflow_in_the_iterates_is_reported(tiny_lp, engine):
    """Failure detection without a GPU fault: a finite warm start of 1.7e308
    overflows when it is scaled (x / D_c with D_c entries below 1) and in the
    extrapolation 2x' - x, and the evaluation that follows reports
    PDHG_ERR_NUMERIC; the context still answers queries afterwards."""
    lp = tiny_lp
    x0 = np.full(lp.n, 1.7e308)
    with P.Solver.from_lp(lp, x0=x0, **engine) as s:
        with pytest.raises(P.PDHGError) as ei:
            s.iterate(640, 1e-8)
        assert ei.value.status == P.PDHG_ERR_NUMERIC
        info = s.info()
        assert info["iterations"] <= 640
