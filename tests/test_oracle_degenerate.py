"""The oracle on the method's degenerate cases, pinned by the mathematics of
PDHG on LPs without optimal solutions (the differences of the iterates tend to
an infeasibility certificate) and by closed-form optima of degenerate LPs.

* Primal infeasible: the dual iterates grow along a Farkas certificate
  (A^T d <= 0, b^T d > 0); on the 2x2 example it is (-1, 1)/sqrt(2).
* Dual infeasible: the primal iterates grow along a ray (A d = 0, d >= 0,
  c^T d < 0); on the 1x2 example it is (1, 1)/sqrt(2).
* c = 0: the method converges to a feasible point with objective 0.
* b = 0, c > 0: the optimum is x = 0 (unique)."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from tests import degenerate_lps as D


def _run(lp, k, tol=0.0, **opts):
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(**opts))
    o.run(k, tol)
    return o


def _direction(o, k, part):
    """Unit direction of the change of the unscaled iterate over k more
    iterations."""
    x0, y0, _ = o.solution()
    o.run(k)
    x1, y1, _ = o.solution()
    d = (y1 - y0) if part == "y" else (x1 - x0)
    return d / np.linalg.norm(d)


@pytest.mark.parametrize("opts", [dict(restarts=False, primal_weight=False), dict()])
def test_infeasible_2x2_dual_iterates_follow_the_farkas_certificate(opts):
    lp = D.infeasible_2x2()
    o = _run(lp, 2000, **opts)
    d = _direction(o, 128, "y")
    np.testing.assert_allclose(d, np.array([-1.0, 1.0]) / np.sqrt(2.0), atol=1e-6)


def test_unbounded_1x2_primal_iterates_follow_the_ray():
    lp = D.unbounded_1x2()
    o = _run(lp, 2000, restarts=False, primal_weight=False)
    d = _direction(o, 128, "x")
    np.testing.assert_allclose(d, np.array([1.0, 1.0]) / np.sqrt(2.0), atol=1e-6)


@pytest.mark.parametrize("opts,bound", [(dict(restarts=False, primal_weight=False), 2e-3), (dict(), 1e-9)])
def test_infeasible_tiny_certificate_properties(opts, bound):
    """Without restarts the direction approaches the certificate slowly
    (max A^T d is 7.6e-4 after 4000 iterations, 2.0e-4 after 20000); with
    restarts it is exact to rounding."""
    lp = D.infeasible_tiny()
    o = _run(lp, 4000, **opts)
    d = _direction(o, 256, "y")
    assert float(lp.b @ d) > 0.5
    assert float(np.max(lp.dense.T @ d)) <= bound


def test_zero_objective_reaches_a_feasible_point():
    lp = D.zero_objective_tiny()
    o = _run(lp, 200000, 1e-9)
    assert o.done
    x, y, _ = o.solution()
    A = O.csr_matrix(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
    assert np.linalg.norm(lp.b - A @ x) <= 1e-9 * (1 + np.linalg.norm(lp.b))
    assert float(x.min()) >= 0.0
    assert abs(float(lp.b @ y)) <= 1e-8  # dual objective of a zero-cost LP is 0 at optimality


def test_zero_rhs_has_the_zero_optimum():
    lp = D.zero_rhs_tiny()
    o = _run(lp, 200000, 1e-10)
    assert o.done
    x, _, _ = o.solution()
    assert np.linalg.norm(x) <= 1e-8
