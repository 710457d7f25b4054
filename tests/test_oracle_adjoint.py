"""Pins for the oracle's reverse pass through unrolled PDHG iterations:
central finite differences of the oracle's forward pass (a different
computation than the reverse pass) and the dot-product identity of the
linearised map with the projection masks frozen."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen


def _setup(K=60, seed=0, primal_weight=False):
    lp = lpgen.tiny_lp(seed)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                   O.Options(restarts=False, primal_weight=primal_weight))
    xt = lpgen.x_target(lp, seed=7)
    return lp, orc, xt, K


@pytest.mark.parametrize("primal_weight", [False, True])
def test_adjoint_matches_central_differences(primal_weight):
    """primal_weight=True keeps omega at omega0 != 1 (no restarts, so no
    updates), so tau != sigma and a swapped step size fails."""
    lp, orc, xt, K = _setup(primal_weight=primal_weight)
    assert primal_weight == (abs(orc.tau - orc.sigma) > 1e-3 * orc.tau)
    xs, _ = O.unrolled_forward(orc, K)
    gxK = orc.d_c * xs[-1] - xt
    gc, gb = O.unrolled_adjoint(orc, K, gxK)
    rng = np.random.default_rng(3)
    h = 1e-6
    checked = 0
    for _ in range(20):
        dc, db = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
        nrm = np.sqrt(dc @ dc + db @ db)
        dc, db = dc / nrm, db / nrm
        # skip directions whose +-h perturbation changes a projection mask (a kink)
        xp, _ = O.unrolled_forward(orc, K, c=lp.c + h * dc, b=lp.b + h * db)
        xm, _ = O.unrolled_forward(orc, K, c=lp.c - h * dc, b=lp.b - h * db)
        if any(np.any((a > 0) != (bb > 0)) for a, bb in zip(xp, xm)):
            continue
        fd = (O.unrolled_loss(orc, K, xt, c=lp.c + h * dc, b=lp.b + h * db)
              - O.unrolled_loss(orc, K, xt, c=lp.c - h * dc, b=lp.b - h * db)) / (2 * h)
        ad = gc @ dc + gb @ db
        assert ad == pytest.approx(fd, rel=1e-5, abs=1e-9)
        checked += 1
    assert checked >= 15


def test_adjoint_dot_product_identity():
    """<J v, w> = <v, J^T w> for the Jacobian of x_K(c, b) with frozen masks:
    J v computed by forward differences of the linearised recursion."""
    lp, orc, xt, K = _setup(K=40)
    xs, _ = O.unrolled_forward(orc, K)
    rng = np.random.default_rng(5)
    dc, db = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
    w = rng.standard_normal(lp.n)
    # tangent recursion with the masks of the base trajectory
    dch, dbh = orc.d_c * dc, orc.d_r * db
    dx, dy = np.zeros(lp.n), np.zeros(lp.m)
    for k in range(K):
        du = dx - orc.tau * (dch - orc.AhT @ dy)
        dx1 = np.where(xs[k + 1] > 0, du, 0.0)
        dv = 2 * dx1 - dx
        dy = dy + orc.sigma * (dbh - orc.Ah @ dv)
        dx = dx1
    Jv = orc.d_c * dx
    gc, gb = O.unrolled_adjoint(orc, K, w)
    assert float(Jv @ w) == pytest.approx(float(gc @ dc + gb @ db), rel=1e-11)
