"""Pins of the oracle's reflected Halpern variant (the cuPDLP+ line the paper's
solver follows, Section 4.1).

Pinned against values and mathematics, not against the formula itself:
hand-worked steps on a 1x1 LP (weights, reflection, anchor); an optimal pair
is a fixed point; Halpern's rate on the fixed-point residual of a nonexpansive
map holds in the metric in which PDHG is firmly nonexpansive; restarted runs
reach the generator's closed-form optimum and the vertex-enumerated optimum."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen


def _metric_norm(o, dx, dy):
    """||(dx, dy)||_M with M = [[I/tau, Ahat^T], [Ahat, I/sigma]]: PDHG on this
    LP is a preconditioned proximal point step in M, so its map T is firmly
    nonexpansive in this norm when tau sigma ||Ahat||^2 < 1."""
    q = dx @ dx / o.tau + 2.0 * float(dy @ (o.Ah @ dx)) + dy @ dy / o.sigma
    return math.sqrt(max(q, 0.0))


def test_hand_worked_steps_1x1():
    """Exact steps on min x s.t. x = 1, x >= 0 (tests/golden/halpern_1x1.json):
    pins the weight schedule, the reflection and the anchor."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "halpern_1x1.json")) as f:
        g = json.load(f)
    for rho, key in ((1.0, "rho_1"), (0.0, "rho_0")):
        o = O.Oracle(1, 1, np.array([0, 1]), np.array([0]), np.array([1.0]), np.array([1.0]), np.array([1.0]),
                     O.Options(ruiz_iters=0, pock_chambolle=False, restarts=False, primal_weight=False, halpern=True,
                               halpern_reflect=rho))
        assert o.tau == pytest.approx(0.9, rel=1e-15) and o.sigma == pytest.approx(0.9, rel=1e-15)
        for xk, yk in g[key]:
            o.iterate_once()
            assert float(o.x[0]) == pytest.approx(xk, rel=1e-13, abs=1e-15)
            assert float(o.y[0]) == pytest.approx(yk, rel=1e-13, abs=1e-15)


def test_optimal_pair_is_a_fixed_point(tiny_lp):
    lp = tiny_lp
    for rho in (0.0, 0.5, 1.0):
        o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                     O.Options(halpern=True, halpern_reflect=rho, restarts=False, primal_weight=False),
                     x0=lp.x_star, y0=lp.y_star)
        x0, y0 = o.x.copy(), o.y.copy()
        for _ in range(64):
            o.iterate_once()
        assert np.linalg.norm(o.x - x0) <= 1e-13 * np.linalg.norm(x0)
        assert np.linalg.norm(o.y - y0) <= 1e-12 * np.linalg.norm(y0)


def test_metric_makes_the_pdhg_map_firmly_nonexpansive(tiny_lp):
    """Check of the metric used below: for two random points, the PDHG map
    satisfies ||Tu - Tv||_M^2 <= <Tu - Tv, u - v>_M (firm nonexpansiveness)."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                 O.Options(restarts=False, primal_weight=False))
    rng = np.random.default_rng(3)
    for _ in range(5):
        u = (rng.standard_normal(lp.n), rng.standard_normal(lp.m))
        v = (rng.standard_normal(lp.n), rng.standard_normal(lp.m))
        tu = O.pdhg_iteration(o.Ah, o.AhT, o.bh, o.ch, u[0], u[1], o.tau, o.sigma)
        tv = O.pdhg_iteration(o.Ah, o.AhT, o.bh, o.ch, v[0], v[1], o.tau, o.sigma)
        dtx, dty = tu[0] - tv[0], tu[2] - tv[2]
        dx, dy = u[0] - v[0], u[1] - v[1]
        inner = dtx @ dx / o.tau + float(dty @ (o.Ah @ dx)) + float(dy @ (o.Ah @ dtx)) + dty @ dy / o.sigma
        assert _metric_norm(o, dtx, dty) ** 2 <= inner * (1 + 1e-12) + 1e-12


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_halpern_rate_on_the_fixed_point_residual(tiny_lp, rho):
    """Halpern's iteration of a nonexpansive map S anchored at z0 satisfies
    ||z_k - S z_k|| <= 2 ||z0 - z*|| / (k + 1) (Lieder's bound). Here S =
    (1 + rho) T - rho I, nonexpansive in M because T is firmly nonexpansive,
    and ||z - S z|| = (1 + rho) ||z - T z||."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                 O.Options(halpern=True, halpern_reflect=rho, restarts=False, primal_weight=False))
    xs, ys = lp.x_star / o.d_c, lp.y_star / o.d_r  # a fixed point of T (scaled)
    d0 = _metric_norm(o, o.x - xs, o.y - ys)
    assert d0 > 0
    worst = 0.0
    for k in range(0, 2001):
        if k in (0, 1, 2, 5, 10, 50, 200, 1000, 2000):
            tx, _, ty = O.pdhg_iteration(o.Ah, o.AhT, o.bh, o.ch, o.x, o.y, o.tau, o.sigma)
            res = (1.0 + rho) * _metric_norm(o, o.x - tx, o.y - ty)
            bound = 2.0 * d0 / (k + 1)
            assert res <= bound * (1 + 1e-9), (k, res, bound)
            worst = max(worst, res / bound)
        o.iterate_once()
    # the residual does shrink (a map left at its anchor would not)
    assert worst > 1e-6


@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_restarted_halpern_reaches_generator_optimum(tiny_lp, rho):
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                 O.Options(halpern=True, halpern_reflect=rho))
    assert o.run(200_000, 1e-9)
    x, _, _ = o.solution()
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-7)
    assert np.linalg.norm(x - lp.x_star) <= 1e-6 * np.linalg.norm(lp.x_star)
    assert all(r.candidate == O.RESTART_TO_CURRENT for r in o.trace)  # no averages


def _vertex_optimum(A, b, c):
    m, n = A.shape
    best = math.inf
    for B in itertools.combinations(range(n), m):
        AB = A[:, B]
        if abs(np.linalg.det(AB)) < 1e-12:
            continue
        xB = np.linalg.solve(AB, b)
        if np.all(xB >= -1e-10):
            best = min(best, float(c[list(B)] @ xB))
    return best


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_halpern_reaches_vertex_enumeration_optimum(seed):
    lp = lpgen.generate(4, 9, seed, nnz_per_col=3, support=3)
    f_vert = _vertex_optimum(lp.dense(), lp.b, lp.c)
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(halpern=True))
    assert o.run(2_000_000, 1e-10)
    x, _, _ = o.solution()
    assert float(lp.c @ x) == pytest.approx(f_vert, rel=1e-8, abs=1e-8)
