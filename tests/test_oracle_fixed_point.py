"""Pins of the oracle's fixed-point residual restart scheme and PID primal
weight (Options.restart_scheme = 1; the cuPDLP+ line the paper's solver
follows, Section 4.1, which gives no formula, so the scheme is a reading).

Pinned against mathematics and hand-worked values, not against the code's own
formulas: the residual against a dense matrix form of the metric, zero at an
optimal pair and positive elsewhere; the PID step on dyadic cases worked by
hand and against PDLP's smoothing update, which it must equal with gains
(theta, 0, 0); two restarted steps on a 1x1 LP worked by hand (a restart moves
to the PDHG step T(z) and makes it the anchor); convergence of restarted runs
to the generator's closed-form optimum and to the vertex-enumerated optimum."""
import itertools
import math

import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen


def test_residual_equals_the_dense_metric_form(tiny_lp):
    """r(z)^2 = w^T M w with w = z - T(z) and M = [[I/tau, Ahat^T], [Ahat,
    I/sigma]] built as a dense matrix."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options())
    Ah = o.Ah.toarray()
    M = np.block([[np.eye(lp.n) / o.tau, Ah.T], [Ah, np.eye(lp.m) / o.sigma]])
    rng = np.random.default_rng(7)
    for _ in range(3):
        x, y = np.abs(rng.standard_normal(lp.n)), rng.standard_normal(lp.m)
        r, xt, yt = O.fixed_point_residual(o.Ah, o.AhT, o.bh, o.ch, x, y, o.tau, o.sigma)
        w = np.concatenate([x - xt, y - yt])
        assert r == pytest.approx(math.sqrt(w @ M @ w), rel=1e-12)
        assert r > 0


def test_residual_vanishes_at_an_optimal_pair(tiny_lp):
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(), x0=lp.x_star, y0=lp.y_star)
    r, _, _ = o.fixed_point_measure(o.x, o.y)
    r0, _, _ = o.fixed_point_measure(np.zeros(lp.n), np.zeros(lp.m))
    assert r <= 1e-13 * r0


def test_pid_step_dyadic_cases():
    pid = O.pid_primal_weight
    # proportional gain 1: one step balances omega dx with dy (omega' = dy / dx)
    w, integral, e = pid(3.0, 2.0, 8.0, 0.0, 0.0, 1.0, 0.0, 0.0)
    assert w == pytest.approx(4.0, rel=1e-15) and e == pytest.approx(math.log(0.75), rel=1e-15)
    # integral gain 1: omega 1, dx / dy = 2 twice -> 1/2, then 1/4 (the second
    # error is 0, but the integral keeps ln 2)
    w, integral, e = pid(1.0, 2.0, 1.0, 0.0, 0.0, 0.0, 1.0, 0.0)
    assert w == pytest.approx(0.5, rel=1e-15) and integral == pytest.approx(math.log(2.0), rel=1e-15)
    w, integral, e = pid(w, 2.0, 1.0, integral, e, 0.0, 1.0, 0.0)
    assert w == pytest.approx(0.25, rel=1e-15) and e == pytest.approx(0.0, abs=1e-15)
    # derivative gain 1: the first step sees e - 0 = ln 2 (1/2); the second,
    # dx / dy = 4, sees the same error ln 2 and leaves omega
    w, integral, e = pid(1.0, 2.0, 1.0, 0.0, 0.0, 0.0, 0.0, 1.0)
    assert w == pytest.approx(0.5, rel=1e-15)
    w, integral, e = pid(w, 4.0, 1.0, integral, e, 0.0, 0.0, 1.0)
    assert w == pytest.approx(0.5, rel=1e-15)
    # a move at or below 1e-10 leaves everything unchanged
    assert pid(2.0, 1e-11, 1.0, 0.3, 0.2, 0.99, 0.01, 0.0) == (2.0, 0.3, 0.2)
    assert pid(2.0, 1.0, 1e-10, 0.3, 0.2, 0.99, 0.01, 0.0) == (2.0, 0.3, 0.2)


def test_pid_with_gains_theta_0_0_is_pdlp_smoothing():
    rng = np.random.default_rng(11)
    for _ in range(20):
        omega, dx, dy, theta = np.exp(rng.normal(size=3)).tolist() + [float(rng.uniform(0.1, 0.9))]
        w, _, _ = O.pid_primal_weight(omega, dx, dy, 0.0, 0.0, theta, 0.0, 0.0)
        assert w == pytest.approx(O.primal_weight_update(omega, dx, dy, theta), rel=1e-13)


def test_hand_worked_restarts_1x1():
    """min x s.t. x = 1, x >= 0 with no scaling, omega = 1, tau = sigma = 0.9,
    reflected Halpern (rho = 1), an evaluation after every iteration and a
    restart at every evaluation (beta_art = 0):
      step 1 from z0 = (0, 0), t = 0, w = 1/2: T(z0) = (0, 0.9), z1 = (0, 0.9);
      evaluation: T(z1) = (max(0, -0.09), 0.9 + 0.9 (1 - 0)) = (0, 1.8),
        r(z1) = |0.9| / sqrt(0.9) = sqrt(0.9); restart to (0, 1.8), anchor too;
      step 2 from z = (0, 1.8), t = 0: T(z) = (max(0, 0.72), 1.8 + 0.9 (1 -
        1.44)) = (0.72, 1.404), z2 = 2 T(z) / 2 = (0.72, 1.404);
      evaluation: T(z2) = (max(0, 0.72 - 0.9 (1 - 1.404)), 1.404 + 0.9 (1 -
        (2 * 1.0836 - 0.72))) = (1.0836, 1.404 - 0.40248) = (1.0836, 1.00152)."""
    o = O.Oracle(1, 1, np.array([0, 1]), np.array([0]), np.array([1.0]), np.array([1.0]), np.array([1.0]),
                 O.Options(ruiz_iters=0, pock_chambolle=False, primal_weight=False, halpern=True, restart_scheme=1,
                           eval_every=1, beta_art=0.0))
    assert o.tau == pytest.approx(0.9, rel=1e-15)
    assert o.r_restart == pytest.approx(math.sqrt(0.81 / 0.9), rel=1e-14)  # r(z0): T(z0) - z0 = (0, 0.9)
    o.run(1)
    assert (float(o.x[0]), float(o.y[0])) == pytest.approx((0.0, 1.8), abs=1e-15)
    assert (float(o.x_r[0]), float(o.y_r[0])) == pytest.approx((0.0, 1.8), abs=1e-15)
    assert o.trace[-1].kind == O.RESTART_TO_PDHG_STEP and o.t == 0
    assert o.r_restart == pytest.approx(math.sqrt(0.9), rel=1e-14)
    o.run(1)
    assert (float(o.x[0]), float(o.y[0])) == pytest.approx((1.0836, 1.00152), rel=1e-13)
    assert o.restart_count == 2


def test_restarted_run_reaches_generator_optimum(tiny_lp):
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(halpern=True, restart_scheme=1))
    assert o.run(200_000, 1e-9)
    x, _, _ = o.solution()
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-7)
    assert np.linalg.norm(x - lp.x_star) <= 1e-6 * np.linalg.norm(lp.x_star)
    kinds = {r.kind for r in o.trace}
    assert O.RESTART_TO_PDHG_STEP in kinds and kinds <= {O.NO_RESTART, O.RESTART_TO_PDHG_STEP}
    assert len({round(r.omega, 12) for r in o.trace}) > 2  # the PID controller moved the weight


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
def test_reaches_vertex_enumeration_optimum(seed):
    lp = lpgen.generate(4, 9, seed, nnz_per_col=3, support=3)
    f_vert = _vertex_optimum(lp.dense(), lp.b, lp.c)
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(halpern=True, restart_scheme=1))
    assert o.run(2_000_000, 1e-10)
    x, _, _ = o.solution()
    assert float(lp.c @ x) == pytest.approx(f_vert, rel=1e-8, abs=1e-8)


def test_restart_rules_see_the_residual_not_the_kkt_error(tiny_lp):
    """With beta_suff = 1 the sufficient-decay rule restarts at the first
    evaluation exactly when r(z_64) <= r(z_0); the run's first decision must
    follow that comparison of residuals computed here from the definition."""
    lp = tiny_lp
    opt = O.Options(halpern=True, restart_scheme=1, beta_suff=1.0, beta_nec=0.0, beta_art=10.0)
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, opt)
    r0 = o.r_restart
    for _ in range(64):
        o.iterate_once()
    r64, _, _ = o.fixed_point_measure(o.x, o.y)
    o.evaluate(0.0)
    assert (o.trace[-1].kind == O.RESTART_TO_PDHG_STEP) == (r64 <= r0)
