"""Pins for the FP64 oracle: each test checks it against something other than
itself (hand-worked values, closed forms, brute force, a library solver, or a
property the mathematics fixes)."""
import itertools
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _expr(s):
    return float(eval(s, {"sqrt": math.sqrt}))


def _golden_2x3():
    with open(os.path.join(GOLDEN, "lp2x3_step_kkt.json")) as f:
        return json.load(f)


def test_kkt_hand_computed_2x3():
    g = _golden_2x3()
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    b, c = np.array(g["b"], float), np.array(g["c"], float)
    for point in ("kkt_point", "kkt_point_negative_residual", "kkt_point_negative_x",
                  "kkt_point_negative_x_with_slack"):
        p = g[point]
        info = O.kkt(A, b, c, np.array(p["x"], float), np.array(p["y"], float))
        for key, expr in p["expect"].items():
            assert info[key] == pytest.approx(_expr(expr), rel=1e-15, abs=1e-15), (point, key)


def test_kkt_with_a_given_z_2x3():
    """With z given (here 0) the dual residual A^T y + z - c can be negative:
    its infinity norm is the largest magnitude."""
    g = _golden_2x3()
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    b, c = np.array(g["b"], float), np.array(g["c"], float)
    p = g["kkt_point_given_z"]
    info = O.kkt(A, b, c, np.array(p["x"], float), np.array(p["y"], float), np.array(p["z"], float))
    for key, expr in p["expect"].items():
        assert info[key] == pytest.approx(_expr(expr), rel=1e-15, abs=1e-15), key


def test_power_iteration_two_steps_closed_form():
    """On diag(2, 1) from the start w = 0.5 + u (u from the first two
    SplitMix64 outputs, tests/golden/splitmix64_seed0.json): the second
    estimate is ||A v1|| with v1 along A^T A w = (4 w1, w2), i.e.
    sqrt(64 w1^2 + w2^2) / sqrt(16 w1^2 + w2^2)."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.json")) as f:
        ref = [int(h, 16) for h in json.load(f)["outputs_hex"]]
    w1, w2 = (0.5 + (r >> 11) * 2.0 ** -53 for r in ref[:2])
    Ah = sp.csr_matrix(np.diag([2.0, 1.0]))
    assert O.power_norm(Ah, 1) == pytest.approx(math.sqrt(4 * w1 * w1 + w2 * w2) / math.hypot(w1, w2), rel=1e-15)
    assert O.power_norm(Ah, 2) == pytest.approx(math.sqrt(64 * w1 * w1 + w2 * w2) / math.hypot(4 * w1, w2),
                                                rel=1e-15)


def test_scaled_measures_of_the_restart_rules_2x3():
    """Without scaling (no Ruiz or Pock-Chambolle passes) the restart rules'
    measures (||r_P||, ||r_D||, |c^T x - b^T y|) equal the hand-computed
    unscaled ones."""
    g = _golden_2x3()
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    b, c = np.array(g["b"], float), np.array(g["c"], float)
    o = O.Oracle(2, 3, A.indptr, A.indices, A.data, b, c, O.Options(ruiz_iters=0, pock_chambolle=False))
    for point in ("kkt_point", "kkt_point_negative_residual"):
        p = g[point]
        e = p["expect"]
        got = o.scaled_norms(np.array(p["x"], float), np.array(p["y"], float))
        want = (_expr(e["rp_norm2"]), _expr(e["rd_norm2"]), _expr(e["gap"]))
        assert got == pytest.approx(want, rel=1e-15, abs=1e-15), point


def test_step_hand_computed_2x3():
    g = _golden_2x3()
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    AT = sp.csr_matrix(A.T)
    b, c = np.array(g["b"], float), np.array(g["c"], float)
    for st in g["steps"]:
        x_new, xbar, y_new = O.pdhg_iteration(A, AT, b, c, np.array(st["x"], float), np.array(st["y"], float),
                                              st["tau"], st["sigma"])
        np.testing.assert_array_equal(x_new, np.array(st["x_new"], float))
        np.testing.assert_array_equal(xbar, np.array(st["xbar"], float))
        np.testing.assert_array_equal(y_new, np.array(st["y_new"], float))


def test_kkt_zero_at_generator_optimum(tiny_lp):
    A = O.csr_matrix(tiny_lp.m, tiny_lp.n, tiny_lp.row_ptr, tiny_lp.col_idx, tiny_lp.val)
    info = O.kkt(A, tiny_lp.b, tiny_lp.c, tiny_lp.x_star, tiny_lp.y_star, tiny_lp.z_star)
    assert info["rel_kkt"] < 1e-14
    assert info["complementarity"] == 0.0
    # the generator's z* is the oracle's dual slack at y*
    np.testing.assert_allclose(O.dual_slack(A, tiny_lp.c, tiny_lp.y_star), tiny_lp.z_star, atol=1e-13)


def test_fixed_point_of_pdhg_map(tiny_lp):
    """An optimal pair is left unchanged by the PDHG map (in scaled space)."""
    lp = tiny_lp
    for pc in (False, True):
        o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                     O.Options(pock_chambolle=pc), x0=lp.x_star, y0=lp.y_star)
        x1, xbar, y1 = O.pdhg_iteration(o.Ah, o.AhT, o.bh, o.ch, o.x, o.y, o.tau, o.sigma)
        assert np.linalg.norm(x1 - o.x) <= 1e-14 * np.linalg.norm(o.x)
        assert np.linalg.norm(xbar - o.x) <= 1e-14 * np.linalg.norm(o.x)
        assert np.linalg.norm(y1 - o.y) <= 1e-13 * np.linalg.norm(o.y)
        # a non-optimal point moves
        x2, _, y2 = O.pdhg_iteration(o.Ah, o.AhT, o.bh, o.ch, o.x * 1.01, o.y, o.tau, o.sigma)
        assert np.linalg.norm(y2 - o.y) > 1e-6


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


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("restarts", [False, True])
def test_converges_to_vertex_enumeration_optimum(seed, restarts):
    lp = lpgen.generate(4, 9, seed, nnz_per_col=3, support=3)
    A = lp.dense()
    f_vert = _vertex_optimum(A, lp.b, lp.c)
    assert f_vert == pytest.approx(lp.f_star, rel=1e-10, abs=1e-10)
    opt = O.Options(restarts=restarts, primal_weight=restarts, pock_chambolle=restarts)
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, opt)
    assert o.run(2_000_000, 1e-10)
    x, y, z = o.solution()
    assert float(lp.c @ x) == pytest.approx(f_vert, rel=1e-8, abs=1e-8)


@pytest.mark.parametrize("restarts", [False, True])
def test_tiny_lp_reaches_generator_optimum(tiny_lp, restarts):
    lp = tiny_lp
    opt = O.Options(restarts=restarts, primal_weight=restarts, pock_chambolle=restarts)
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, opt)
    assert o.run(200_000, 1e-9)
    x, y, z = o.solution()
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-7)
    # x* is unique (columns on its support are independent), so x itself converges
    A = lp.dense()
    assert np.linalg.matrix_rank(A[:, lp.x_star > 0]) == int((lp.x_star > 0).sum())
    assert np.linalg.norm(x - lp.x_star) <= 1e-6 * np.linalg.norm(lp.x_star)


def test_tiny_lp_matches_highs(tiny_lp):
    from scipy.optimize import linprog

    lp = tiny_lp
    res = linprog(lp.c, A_eq=lp.dense(), b_eq=lp.b, bounds=(0, None), method="highs")
    assert res.status == 0
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options())
    assert o.run(200_000, 1e-9)
    x, _, _ = o.solution()
    assert float(lp.c @ x) == pytest.approx(res.fun, rel=1e-7)


def test_ruiz_equilibrates(tiny_lp):
    A = O.csr_matrix(tiny_lp.m, tiny_lp.n, tiny_lp.row_ptr, tiny_lp.col_idx, tiny_lp.val)
    for iters, tol in ((10, 2e-2), (40, 1e-8)):
        Ah, d_r, d_c = O.ruiz_scaling(A, iters)
        absA = abs(Ah)
        rmax = np.asarray(absA.max(axis=1).todense()).ravel()
        cmax = np.asarray(absA.max(axis=0).todense()).ravel()
        assert np.max(np.abs(rmax - 1)) < tol and np.max(np.abs(cmax - 1)) < tol
        # Ahat = D_r A D_c
        np.testing.assert_allclose((sp.diags(d_r) @ A @ sp.diags(d_c)).toarray(), Ah.toarray(), rtol=1e-14, atol=0)


def test_ruiz_closed_forms():
    # diagonal matrix: one pass maps it to the identity exactly
    d = np.array([4.0, 0.25, 16.0, 1.0])
    Ah, d_r, d_c = O.ruiz_scaling(sp.csr_matrix(np.diag(d)), 1)
    np.testing.assert_array_equal(Ah.toarray(), np.eye(4))
    np.testing.assert_array_equal(d_r, 1 / np.sqrt(d))
    # empty row and column keep factor 1
    M = sp.csr_matrix(np.array([[2.0, 0.0], [0.0, 0.0]]))
    _, d_r, d_c = O.ruiz_scaling(M, 3)
    assert d_r[1] == 1.0 and d_c[1] == 1.0


def test_pock_chambolle_norm_bound(tiny_lp):
    """With alpha = 1, ||D_r A D_c||_2 <= 1 (Schur test), with equality for an
    all-ones block."""
    A = O.csr_matrix(tiny_lp.m, tiny_lp.n, tiny_lp.row_ptr, tiny_lp.col_idx, tiny_lp.val)
    Ah, r, s = O.pock_chambolle_scaling(A, 1.0)
    assert np.linalg.norm(Ah.toarray(), 2) <= 1 + 1e-12
    J = sp.csr_matrix(np.ones((3, 5)))
    Jh, _, _ = O.pock_chambolle_scaling(J, 1.0)
    np.testing.assert_allclose(Jh.toarray(), np.full((3, 5), 1 / math.sqrt(15)), rtol=1e-15)
    assert np.linalg.norm(Jh.toarray(), 2) == pytest.approx(1.0, rel=1e-14)


def test_pock_chambolle_other_alphas():
    """Closed forms on A = [[2, 0], [1, 3]]: alpha = 0 gives row factors
    1/sqrt(#entries) and column factors 1/sqrt(sum a^2); alpha = 2 the other
    way round."""
    A = sp.csr_matrix(np.array([[2.0, 0.0], [1.0, 3.0]]))
    _, r, s = O.pock_chambolle_scaling(A, 0.0)
    np.testing.assert_allclose(r, [1.0, 1 / math.sqrt(2.0)], rtol=1e-15)
    np.testing.assert_allclose(s, [1 / math.sqrt(5.0), 1 / 3.0], rtol=1e-15)
    _, r, s = O.pock_chambolle_scaling(A, 2.0)
    np.testing.assert_allclose(r, [1 / 2.0, 1 / math.sqrt(10.0)], rtol=1e-15)
    np.testing.assert_allclose(s, [1 / math.sqrt(2.0), 1.0], rtol=1e-15)


def test_power_iteration_vs_svd(tiny_lp):
    A = O.csr_matrix(tiny_lp.m, tiny_lp.n, tiny_lp.row_ptr, tiny_lp.col_idx, tiny_lp.val)
    Ah, _, _ = O.ruiz_scaling(A, 10)
    s_max = np.linalg.norm(Ah.toarray(), 2)
    assert O.power_norm(Ah, 20000) == pytest.approx(s_max, rel=1e-8)
    est = O.power_norm(Ah, 100)
    assert est <= s_max * (1 + 1e-12) and est >= 0.95 * s_max  # Rayleigh quotient never overshoots


def test_power_iteration_when_ahat_maps_ones_to_zero():
    """Ahat = [1, -1] maps the all-ones vector to zero, so a power iteration
    started there estimates 0; the estimate must be sqrt(2) (closed form)."""
    Ah = sp.csr_matrix(np.array([[1.0, -1.0]]))
    assert O.power_norm(Ah, 3) == pytest.approx(math.sqrt(2.0), rel=1e-15)
    Ah = sp.csr_matrix(np.array([[1.0, -1.0, 0.0], [0.0, 1.0, -1.0], [-1.0, 0.0, 1.0]]))  # a cycle's incidence
    assert O.power_norm(Ah, 200) == pytest.approx(math.sqrt(3.0), rel=1e-12)


def test_power_start_is_the_published_splitmix64():
    """The start vector's generator against the published SplitMix64 outputs
    (tests/golden/splitmix64_seed0.json), and the vector's definition."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.json")) as f:
        ref = [int(h, 16) for h in json.load(f)["outputs_hex"]]
    got = O.splitmix64(np.arange(1, len(ref) + 1, dtype=np.uint64))
    assert [int(v) for v in got] == ref
    v = O.power_start(4)
    w = 0.5 + np.array([r >> 11 for r in ref], dtype=np.float64) * 2.0 ** -53
    np.testing.assert_allclose(v, w / np.linalg.norm(w), rtol=1e-15)


def test_restart_rules_hand_cases():
    opt = O.Options()
    # sufficient decay (boundary inclusive; no progress test involved: 0.2 < 0.3)
    assert O.restart_decision(0.2, 1.0, 0.1, 1, 100, opt)
    assert O.restart_decision(0.2, 1.0, 0.3, 1, 100, opt)
    assert O.restart_decision(0.1, 1.0, 0.05, 1, 100, opt)
    # necessary decay and no progress since the previous evaluation
    assert O.restart_decision(0.5, 1.0, 0.4, 1, 100, opt)
    # necessary decay but still progressing -> no restart (equal counts as progressing)
    assert not O.restart_decision(0.5, 1.0, 0.6, 1, 100, opt)
    assert not O.restart_decision(0.5, 1.0, 0.5, 1, 100, opt)
    # no decay at all
    assert not O.restart_decision(0.9, 1.0, 0.5, 1, 100, opt)
    # artificial: t >= 0.36 k (boundary inclusive)
    assert O.restart_decision(0.9, 1.0, 0.5, 36, 100, opt)
    assert not O.restart_decision(0.9, 1.0, 0.5, 35, 100, opt)
    # candidate choice: strictly smaller weighted error wins, ties go to the current iterate
    assert O.choose_candidate((1, 1, 1), (1, 1, 1), 2.0) == O.RESTART_TO_CURRENT
    assert O.choose_candidate((1, 1, 1), (1, 1, 0.5), 2.0) == O.RESTART_TO_AVERAGE
    assert O.weighted_kkt((3.0, 4.0, 0.0), 1.0) == 5.0
    assert O.weighted_kkt((1.0, 1.0, 1.0), 4.0) == pytest.approx(math.sqrt(5.25), rel=1e-16)
    assert O.weighted_kkt((3.0, 4.0, 0.0), 4.0) == pytest.approx(math.sqrt(40.0), rel=1e-16)  # 4*9 + 16/4
    # primal weight: geometric smoothing of dy/dx
    assert O.primal_weight_update(1.0, 1.0, 4.0, 0.5) == pytest.approx(2.0, rel=1e-15)
    assert O.primal_weight_update(4.0, 1.0, 4.0, 0.5) == pytest.approx(4.0, rel=1e-15)
    assert O.primal_weight_update(3.0, 1e-11, 4.0, 0.5) == 3.0
    # theta weighs the new ratio: exp(0.25 ln 4 + 0.75 ln 1) = sqrt(2)
    assert O.primal_weight_update(1.0, 1.0, 4.0, 0.25) == pytest.approx(math.sqrt(2.0), rel=1e-15)


def test_average_is_mean_of_iterates_since_restart(tiny_lp):
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options())
    hist_x, hist_y = [], []
    for _ in range(300):
        restarts_before = o.restart_count
        o.iterate_once()
        hist_x.append(o.x.copy())
        hist_y.append(o.y.copy())
        if o.k % o.opt.eval_every == 0:
            # check before the evaluation can reset the sums
            np.testing.assert_allclose(o.x_avg, np.mean(hist_x[-o.t:], axis=0), rtol=1e-12, atol=1e-15)
            np.testing.assert_allclose(o.y_avg, np.mean(hist_y[-o.t:], axis=0), rtol=1e-12, atol=1e-15)
            o.evaluate(0.0)
            if o.restart_count > restarts_before:
                hist_x, hist_y = [], []
    assert o.restart_count >= 1


def test_algorithm1_snapshot_schedule(tiny_lp):
    """Snapshots fire at the first evaluation with maxresid <= eps_target, and
    eps_target then shrinks tenfold (Algorithm 1, Section 3.1)."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(eps_cross=1e-2, eps_factor=0.1))
    assert o.run(200_000, 1e-7)
    thresholds = [1e-2 * 0.1 ** j for j in range(len(o.snapshots))]
    assert len(o.snapshots) >= 4
    recs = {r.iteration: r for r in o.trace}
    prev_iter = 0
    for snap, thr in zip(o.snapshots, thresholds):
        assert snap["rel_kkt"] <= thr
        # no earlier evaluation since the previous snapshot met this threshold
        earlier = [r for it, r in recs.items() if prev_iter < it < snap["iteration"]]
        assert all(r.rel_kkt > thr for r in earlier)
        prev_iter = snap["iteration"]
        # the snapshot is the unscaled (x, y, z) with z the dual slack of y
        A = O.csr_matrix(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
        assert O.kkt(A, lp.b, lp.c, snap["x"], snap["y"], snap["z"])["rel_kkt"] == pytest.approx(snap["rel_kkt"], rel=1e-12)


def test_separate_gap_tolerance_decides_termination():
    """Section 2's termination test with its own gap tolerance, on a pair that is
    primal feasible (A x = b, x >= 0) and dual feasible (A^T y <= c) but not
    optimal: x = (3, 0, 2), y = 0 on the 2x3 LP, so rel_p = rel_d = 0 and
    rel_gap = |5 - 0| / (1 + 5 + 0) = 5/6. The evaluation of this starting point
    accepts it exactly when the gap tolerance admits 5/6."""
    g = _golden_2x3()
    A = sp.csr_matrix(np.array(g["A"], dtype=float))
    b, c = np.array(g["b"], float), np.array(g["c"], float)
    x0, y0 = np.array([3.0, 0.0, 2.0]), np.zeros(2)
    assert np.array_equal(A @ x0, b) and np.all(A.T @ y0 <= c)
    for gap_tol, accepted in ((0.9, True), (5 / 6 + 1e-9, True), (0.8, False), (0.0, False)):
        o = O.Oracle(2, 3, A.indptr, A.indices, A.data, b, c, O.Options(restarts=False, gap_tol=gap_tol),
                     x0=x0, y0=y0)
        kk = o.kkt_of(o.x, o.y)
        assert kk["rel_p"] <= 1e-15 and kk["rel_d"] == 0.0 and kk["rel_gap"] == pytest.approx(5 / 6, rel=1e-15)
        assert o.evaluate(1e-9) is accepted, gap_tol
