"""Pins of the oracle's feasibility polishing (the PDLP variant described in
Section 5: PDHG iterations with a zero objective inside the main solve, to
reach primal feasibility; the dual counterpart zeroes the right-hand side).

Pinned against mathematics, not against the oracle's own formulas: a feasible
start is a fixed point of each phase; where A x = b, x >= 0 has exactly one
solution the primal phase reaches it (A^{-1} b by a dense solve); with b = 0 and
A nonsingular the dual phase's primal iterate goes to 0 (the only point of
A x = 0); phase results and polished solutions pass an independent check of
their residuals; the attempts follow the stated schedule."""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen


def _square_lp(k=12, seed=3):
    """A diagonally dominant k x k matrix (nonsingular, every row/col full), a
    positive x_pos, b = A x_pos, and c = A^T y0 + z0 with z0 > 0."""
    rng = np.random.default_rng(seed)
    A = rng.uniform(-0.3, 0.3, (k, k)) + np.diag(rng.uniform(2.0, 3.0, k))
    x_pos = rng.uniform(0.5, 2.0, k)
    b = A @ x_pos
    c = A.T @ rng.normal(size=k) + rng.uniform(0.5, 1.0, k)
    S = sp.csr_matrix(A)
    return k, S, A, x_pos, b, c


def _independent_rel(A, b, c, x, y):
    """rel_p, rel_d, rel_gap recomputed with dense numpy (Section 2's ratios)."""
    Ad = A.toarray() if sp.issparse(A) else A
    rp = np.linalg.norm(b - Ad @ x) / (1 + np.linalg.norm(b))
    rd = np.linalg.norm(np.maximum(0.0, Ad.T @ y - c)) / (1 + np.linalg.norm(c))
    cx, by = c @ x, b @ y
    return rp, rd, abs(cx - by) / (1 + abs(cx) + abs(by))


def test_feasible_start_is_a_fixed_point_of_each_phase(tiny_lp):
    """From (x*, 0) the zero-objective problem has A x* = b and no gradient,
    so the primal phase stays at x*; from (0, y*) the zero-right-hand-side
    problem has z* >= 0 and stays at (0, y*)."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(), x0=lp.x_star, y0=lp.y_star)
    xs, ys = o.x.copy(), o.y.copy()
    xp, yp, k, _ = o.feasibility_phase(xs, np.zeros(lp.m), "primal", 0.0, 256)
    assert k == 256
    assert np.linalg.norm(xp - xs) <= 1e-12 * np.linalg.norm(xs)
    assert np.linalg.norm(yp) <= 1e-12 * np.linalg.norm(ys)
    xd, yd, _, _ = o.feasibility_phase(np.zeros(lp.n), ys, "dual", 0.0, 256)
    assert np.linalg.norm(yd - ys) <= 1e-12 * np.linalg.norm(ys)
    assert np.linalg.norm(xd) <= 1e-12 * np.linalg.norm(xs)
    # the main solver is untouched by its phases
    assert np.array_equal(o.x, xs) and np.array_equal(o.y, ys) and o.k == 0


def test_primal_phase_reaches_the_only_feasible_point():
    k, S, A, x_pos, b, c = _square_lp()
    o = O.Oracle(k, k, S.indptr, S.indices, S.data, b, c, O.Options())
    x_start = np.full(k, 1.0) / o.d_c  # scaled start, unscaled all ones
    xp, _, iters, ok = o.feasibility_phase(x_start, np.zeros(k), "primal", 1e-12, 200000)
    assert ok and iters < 200000
    x_unscaled = o.d_c * xp
    np.testing.assert_allclose(x_unscaled, np.linalg.solve(A, b), rtol=1e-9)
    np.testing.assert_allclose(x_unscaled, x_pos, rtol=1e-9)


def test_dual_phase_primal_iterate_goes_to_zero():
    """With b = 0 the phase's primal problem is min c^T x, A x = 0, x >= 0,
    whose only feasible point is 0 when A is nonsingular; its y ends dual
    feasible (A^T y <= c up to the tolerance)."""
    k, S, A, _, b, c = _square_lp(seed=5)
    o = O.Oracle(k, k, S.indptr, S.indices, S.data, b, c, O.Options())
    y_start = np.random.default_rng(1).normal(size=k) * 5.0 / o.d_r
    xd, yd, iters, ok = o.feasibility_phase(np.zeros(k), y_start, "dual", 1e-11, 200000)
    assert ok
    y = o.d_r * yd
    assert np.linalg.norm(np.maximum(0.0, A.T @ y - c)) <= 1e-11 * (1 + np.linalg.norm(c))
    # x of the phase: PDHG iterate of a problem whose primal optimum is 0
    assert np.linalg.norm(o.d_c * xd) <= 1e-6


def test_polished_solutions_pass_an_independent_check():
    """Main solves with polishing (loose gap tolerance): whenever an attempt
    succeeds the returned pair meets rel_p, rel_d <= tol and rel_gap <= gap_tol
    by a dense recomputation, and the objective is close to the generator's
    known optimum."""
    tol, gtol = 1e-8, 1e-4
    hit = 0
    for lp in (lpgen.tiny_lp(0), lpgen.generate(2000, 5000, 1, nnz_per_col=5, support=0.3)):
        o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(feas_polish=True, gap_tol=gtol))
        assert o.run(100000, tol)
        x, y, _ = o.solution()
        rp, rd, rg = _independent_rel(o.A, lp.b, lp.c, x, y)
        assert rp <= tol and rd <= tol and rg <= gtol
        assert abs(lp.c @ x - lp.f_star) <= 10 * gtol * (1 + abs(lp.f_star))
        hit += any(r["dual_ok"] and r["rel_kkt"] < math.inf and r["rel_gap"] <= gtol for r in o.polish_log)
    assert hit >= 1  # at least one solve ended by polishing


def test_attempt_schedule_follows_its_rules():
    """Attempts come at evaluations whose candidate has rel_gap <= gap_tol and
    did not pass the test, the first one at the first such evaluation and each
    later one only once the iteration count has at least doubled; every phase
    runs at most ceil(k / (polish_div * eval_every)) evaluation periods."""
    lp = lpgen.generate(20000, 60000, 0, nnz_per_col=None, zipf=(1.5, 10000, 600000), val_range=(0.1, 10.0),
                        support=0.3)
    tol, gtol = 1e-6, 1e-4
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                 O.Options(feas_polish=True, gap_tol=gtol, polish_div=8))
    o.run(4000, tol)
    expected, nxt = [], 0
    for r in o.trace:
        if r.rel_gap <= gtol and r.iteration >= nxt:
            expected.append(r.iteration)
            nxt = 2 * r.iteration
    got = [r["iteration"] for r in o.polish_log]
    assert got == expected and len(got) >= 2
    for r in o.polish_log:
        budget = 64 * max(1, -(-r["iteration"] // 512))
        assert r["budget"] == budget
        assert r["primal_iters"] <= budget and r["dual_iters"] <= budget
        assert r["primal_iters"] % 64 == 0 and r["dual_iters"] % 64 == 0
    assert o.polish_log[0]["budget"] == 64 * math.ceil(o.polish_log[0]["iteration"] / 512)
    # the dual phase runs only after a successful primal phase
    assert all(r["dual_iters"] == 0 for r in o.polish_log if not r["primal_ok"])


def test_a_pair_with_a_large_gap_does_not_end_the_solve():
    """On the Zipf-shaped LP the attempt at 6400 iterations reaches both
    feasibility targets but its pair's relative gap is above gap_tol: the
    solve goes on; every accepted pair has rel_gap <= gap_tol."""
    lp = lpgen.generate(20000, 60000, 0, nnz_per_col=None, zipf=(1.5, 10000, 600000), val_range=(0.1, 10.0),
                        support=0.3)
    tol, gtol = 1e-6, 1e-4
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                 O.Options(feas_polish=True, gap_tol=gtol))
    o.run(6464, tol)
    both = [r for r in o.polish_log if r["primal_ok"] and r["dual_ok"]]
    assert any(r["rel_gap"] > gtol for r in both)
    for r in both:
        ended_here = o.done and o.k == r["iteration"]
        assert ended_here == (r["rel_gap"] <= gtol)


def test_gap_tolerance_equal_to_tol_is_the_single_eps_test(tiny_lp):
    """gap_tol = tol (or 0) gives the same run as Section 2's single-eps test
    (max of the three ratios <= eps)."""
    lp = tiny_lp
    runs = []
    for g in (0.0, 1e-7):
        o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(gap_tol=g))
        o.run(100000, 1e-7)
        runs.append((o.k, o.x.copy()))
        last = o.trace[-1]
        assert last.rel_kkt <= 1e-7 and all(r.rel_kkt > 1e-7 for r in o.trace[:-1])
    assert runs[0][0] == runs[1][0] and np.array_equal(runs[0][1], runs[1][1])


def test_phase_stops_on_its_own_measure_and_starts_its_own_restart_reference(tiny_lp):
    """At (x*, y*) the primal phase's problem (c = 0) is primal feasible
    (rel_p = 0) but not dual optimal (A^T y* != 0), and the dual phase's
    problem (b = 0) dual feasible but not primal (A x* != 0): each phase must
    stop there, on rel_p resp. rel_d alone. Each phase's first restart
    reference is its own start, not the main solver's."""
    lp = tiny_lp
    o = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options())
    xs, ys = lp.x_star / o.d_c, lp.y_star / o.d_r
    for kind in ("primal", "dual"):
        sub = o.phase_solver(xs, ys, kind)
        full = sub.kkt_of(sub.x, sub.y)
        assert full["rel_kkt"] > 1e-3 and full["rel_p" if kind == "primal" else "rel_d"] <= 1e-12
        assert sub.evaluate(1e-8)
        start = o.phase_solver(xs, np.zeros(lp.m), kind)
        assert start.n_restart == start.scaled_norms(xs, np.zeros(lp.m)) != o.n_restart


def test_polished_pair_is_judged_with_the_gap_tolerance():
    """A polishing attempt from a primal-feasible x_c and a dual-feasible y_c
    (each a fixed point of its phase) returns the pair (x_c, y_c), whose
    relative gap is 5/6 on the 2x3 LP (x_c = (3, 0, 2), y_c = 0). The pair ends
    the solve exactly when gap_tol admits 5/6 (Section 2's test with a separate
    gap tolerance; the phases are Section 5's polishing)."""
    A = sp.csr_matrix(np.array([[1.0, 2.0, 0.0], [0.0, 1.0, 1.0]]))
    b, c = np.array([3.0, 2.0]), np.array([1.0, 1.0, 1.0])
    x_c, y_c = np.array([3.0, 0.0, 2.0]), np.zeros(2)
    for gap_tol, accepted in ((0.9, True), (0.8, False)):
        o = O.Oracle(2, 3, A.indptr, A.indices, A.data, b, c, O.Options(gap_tol=gap_tol, feas_polish=True))
        pair = o.feasibility_polish(x_c / o.d_c, y_c / o.d_r, 1e-9)
        rec = o.polish_log[-1]
        assert rec["primal_ok"] and rec["dual_ok"] and rec["rel_gap"] == pytest.approx(5 / 6, rel=1e-9)
        assert (pair is not None) is accepted, gap_tol
        if accepted:
            xp, yd = pair
            assert np.allclose(o.d_c * xp, x_c, rtol=0, atol=1e-12) and np.allclose(o.d_r * yd, y_c, atol=1e-12)
