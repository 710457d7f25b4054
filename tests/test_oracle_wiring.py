"""Pins of the oracle's evaluation bookkeeping (which point each rule looks
at), against the rules' statements: the iterate after convergence is the
candidate, the primal weight after a restart uses the moves from the previous
restart point, the no-progress test compares with the previous evaluation's
candidate, and the snapshot schedules (periodic every 128 iterations;
Algorithm 1's target inclusive, also without restarts and tolerance)."""
import math

import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen


def _oracle(lp, **opts):
    return O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(**opts))


def test_converged_iterate_is_the_candidate():
    """Across LPs and tolerances, the iterate left after convergence has the
    rel_kkt the last evaluation recorded for its candidate (the average when
    the average was chosen); at least one case ends on the average."""
    averages = 0
    for seed in range(4):
        lp = lpgen.tiny_lp(seed)
        for tol in (1e-4, 1e-6, 1e-8):
            o = _oracle(lp)
            assert o.run(200000, tol)
            last = o.trace[-1]
            assert o.kkt_of(o.x, o.y)["rel_kkt"] == pytest.approx(last.rel_kkt, rel=1e-12)
            averages += last.candidate == O.RESTART_TO_AVERAGE
    assert averages >= 1


def test_primal_weight_after_the_first_restart():
    """From a cold start (restart point 0), the first restart with theta = 0.5
    sets omega = sqrt(omega0 * ||y_c|| / ||x_c||), (x_c, y_c) the restart point
    (scaled)."""
    lp = lpgen.tiny_lp(0)
    o = _oracle(lp)
    omega0 = o.omega
    while o.restart_count == 0:
        o.run(64)
    assert o.omega == pytest.approx(math.sqrt(omega0 * np.linalg.norm(o.y_r) / np.linalg.norm(o.x_r)), rel=1e-12)


def test_no_progress_test_compares_with_the_previous_candidate():
    """After an evaluation without a restart, the reference of the no-progress
    test is that evaluation's candidate."""
    lp = lpgen.tiny_lp(0)
    o = _oracle(lp)
    for _ in range(40):
        before = o.restart_count
        o.run(64)
        if o.restart_count == before:
            last = o.trace[-1]
            xc, yc = ((o.x_avg, o.y_avg) if last.candidate == O.RESTART_TO_AVERAGE else (o.x, o.y))
            assert o.n_prev == pytest.approx(o.scaled_norms(xc, yc), rel=1e-14)
            return
    pytest.fail("no evaluation without a restart")


def test_periodic_snapshots_every_128_iterations():
    lp = lpgen.tiny_lp(0)
    o = _oracle(lp, snapshot_every=128)
    o.run(640)
    assert [s["iteration"] for s in o.snapshots] == [128, 256, 384, 512, 640]


def test_algorithm1_target_is_inclusive_and_needs_no_tolerance():
    """Algorithm 1 fires at the first evaluation with maxresid <= target: with
    the target set to the first evaluation's value exactly, it fires there;
    it also fires in plain runs (no restarts, tol = 0)."""
    lp = lpgen.tiny_lp(0)
    probe = _oracle(lp)
    probe.run(64, 1e-300)
    r64 = probe.trace[0].rel_kkt
    o = _oracle(lp, eps_cross=r64)
    o.run(64)
    assert [s["iteration"] for s in o.snapshots] == [64]
    plain = _oracle(lp, restarts=False, primal_weight=False, eps_cross=1.0)
    plain.run(128)
    assert len(plain.snapshots) >= 1


def test_relative_difference_of_the_margin():
    """The margin's relative difference |a - b| / max(|a|, |b|), 0 for a = b = 0."""
    assert O._rel_gap(1.0, 2.0) == 0.5 and O._rel_gap(-3.0, 1.0) == pytest.approx(4.0 / 3.0) and O._rel_gap(0.0, 0.0) == 0.0


def test_decision_margin_sees_the_sufficient_decay_boundary():
    """The margin recorded with each evaluation (how close any of its
    comparisons came to a tie) is ~0 when the candidate's weighted error sits
    exactly on the sufficient-decay boundary (reference = 5 x candidate)."""
    lp = lpgen.tiny_lp(0)
    o = _oracle(lp)
    o.run(63)
    o.iterate_once()  # k = 64, before its evaluation
    n_cur = o.scaled_norms(o.x, o.y)
    n_avg = o.scaled_norms(o.x_avg, o.y_avg)
    cand = n_avg if O.choose_candidate(n_cur, n_avg, o.omega) == O.RESTART_TO_AVERAGE else n_cur
    o.n_restart = tuple(5.0 * v for v in cand)
    o.n_prev = tuple(10.0 * v for v in cand)
    o.evaluate(0.0)
    assert o.trace[-1].margin <= 1e-14
