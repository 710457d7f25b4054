"""FP64 CPU oracle for the PDHG hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product imports this module: only the
tests, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import or run it. It shares no code with
the CUDA path; the only common input is the seeded generator, which holds no
step of the method.

What it computes, with the passage each part follows
-----------------------------------------------------
* The LP pair ``min c^T x, Ax = b, x >= 0`` / ``max b^T y, A^T y + z = c,
  z >= 0`` and the residuals ``r_P = b - A x``, ``r_D = A^T y + z - c``
  (Section 2, "Background"); optimality = zero residuals, ``x, z >= 0`` and zero
  gap ``c^T x - b^T y`` (equivalently ``x^T z = 0``) (Section 2).
* The relative termination test on 2-norms, ``||r_P|| <= eps (1 + ||b||)``,
  ``||r_D|| <= eps (1 + ||c||)``, ``|c^T x - b^T y| <= eps (1 + |c^T x| + |b^T y|)``
  (Section 2). ``rel_kkt`` is the largest of the three ratios; it is the
  "maxresid" that drives the snapshot schedule of Algorithm 1 (Section 3.1).
* The PDHG iteration itself. The paper only says that its PDHG follows the
  PDLP / cuPDLP+ line of work (Section 1, Section 4.1) and gives no formula, so
  the iteration is the standard PDLP-style one, stated here in the notation of
  the paper's LP:

    x'   = max(0, x - tau (c - A^T y))
    xbar = 2 x' - x
    y'   = y + sigma (b - A xbar)

  on the diagonally scaled problem ``Ahat = D_r A D_c``, ``bhat = D_r b``,
  ``chat = D_c c`` (Ruiz equilibration followed by Pock-Chambolle scaling),
  with ``tau = eta / omega``, ``sigma = eta * omega``, ``eta = 0.9 / ||Ahat||_2``
  (power iteration), primal weight ``omega``, uniform averages of the iterates
  since the last restart, and KKT-error adaptive restarts. Every choice the
  paper leaves open is a documented reading (see ``Options``).
* The reflected Halpern variant of that iteration, from the cuPDLP+ line the
  paper's solver follows (Section 4.1; formula not given in the paper, so a
  reading): ``z <- w ((1 + rho) T(z) - rho z) + (1 - w) z_r`` with ``T`` the map
  above, ``w = (t + 1) / (t + 2)``, ``t`` the iterations since the last restart
  and ``z_r`` the last restart point; the current iterate is the only restart
  candidate (no averages).
* Feasibility polishing (Section 5 describes it as periodically running PDHG
  with a zero objective inside the main solve to reach primal feasibility; the
  dual counterpart zeroes the right-hand side). The rules of when and for how
  long are readings, listed at ``Options.feas_polish``.
* Algorithm 1's snapshot schedule: a snapshot of the current solution each time
  ``rel_kkt`` falls to ``eps_target``, after which ``eps_target`` shrinks by
  ``eps_factor`` (0.1 in the paper).

Pins (see the tests): vertex enumeration on tiny LPs, the generator's known
optimum, the fixed-point property of the PDHG map at an optimal pair, a
hand-computed step and KKT on a 2x3 LP, Ruiz/Pock-Chambolle invariants, power
iteration against a dense SVD, and an exact replay of the restart rules on
hand-made KKT sequences. The Halpern variant: the fixed point, the reduction
to the PDHG map at w = 1, rho = 0, and Halpern's O(1/k) bound on the
fixed-point residual in the PDHG metric. Feasibility polishing: a feasible
start is a fixed point of each phase, the primal phase reaches A^{-1} b where
that is the only feasible point, the dual phase's primal iterate goes to 0,
the phase results meet their feasibility tolerance, and the schedule of
attempts follows its rules.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

# restart kinds recorded in the trace
NO_RESTART, RESTART_TO_CURRENT, RESTART_TO_AVERAGE, RESTART_TO_PDHG_STEP = 0, 1, 2, 3


@dataclasses.dataclass
class Options:
    """Knobs of the method. Defaults are the large-LP configuration.

    Readings of points the paper leaves open:
      * ``ruiz_iters``/``pock_chambolle``: 10 Ruiz passes then one
        Pock-Chambolle pass with alpha = 1.
      * ``power_iters``: a fixed number of power iterations on Ahat^T Ahat,
        started from a fixed pseudo-random vector (``power_start``), so that
        every implementation computes the same estimate.
      * ``step_factor``: eta = step_factor / ||Ahat||_2.
      * ``restarts``/``primal_weight`` off gives plain fixed-step PDHG with
        omega = 1 (the tiny-LP configuration).
      * restart thresholds (beta_suff, beta_nec, beta_art) and the primal-weight
        smoothing theta follow PDLP's published defaults.
    """

    ruiz_iters: int = 10
    pock_chambolle: bool = True
    pc_alpha: float = 1.0
    power_iters: int = 100
    step_factor: float = 0.9
    restarts: bool = True
    primal_weight: bool = True
    eval_every: int = 64
    beta_suff: float = 0.2
    beta_nec: float = 0.8
    beta_art: float = 0.36
    theta: float = 0.5
    eps_cross: float = 0.0  # 0 disables Algorithm 1's snapshot schedule
    eps_factor: float = 0.1
    snapshot_every: int = 0
    # reflected Halpern iteration (the cuPDLP+ line the paper's solver follows,
    # Section 4.1): z <- w ((1 + rho) T(z) - rho z) + (1 - w) z_r with T the
    # PDHG map, w = (t + 1) / (t + 2), t the iterations since the last restart
    # and z_r the last restart point; no averaging (the candidate is always the
    # current iterate)
    halpern: bool = False
    halpern_reflect: float = 1.0
    # feasibility polishing (the PDLP variant the paper describes in Section 5:
    # PDHG iterations with a zero objective, to reach primal feasibility, inside
    # the main solve). Readings: tried at an evaluation whose candidate has
    # rel_gap <= tol but is not yet converged, at most once until the iteration
    # count has doubled; a primal phase (objective 0, from (x_c, 0)) until
    # rel_p <= tol, then a dual phase (right-hand side 0, from (0, y_c)) until
    # rel_d <= tol, each for at most polish_div-th of the main iterations so far
    # (rounded up to whole evaluation periods); the pair (x_p, y_d) ends the
    # solve if its rel_kkt <= tol, otherwise the main iteration goes on as if
    # nothing had happened
    feas_polish: bool = False
    polish_div: int = 8
    # relative-gap tolerance of the termination test; 0 = the same tolerance as
    # the two residuals (the single-eps test of Section 2). Feasibility
    # polishing pays off when the gap tolerance is the looser one.
    gap_tol: float = 0.0
    # restart scheme: 0 = PDLP's weighted KKT error (readings above); 1 = the
    # fixed-point residual scheme of the cuPDLP+ line the paper's solver
    # follows (Section 4.1, which gives no formula, so these are readings), for
    # the reflected Halpern form: at an evaluation the candidate is the current
    # point z, its measure is r(z) = ||z - T(z)||_M (T the PDHG map, M the
    # metric in which T is firmly nonexpansive, see ``fixed_point_residual``);
    # the three restart rules above compare r(z) with r at the last restart and
    # at the previous evaluation; a restart moves to T(z), which becomes the
    # anchor; and the primal weight follows a PID controller on
    # e = ln(omega dx / dy): ln omega -= pid_kp e + pid_ki sum(e) + pid_kd (e -
    # e_prev), dx and dy the moves of the restart point (with pid_kp = theta
    # and the other gains 0 it is PDLP's update)
    restart_scheme: int = 0
    pid_kp: float = 0.99
    pid_ki: float = 0.01
    pid_kd: float = 0.0


def csr_matrix(m, n, row_ptr, col_idx, val) -> sp.csr_matrix:
    """The constraint matrix A of Section 2's primal LP (rows = constraints)
    from its CSR arrays."""
    return sp.csr_matrix((np.asarray(val, dtype=np.float64), np.asarray(col_idx), np.asarray(row_ptr)), shape=(m, n))


# ---------------------------------------------------------------------------
# Section 2: residuals, optimality measures and the relative termination test
# ---------------------------------------------------------------------------

def dual_slack(A: sp.csr_matrix, c: np.ndarray, y: np.ndarray) -> np.ndarray:
    """z for a dual estimate y: the smallest z >= 0 with A^T y + z - c as small as
    possible, z = max(0, c - A^T y). (Section 2 names (x, y, z) but gives no rule
    for z; this is the reading used throughout.)"""
    return np.maximum(0.0, c - A.T @ y)


def kkt(A: sp.csr_matrix, b: np.ndarray, c: np.ndarray, x: np.ndarray, y: np.ndarray,
        z: np.ndarray | None = None) -> dict:
    """All optimality measures of a candidate (x, y, z) on the problem as given.

    r_P = b - A x and r_D = A^T y + z - c (Section 2); the three relative ratios
    of the termination test (Section 2) and their maximum, rel_kkt."""
    if z is None:
        z = dual_slack(A, c, y)
    r_p = b - A @ x
    r_d = A.T @ y + z - c
    cx = float(c @ x)
    by = float(b @ y)
    gap = abs(cx - by)
    out = dict(
        rp_norm2=float(np.linalg.norm(r_p)),
        rp_norminf=float(np.max(np.abs(r_p))) if r_p.size else 0.0,
        rd_norm2=float(np.linalg.norm(r_d)),
        rd_norminf=float(np.max(np.abs(r_d))) if r_d.size else 0.0,
        primal_obj=cx,
        dual_obj=by,
        gap=gap,
        complementarity=float(x @ z),
    )
    out["rel_p"] = out["rp_norm2"] / (1.0 + float(np.linalg.norm(b)))
    out["rel_d"] = out["rd_norm2"] / (1.0 + float(np.linalg.norm(c)))
    out["rel_gap"] = gap / (1.0 + abs(cx) + abs(by))
    out["rel_kkt"] = max(out["rel_p"], out["rel_d"], out["rel_gap"])
    return out


# ---------------------------------------------------------------------------
# Diagonal scaling (PDLP preprocessing; the paper is silent on its details)
# ---------------------------------------------------------------------------

def _inv_sqrt_or_one(v: np.ndarray) -> np.ndarray:
    """1/sqrt(v) where v > 0, else 1: the scaling factor of a row or column,
    with an empty row or column left unscaled (Ruiz and Pock-Chambolle
    scaling, a reading: the paper names its solver's line of work, Section 4.1,
    not its scaling)."""
    out = np.ones_like(v)
    nz = v > 0
    out[nz] = 1.0 / np.sqrt(v[nz])
    return out


def ruiz_scaling(A: sp.csr_matrix, iters: int):
    """Ruiz equilibration: repeat ``iters`` times
    r_i = 1/sqrt(max_j |Ahat_ij|), s_j = 1/sqrt(max_i |Ahat_ij|) (1 for an empty
    row/column), Ahat <- diag(r) Ahat diag(s). Returns (Ahat, d_r, d_c)."""
    Ah = A.copy().astype(np.float64)
    d_r = np.ones(A.shape[0])
    d_c = np.ones(A.shape[1])
    for _ in range(iters):
        absA = abs(Ah)
        row_max = np.asarray(absA.max(axis=1).todense()).ravel()
        col_max = np.asarray(absA.max(axis=0).todense()).ravel()
        r = _inv_sqrt_or_one(row_max)
        s = _inv_sqrt_or_one(col_max)
        Ah = sp.diags(r) @ Ah @ sp.diags(s)
        d_r *= r
        d_c *= s
    return sp.csr_matrix(Ah), d_r, d_c


def _abs_power(A: sp.csr_matrix, p: float) -> sp.csr_matrix:
    """|A_ij|^p on the stored entries, with 0^p = 0 also for p = 0 (a stored
    zero counts as absent): the entry powers of Pock-Chambolle scaling with
    parameter alpha (a reading, as for the rest of the scaling)."""
    B = abs(A).tocsr(copy=True)
    B.data = np.where(B.data > 0, B.data ** p, 0.0)
    return B


def pock_chambolle_scaling(A: sp.csr_matrix, alpha: float = 1.0):
    """Pock-Chambolle diagonal preconditioning with parameter alpha in [0, 2]:
    r_i = 1/sqrt(sum_j |A_ij|^alpha), s_j = 1/sqrt(sum_i |A_ij|^(2 - alpha)).
    Returns (Ahat, r, s)."""
    row_sum = np.asarray(_abs_power(A, alpha).sum(axis=1)).ravel()
    col_sum = np.asarray(_abs_power(A, 2.0 - alpha).sum(axis=0)).ravel()
    r = _inv_sqrt_or_one(row_sum)
    s = _inv_sqrt_or_one(col_sum)
    return sp.csr_matrix(sp.diags(r) @ A @ sp.diags(s)), r, s


def scale_problem(A: sp.csr_matrix, b: np.ndarray, c: np.ndarray, opt: Options):
    """Ahat = D_r A D_c, bhat = D_r b, chat = D_c c: the diagonally scaled LP
    that the PDLP line of work (Section 1, Section 4.1) iterates on; Ruiz
    passes then one Pock-Chambolle pass (readings at ``Options``)."""
    Ah, d_r, d_c = ruiz_scaling(A, opt.ruiz_iters)
    if opt.pock_chambolle:
        Ah, r, s = pock_chambolle_scaling(Ah, opt.pc_alpha)
        d_r = d_r * r
        d_c = d_c * s
    return Ah, d_r * b, d_c * c, d_r, d_c


_SM_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_SM_M1 = np.uint64(0xBF58476D1CE4E5B9)
_SM_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """SplitMix64 (Steele, Lea and Flood 2014, with the finalizer constants of
    Vigna's reference splitmix64.c) as a counter-based generator: the output
    for state counter * 0x9E3779B97F4A7C15 (mod 2^64), i.e. the counter-th
    output of the sequential generator seeded with 0."""
    z = np.asarray(counter, dtype=np.uint64) * _SM_GAMMA
    z = (z ^ (z >> np.uint64(30))) * _SM_M1
    z = (z ^ (z >> np.uint64(27))) * _SM_M2
    return z ^ (z >> np.uint64(31))


def power_start(n: int) -> np.ndarray:
    """Start vector of the power iteration: w_j = 0.5 + u_j, u_j in [0, 1) the
    top 53 bits of splitmix64(j + 1) (j the column of A), normalized to unit
    length. A fixed pseudo-random vector is orthogonal to the leading singular
    vector of no matrix met in practice; the all-ones vector is orthogonal to it
    whenever Ahat 1 = 0 (e.g. Ahat = [1, -1]), and the estimate is then 0."""
    u = (splitmix64(np.arange(1, n + 1, dtype=np.uint64)) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    w = 0.5 + u
    return w / np.linalg.norm(w)


def power_norm(Ah: sp.csr_matrix, iters: int) -> float:
    """Estimate ||Ahat||_2 by ``iters`` power iterations on Ahat^T Ahat from
    ``power_start``: u = Ahat v, w = Ahat^T u, estimate = ||u||, v <- w/||w||."""
    n = Ah.shape[1]
    if n == 0 or Ah.nnz == 0:
        return 0.0
    v = power_start(n)
    est = 0.0
    for _ in range(iters):
        u = Ah @ v
        est = float(np.linalg.norm(u))
        w = Ah.T @ u
        wn = float(np.linalg.norm(w))
        if wn == 0.0:
            break
        v = w / wn
    return est


# ---------------------------------------------------------------------------
# One PDHG iteration (Algorithm 1, "Perform PDHG iteration")
# ---------------------------------------------------------------------------

def pdhg_iteration(Ah, AhT, bh, ch, x, y, tau, sigma):
    """x' = max(0, x - tau (chat - Ahat^T y)); xbar = 2x' - x;
    y' = y + sigma (bhat - Ahat xbar). Returns (x', xbar, y'). The "Perform
    PDHG iteration" step of Algorithm 1 (Section 3.1), in the PDLP form the
    paper's solver follows (Section 4.1; the formula is a reading)."""
    x_new = np.maximum(0.0, x - tau * (ch - AhT @ y))
    xbar = 2.0 * x_new - x
    y_new = y + sigma * (bh - Ah @ xbar)
    return x_new, xbar, y_new


def halpern_iteration(Ah, AhT, bh, ch, x, y, x_anchor, y_anchor, tau, sigma, t, rho):
    """One reflected Halpern step: with (x~, y~) = T(x, y) the PDHG map above,
    w = (t + 1) / (t + 2), returns w ((1 + rho) (x~, y~) - rho (x, y)) + (1 - w)
    (x_anchor, y_anchor). rho = 0 is the plain Halpern iteration of T; rho = 1
    applies it to the reflection 2T - I."""
    xt, _, yt = pdhg_iteration(Ah, AhT, bh, ch, x, y, tau, sigma)
    w = (t + 1.0) / (t + 2.0)
    x_new = w * ((1.0 + rho) * xt - rho * x) + (1.0 - w) * x_anchor
    y_new = w * ((1.0 + rho) * yt - rho * y) + (1.0 - w) * y_anchor
    return x_new, y_new


# ---------------------------------------------------------------------------
# Restart rules
# ---------------------------------------------------------------------------

def weighted_kkt(norms, omega: float) -> float:
    """KKT_omega = sqrt(omega ||r_P||^2 + ||r_D||^2 / omega + gap^2) from the
    (||r_P||, ||r_D||, gap) of a point of the scaled problem: Section 2's
    residuals and gap combined with the primal weight, the measure of PDLP's
    KKT-error restart scheme (a reading; the paper gives no restart rule)."""
    p, d, g = norms
    return math.sqrt(omega * p * p + d * d / omega + g * g)


def choose_candidate(n_cur, n_avg, omega) -> int:
    """The restart candidate of PDLP's scheme (a reading): the average wins
    only if its weighted KKT error is strictly smaller."""
    return RESTART_TO_AVERAGE if weighted_kkt(n_avg, omega) < weighted_kkt(n_cur, omega) else RESTART_TO_CURRENT


def restart_decision(k_cand, k_last_restart, k_prev_cand, t_since, k_total, opt: Options) -> bool:
    """PDLP's three restart criteria on weighted KKT errors:
    sufficient decay, necessary decay with no progress since the previous
    evaluation, or an artificial restart after a long run."""
    if k_cand <= opt.beta_suff * k_last_restart:
        return True
    if k_cand <= opt.beta_nec * k_last_restart and k_cand > k_prev_cand:
        return True
    return t_since >= opt.beta_art * k_total


def _rel_gap(a: float, b: float) -> float:
    """|a - b| / max(|a|, |b|) (0 when both are 0): the relative margin of a
    restart comparison, recorded so that a test can tell a decision taken at
    rounding level from a clear one; no part of the method."""
    d = max(abs(a), abs(b))
    return abs(a - b) / d if d > 0 else 0.0


def primal_weight_update(omega: float, dx: float, dy: float, theta: float) -> float:
    """omega <- exp(theta ln(dy/dx) + (1 - theta) ln omega) when both moves are
    above 1e-10; unchanged otherwise. PDLP's primal-weight update at a restart
    (a reading; the paper gives none), dx and dy the moves of x and y since the
    previous restart point on the scaled problem."""
    if dx > 1e-10 and dy > 1e-10:
        return math.exp(theta * math.log(dy / dx) + (1.0 - theta) * math.log(omega))
    return omega


def fixed_point_residual(Ah, AhT, bh, ch, xh, yh, tau, sigma):
    """(r, x~, y~): the PDHG map's output (x~, y~) = T(xh, yh) and the
    fixed-point residual r = ||z - T(z)||_M of z = (xh, yh) in the metric
    ||(dx, dy)||_M^2 = ||dx||^2 / tau + 2 dy^T Ahat dx + ||dy||^2 / sigma, in
    which the PDHG map is firmly nonexpansive (tau sigma ||Ahat||^2 < 1). The
    measure of the cuPDLP+ restart scheme (Section 4.1 names the line of work;
    the formula is a reading)."""
    xt, _, yt = pdhg_iteration(Ah, AhT, bh, ch, xh, yh, tau, sigma)
    dx, dy = xt - xh, yt - yh
    q = float(dx @ dx) / tau + 2.0 * float(dy @ (Ah @ dx)) + float(dy @ dy) / sigma
    return math.sqrt(max(q, 0.0)), xt, yt


def pid_primal_weight(omega: float, dx: float, dy: float, integral: float, e_prev: float, kp: float, ki: float,
                      kd: float):
    """(omega', integral', e) after one PID step on the error
    e = ln(omega dx / dy), which is 0 when the weighted moves omega dx and dy
    balance: ln omega' = ln omega - kp e - ki (integral + e) - kd (e - e_prev).
    Unchanged when a move is at most 1e-10. The cuPDLP+ primal weight (a
    reading; the paper gives no formula); kp = theta, ki = kd = 0 is PDLP's
    update ``primal_weight_update``."""
    if not (dx > 1e-10 and dy > 1e-10):
        return omega, integral, e_prev
    e = math.log(omega * dx / dy)
    integral = integral + e
    return math.exp(math.log(omega) - kp * e - ki * integral - kd * (e - e_prev)), integral, e


# ---------------------------------------------------------------------------
# The solver
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class EvalRecord:
    """What one evaluation of Algorithm 1's loop decided (Section 3.1; the
    restart fields follow PDLP's scheme, a reading), recorded for comparison
    with the engine's trace."""

    iteration: int
    kind: int  # NO_RESTART / RESTART_TO_CURRENT / RESTART_TO_AVERAGE
    candidate: int  # RESTART_TO_CURRENT / RESTART_TO_AVERAGE
    omega: float  # after the update
    rel_kkt: float  # of the candidate, on the problem as given
    # smallest relative gap between the two sides of any comparison that took
    # part in this evaluation's decisions (candidate choice, restart tests);
    # an implementation that rounds differently may decide otherwise only
    # when this is at rounding level
    margin: float = math.inf
    rel_gap: float = math.nan  # of the candidate, on the problem as given


class Oracle:
    """Plain FP64 PDHG for ``min c^T x, Ax = b, x >= 0`` (Section 2's LP):
    the PDHG loop of Algorithm 1 (Section 3.1) with its evaluations, restarts
    and snapshots; the crossover threads Algorithm 1 launches are not part of
    it."""

    def __init__(self, m, n, row_ptr, col_idx, val, b, c, opt: Options | None = None,
                 x0=None, y0=None):
        self.opt = opt or Options()
        if self.opt.restart_scheme not in (0, 1) or (self.opt.restart_scheme == 1 and self.opt.feas_polish):
            raise ValueError("restart_scheme must be 0 or 1, and 1 is not combined with feasibility polishing")
        self.A = csr_matrix(m, n, row_ptr, col_idx, val)
        self.b = np.asarray(b, dtype=np.float64).copy()
        self.c = np.asarray(c, dtype=np.float64).copy()
        self.m, self.n = m, n
        self.Ah, self.bh, self.ch, self.d_r, self.d_c = scale_problem(self.A, self.b, self.c, self.opt)
        self.AhT = sp.csr_matrix(self.Ah.T)
        self.norm_est = power_norm(self.Ah, self.opt.power_iters)
        self.eta = self.opt.step_factor / self.norm_est if self.norm_est > 0 else 1.0
        if self.opt.primal_weight:
            cn, bn = float(np.linalg.norm(self.ch)), float(np.linalg.norm(self.bh))
            self.omega = cn / bn if (cn > 1e-10 and bn > 1e-10) else 1.0
        else:
            self.omega = 1.0
        # iterate in scaled space: x = D_c xhat, y = D_r yhat
        self.x = np.zeros(n) if x0 is None else np.asarray(x0, dtype=np.float64) / self.d_c
        self.y = np.zeros(m) if y0 is None else np.asarray(y0, dtype=np.float64) / self.d_r
        self.x_sum = np.zeros(n)
        self.y_sum = np.zeros(m)
        self.t = 0
        self.k = 0
        self.trace: list[EvalRecord] = []
        self.snapshots: list[dict] = []
        self.eps_target = self.opt.eps_cross
        self.next_snapshot = self.opt.snapshot_every
        self.restart_count = 0
        self.done = False
        # termination measure: "rel_kkt" for the LP itself, "rel_p" / "rel_d" in
        # the phases of feasibility polishing
        self.term = "rel_kkt"
        self.next_polish = 0
        self.polish_log: list[dict] = []
        # restart reference = the starting point
        self.x_r, self.y_r = self.x.copy(), self.y.copy()
        self.n_restart = self.scaled_norms(self.x, self.y)
        self.n_prev = self.n_restart
        # fixed-point residual scheme: r at the last restart and at the
        # previous evaluation, and the PID controller's state
        self.r_restart = self.r_prev = self.fixed_point_measure(self.x, self.y)[0]
        self.pid_integral, self.pid_prev = 0.0, 0.0

    # -- step sizes --------------------------------------------------------
    @property
    def tau(self) -> float:
        """Primal step eta / omega (PDLP's step split by the primal weight, a
        reading)."""
        return self.eta / self.omega

    @property
    def sigma(self) -> float:
        """Dual step eta * omega (as ``tau``)."""
        return self.eta * self.omega

    # -- measures on the scaled problem (restart rules) --------------------
    def scaled_norms(self, xh, yh):
        """(||bhat - Ahat xhat||, ||max(0, Ahat^T yhat - chat)||, |chat^T xhat - bhat^T yhat|):
        Section 2's residual norms and gap on the scaled problem, the inputs of
        the restart rules (a reading: they measure on the problem they iterate)."""
        rp = self.bh - self.Ah @ xh
        rd = np.maximum(0.0, self.AhT @ yh - self.ch)
        return (float(np.linalg.norm(rp)), float(np.linalg.norm(rd)), abs(float(self.ch @ xh) - float(self.bh @ yh)))

    def fixed_point_measure(self, xh, yh):
        """``fixed_point_residual`` of a scaled point with the current step
        sizes: (r, x~, y~)."""
        return fixed_point_residual(self.Ah, self.AhT, self.bh, self.ch, xh, yh, self.tau, self.sigma)

    # -- unscaled quantities -----------------------------------------------
    def unscale(self, xh, yh):
        """(x, y, z) of the problem as given from a scaled point:
        x = D_c xhat, y = D_r yhat and Section 2's z = max(0, c - A^T y)."""
        x = self.d_c * xh
        y = self.d_r * yh
        return x, y, dual_slack(self.A, self.c, y)

    def kkt_of(self, xh, yh) -> dict:
        """Section 2's KKT measures (``kkt``) of a scaled point, on the problem
        as given."""
        x, y, z = self.unscale(xh, yh)
        return kkt(self.A, self.b, self.c, x, y, z)

    @property
    def x_avg(self):
        """Uniform average of the x iterates since the last restart (PDLP's
        averaged restart candidate, a reading); the current x before any."""
        return self.x_sum / self.t if self.t > 0 else self.x.copy()

    @property
    def y_avg(self):
        """As ``x_avg``, for y."""
        return self.y_sum / self.t if self.t > 0 else self.y.copy()

    # -- iteration -----------------------------------------------------------
    def iterate_once(self):
        """One iteration of Algorithm 1's PDHG loop (Section 3.1): the PDHG map
        (or its reflected Halpern form), then the running sums of the average
        since the last restart."""
        if self.opt.halpern:
            self.x, self.y = halpern_iteration(self.Ah, self.AhT, self.bh, self.ch, self.x, self.y, self.x_r, self.y_r,
                                               self.tau, self.sigma, self.t, self.opt.halpern_reflect)
            self.t += 1
            self.k += 1
            return
        x_new, _, y_new = pdhg_iteration(self.Ah, self.AhT, self.bh, self.ch, self.x, self.y, self.tau, self.sigma)
        self.x, self.y = x_new, y_new
        if self.opt.restarts:
            self.x_sum += x_new
            self.y_sum += y_new
        self.t += 1
        self.k += 1

    def evaluate(self, tol: float) -> bool:
        """One evaluation: candidate choice, termination (Section 2's relative
        test), Algorithm 1's snapshots (Section 3.1), restart and primal-weight
        update (PDLP's scheme, a reading), then a feasibility polishing attempt
        when its rules allow (Section 5, readings at ``Options``). Returns True
        when the method has converged."""
        opt = self.opt
        if opt.restart_scheme == 1:
            return self.evaluate_fixed_point(tol)
        if opt.restarts and self.t > 0 and not opt.halpern:
            xa, ya = self.x_avg, self.y_avg
            n_cur = self.scaled_norms(self.x, self.y)
            n_avg = self.scaled_norms(xa, ya)
            which = choose_candidate(n_cur, n_avg, self.omega)
        else:
            xa = ya = None
            n_cur = self.scaled_norms(self.x, self.y)
            n_avg = None
            which = RESTART_TO_CURRENT
        if which == RESTART_TO_AVERAGE:
            xc, yc, n_c = xa, ya, n_avg
        else:
            xc, yc, n_c = self.x, self.y, n_cur
        kk = self.kkt_of(xc, yc)
        rel = kk[self.term]
        gtol = opt.gap_tol if opt.gap_tol > 0 else tol

        if self.term == "rel_kkt":
            converged = tol > 0 and kk["rel_p"] <= tol and kk["rel_d"] <= tol and kk["rel_gap"] <= gtol
        else:
            converged = tol > 0 and rel <= tol
        # Algorithm 1: snapshot when maxresid <= eps_target, then shrink eps_target.
        if self.eps_target > 0 and rel <= self.eps_target:
            self._snapshot(xc, yc, rel, "threshold")
            self.eps_target *= opt.eps_factor
        if opt.snapshot_every > 0 and self.k >= self.next_snapshot:
            self._snapshot(xc, yc, rel, "periodic")
            while self.next_snapshot <= self.k:
                self.next_snapshot += opt.snapshot_every

        kind = NO_RESTART
        margin = math.inf
        if n_avg is not None:
            ka, kc0 = weighted_kkt(n_avg, self.omega), weighted_kkt(n_cur, self.omega)
            margin = _rel_gap(ka, kc0)
        if converged:
            self.x, self.y = xc.copy(), yc.copy()
        elif opt.restarts:
            om = self.omega
            k_c = weighted_kkt(n_c, om)
            k_r, k_p = weighted_kkt(self.n_restart, om), weighted_kkt(self.n_prev, om)
            margin = min(margin, _rel_gap(k_c, opt.beta_suff * k_r), _rel_gap(k_c, opt.beta_nec * k_r),
                         _rel_gap(k_c, k_p))
            if restart_decision(k_c, k_r, k_p, self.t, self.k, opt):
                kind = which
                if opt.primal_weight:
                    dx = float(np.linalg.norm(xc - self.x_r))
                    dy = float(np.linalg.norm(yc - self.y_r))
                    self.omega = primal_weight_update(self.omega, dx, dy, opt.theta)
                self.x, self.y = xc.copy(), yc.copy()
                self.x_r, self.y_r = xc.copy(), yc.copy()
                self.n_restart = n_c
                self.x_sum[:] = 0.0
                self.y_sum[:] = 0.0
                self.t = 0
                self.restart_count += 1
            self.n_prev = n_c
        self.trace.append(EvalRecord(self.k, kind, which, self.omega, rel, margin, kk["rel_gap"]))
        if (not converged and opt.feas_polish and tol > 0 and self.term == "rel_kkt" and self.k >= self.next_polish
                and kk["rel_gap"] <= gtol):
            self.next_polish = 2 * self.k
            polished = self.feasibility_polish(xc, yc, tol)
            if polished is not None:
                self.x, self.y = polished
                converged = True
        return converged

    def evaluate_fixed_point(self, tol: float) -> bool:
        """One evaluation under the fixed-point residual restart scheme
        (``Options.restart_scheme`` = 1, the cuPDLP+ line, readings): the
        candidate is the current point; termination and Algorithm 1's
        snapshots as in ``evaluate``; the three restart rules on r(z); a
        restart moves the iterate and the anchor to T(z) and updates the
        primal weight by ``pid_primal_weight``."""
        opt = self.opt
        kk = self.kkt_of(self.x, self.y)
        rel = kk[self.term]
        gtol = opt.gap_tol if opt.gap_tol > 0 else tol
        converged = tol > 0 and kk["rel_p"] <= tol and kk["rel_d"] <= tol and kk["rel_gap"] <= gtol
        if self.eps_target > 0 and rel <= self.eps_target:
            self._snapshot(self.x, self.y, rel, "threshold")
            self.eps_target *= opt.eps_factor
        if opt.snapshot_every > 0 and self.k >= self.next_snapshot:
            self._snapshot(self.x, self.y, rel, "periodic")
            while self.next_snapshot <= self.k:
                self.next_snapshot += opt.snapshot_every
        kind = NO_RESTART
        margin = math.inf
        if not converged and opt.restarts:
            r_c, xt, yt = self.fixed_point_measure(self.x, self.y)
            margin = min(_rel_gap(r_c, opt.beta_suff * self.r_restart), _rel_gap(r_c, opt.beta_nec * self.r_restart),
                         _rel_gap(r_c, self.r_prev))
            if restart_decision(r_c, self.r_restart, self.r_prev, self.t, self.k, opt):
                kind = RESTART_TO_PDHG_STEP
                if opt.primal_weight:
                    dx = float(np.linalg.norm(xt - self.x_r))
                    dy = float(np.linalg.norm(yt - self.y_r))
                    self.omega, self.pid_integral, self.pid_prev = pid_primal_weight(
                        self.omega, dx, dy, self.pid_integral, self.pid_prev, opt.pid_kp, opt.pid_ki, opt.pid_kd)
                self.x, self.y = xt.copy(), yt.copy()
                self.x_r, self.y_r = xt.copy(), yt.copy()
                self.r_restart = r_c
                self.t = 0
                self.restart_count += 1
            self.r_prev = r_c
        self.trace.append(EvalRecord(self.k, kind, RESTART_TO_CURRENT, self.omega, rel, margin, kk["rel_gap"]))
        return converged

    # -- feasibility polishing ---------------------------------------------
    def phase_solver(self, xh0, yh0, kind: str) -> "Oracle":
        """The solver of one polishing phase, before its first iteration: PDHG
        on the problem with the objective (kind "primal") or the right-hand
        side (kind "dual") set to zero, from the scaled point (xh0, yh0), with
        this solver's scaling, eta and current primal weight, empty averages,
        the start as its restart reference, the same restart rules, and rel_p
        (primal) or rel_d (dual) of its candidate as the termination measure.
        Section 5's polishing phases; their start points and measures are
        readings (see ``Options``)."""
        sub = Oracle.__new__(Oracle)
        sub.__dict__.update(self.__dict__)
        sub.opt = dataclasses.replace(self.opt, eps_cross=0.0, snapshot_every=0, feas_polish=False)
        if kind == "primal":
            sub.c = np.zeros(self.n)
            sub.ch = np.zeros(self.n)
            sub.term = "rel_p"
        else:
            sub.b = np.zeros(self.m)
            sub.bh = np.zeros(self.m)
            sub.term = "rel_d"
        sub.x, sub.y = np.array(xh0, dtype=np.float64), np.array(yh0, dtype=np.float64)
        sub.x_sum, sub.y_sum = np.zeros(self.n), np.zeros(self.m)
        sub.t = sub.k = 0
        sub.trace, sub.snapshots, sub.polish_log = [], [], []
        sub.eps_target, sub.next_snapshot = 0.0, 0
        sub.restart_count = 0
        sub.done = False
        sub.x_r, sub.y_r = sub.x.copy(), sub.y.copy()
        sub.n_restart = sub.scaled_norms(sub.x, sub.y)
        sub.n_prev = sub.n_restart
        return sub

    def feasibility_phase(self, xh0, yh0, kind: str, tol: float, budget: int):
        """One polishing phase (see ``phase_solver``): it stops at the first
        evaluation where its termination measure is <= tol, or after
        ``budget`` iterations (Section 5's polishing, readings at
        ``Options``). Returns (xhat, yhat, iterations, reached)."""
        sub = self.phase_solver(xh0, yh0, kind)
        reached = sub.run(budget, tol)
        return sub.x, sub.y, sub.k, reached

    def polish_budget(self) -> int:
        """Iterations allowed to each phase: the main iterations so far divided
        by polish_div, rounded up to whole evaluation periods (at least one);
        a reading, since Section 5 gives no budget."""
        e = self.opt.eval_every
        return e * max(1, -(-self.k // (self.opt.polish_div * e)))

    def feasibility_polish(self, xh_c, yh_c, tol: float):
        """One attempt of Section 5's feasibility polishing (the phases and
        their order are readings): primal phase from (x_c, 0), then (if it
        reached rel_p <= tol) dual phase from (0, y_c); returns the scaled pair
        (x_p, y_d) when it passes Section 2's termination test on the LP as
        given, else None."""
        budget = self.polish_budget()
        rec = dict(iteration=self.k, budget=budget, primal_iters=0, primal_ok=False, dual_iters=0, dual_ok=False,
                   rel_kkt=math.inf)
        self.polish_log.append(rec)
        xp, _, kp, okp = self.feasibility_phase(xh_c, np.zeros(self.m), "primal", tol, budget)
        rec.update(primal_iters=kp, primal_ok=okp)
        if not okp:
            return None
        _, yd, kd, okd = self.feasibility_phase(np.zeros(self.n), yh_c, "dual", tol, budget)
        rec.update(dual_iters=kd, dual_ok=okd)
        if not okd:
            return None
        kk = self.kkt_of(xp, yd)
        rec["rel_kkt"] = kk["rel_kkt"]
        rec["rel_gap"] = kk["rel_gap"]
        gtol = self.opt.gap_tol if self.opt.gap_tol > 0 else tol
        if kk["rel_p"] <= tol and kk["rel_d"] <= tol and kk["rel_gap"] <= gtol:
            return xp.copy(), yd.copy()
        return None

    def _snapshot(self, xh, yh, rel, why):
        """Record (x_k, y_k, z_k) on the problem as given: the copy Algorithm 1
        hands to a crossover thread (Section 3.1)."""
        x, y, z = self.unscale(xh, yh)
        self.snapshots.append(dict(iteration=self.k, x=x, y=y, z=z, rel_kkt=rel, why=why))

    def run(self, max_iters: int, tol: float = 0.0) -> bool:
        """Algorithm 1's PDHG loop (Section 3.1): iterate until the candidate
        passes the termination test of Section 2 (rel_p, rel_d <= tol and
        rel_gap <= gap_tol, or tol) at an evaluation or max_iters iterations.
        Evaluations happen every ``eval_every`` iterations when restarts are on or
        tol > 0; with restarts off and tol = 0 this is plain fixed-step PDHG."""
        evaluating = self.opt.restarts or tol > 0 or self.opt.eps_cross > 0 or self.opt.snapshot_every > 0
        for _ in range(max_iters):
            if self.done:
                break
            self.iterate_once()
            if evaluating and self.k % self.opt.eval_every == 0:
                if self.evaluate(tol):
                    self.done = True
        return self.done

    # -- results ---------------------------------------------------------------
    def solution(self):
        """Unscaled (x, y, z) of the current iterate: Section 2's primal x, dual
        y and reduced costs z = max(0, c - A^T y)."""
        return self.unscale(self.x, self.y)


# ---------------------------------------------------------------------------
# Differentiating K unrolled iterations (fixed step, no restarts, omega fixed)
# ---------------------------------------------------------------------------

def unrolled_forward(orc: Oracle, K: int, c=None, b=None):
    """K plain PDHG iterations of ``orc``'s scaled problem from its current
    point, optionally with a different objective c or right-hand side b (the
    scaling, eta and omega stay those of ``orc``). Returns the scaled iterates
    x_0..x_K and y_0..y_K. The map of Algorithm 1's "Perform PDHG iteration"
    step (Section 3.1) applied K times; differentiating it has no counterpart
    in the paper."""
    ch = orc.d_c * (orc.c if c is None else np.asarray(c, dtype=np.float64))
    bh = orc.d_r * (orc.b if b is None else np.asarray(b, dtype=np.float64))
    xs, ys = [orc.x.copy()], [orc.y.copy()]
    for _ in range(K):
        x1, _, y1 = pdhg_iteration(orc.Ah, orc.AhT, bh, ch, xs[-1], ys[-1], orc.tau, orc.sigma)
        xs.append(x1)
        ys.append(y1)
    return xs, ys


def unrolled_adjoint(orc: Oracle, K: int, gx_K, gy_K=None):
    """Reverse pass through K unrolled iterations: given dL/dx_K and dL/dy_K
    on the problem as given (x = D_c xhat, y = D_r yhat), return (dL/dc, dL/db).
    The chain rule through the map of ``unrolled_forward``; no counterpart in
    the paper.

    One iteration, u = x - tau (chat - Ahat^T y), x' = max(u, 0),
    v = 2x' - x, y' = y + sigma (bhat - Ahat v), is reversed as
        g_v   = -sigma Ahat^T g_y'
        g_u   = [u > 0] (g_x' + 2 g_v)        (derivative 0 at u = 0)
        g_x   = -g_v + g_u
        g_y   = g_y' + tau Ahat g_u
        g_bhat += sigma g_y',  g_chat += -tau g_u
    with chat = D_c c and bhat = D_r b."""
    xs, _ = unrolled_forward(orc, K)
    gx = orc.d_c * np.asarray(gx_K, dtype=np.float64)
    gy = np.zeros(orc.m) if gy_K is None else orc.d_r * np.asarray(gy_K, dtype=np.float64)
    g_ch = np.zeros(orc.n)
    g_bh = np.zeros(orc.m)
    for k in range(K - 1, -1, -1):
        g_v = -orc.sigma * (orc.AhT @ gy)
        g_u = np.where(xs[k + 1] > 0, gx + 2.0 * g_v, 0.0)
        g_bh += orc.sigma * gy
        g_ch += -orc.tau * g_u
        gx = -g_v + g_u
        gy = gy + orc.tau * (orc.Ah @ g_u)
    return orc.d_c * g_ch, orc.d_r * g_bh


def unrolled_loss(orc: Oracle, K: int, x_target, c=None, b=None) -> float:
    """0.5 ||x_K - x_target||^2 with x_K on the problem as given: the loss
    through which the unrolled iterations are differentiated (no counterpart in
    the paper; a test function for ``unrolled_adjoint``)."""
    xs, _ = unrolled_forward(orc, K, c=c, b=b)
    r = orc.d_c * xs[-1] - x_target
    return 0.5 * float(r @ r)
