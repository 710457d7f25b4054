// The decisions of one evaluation (restart scheme, primal weight,
// termination, snapshot schedule), shared by the multi-launch engine and the
// single-block solve loop (internal). Termination is Section 2's relative test,
// the snapshot schedule Algorithm 1's thresholds (Section 3.1); the restart
// scheme and primal weight are PDLP's (readings: the paper gives neither).
#pragma once

#include "common.cuh"

namespace pdhg {

__device__ __forceinline__ void scaled_norms(const EvalSums& e, double& p, double& d, double& g) {
  p = sqrt(e.q[Q_RP2S]);
  d = sqrt(e.q[Q_RD2S]);
  g = fabs(e.q[Q_CX] - e.q[Q_BY]);
}

__device__ __forceinline__ double weighted_kkt(double p, double d, double g, double omega) {
  return sqrt(omega * p * p + d * d / omega + g * g);
}

// The fixed-point residual ||z - T(z)||_M of an evaluated point in the
// metric ||(dx, dy)||_M^2 = ||dx||^2 / tau + 2 dy^T Ahat dx + ||dy||^2 / sigma
// (the cuPDLP+ restart measure; a reading)
__device__ __forceinline__ double fixed_residual(const EvalSums& e, double tau, double sigma) {
  const double q = e.q[Q_FX2] / tau + 2.0 * e.q[Q_FXY] + e.q[Q_FY2] / sigma;
  return sqrt(q > 0.0 ? q : 0.0);
}

// One PID step of the primal weight on e = ln(omega dx / dy) (the cuPDLP+
// primal weight; a reading): ln omega -= kp e + ki (sum of e) + kd (e - e_prev)
__device__ __forceinline__ void pid_primal_weight(DevState* st, double dx, double dy) {
  if (!(dx > 1e-10 && dy > 1e-10)) return;
  const double e = log(st->omega * dx / dy);
  st->pid_int += e;
  st->omega = exp(log(st->omega) - st->pid_kp * e - st->pid_ki * st->pid_int - st->pid_kd * (e - st->pid_prev));
  st->pid_prev = e;
}

// One evaluation's decisions (single thread): candidate, termination,
// snapshot schedule (Algorithm 1), restart test, primal-weight update.
static __device__ void decide_one(DevState* st, TraceRec* trace) {
  double cp, cd, cg;
  scaled_norms(st->cur, cp, cd, cg);
  int which = KIND_CUR;
  if (st->restarts_on && st->t > 0 && !st->halpern) {  // Halpern: no averages
    double ap, ad, ag;
    scaled_norms(st->avg, ap, ad, ag);
    if (weighted_kkt(ap, ad, ag, st->omega) < weighted_kkt(cp, cd, cg, st->omega)) {
      which = KIND_AVG;
      cp = ap;
      cd = ad;
      cg = ag;
    }
  }
  const EvalSums& e = which == KIND_AVG ? st->avg : st->cur;
  const double cx = e.q[Q_CX], by = e.q[Q_BY];
  const double rel_p = sqrt(e.q[Q_RP2U]) / (1.0 + st->b_norm);
  const double rel_d = sqrt(e.q[Q_RD2U]) / (1.0 + st->c_norm);
  const double rel_g = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
  // the termination measure: rel_kkt for the LP itself, rel_p / rel_d in the
  // phases of feasibility polishing
  const double rel = st->term_mode == TERM_PRIMAL ? rel_p
                     : st->term_mode == TERM_DUAL ? rel_d
                                                  : fmax(rel_p, fmax(rel_d, rel_g));
  st->numeric = !(isfinite(rel_p) && isfinite(rel_d) && isfinite(rel_g) && isfinite(cp) && isfinite(cd));
  st->candidate = which;
  st->cand_rel_kkt = rel;
  st->cand_rel_gap = rel_g;

  const double gtol = st->gap_tol > 0.0 ? st->gap_tol : st->tol;
  int converged;
  if (st->term_mode == TERM_PRIMAL)
    converged = st->tol > 0.0 && rel_p <= st->tol;
  else if (st->term_mode == TERM_DUAL)
    converged = st->tol > 0.0 && rel_d <= st->tol;
  else
    converged = st->tol > 0.0 && rel_p <= st->tol && rel_d <= st->tol && rel_g <= gtol;
  int snap = 0;
  if (st->eps_target > 0.0 && rel <= st->eps_target) {
    snap = 1;
    st->eps_target *= st->eps_factor;
  }
  if (st->snapshot_every > 0 && st->k >= st->next_snapshot) {
    snap = 1;
    while (st->next_snapshot <= st->k) st->next_snapshot += st->snapshot_every;
  }
  st->snapshot_flag = snap;
  if (snap) {
    st->snapshots += 1;
    st->snap_k = st->k;
    st->snap_rel = rel;
  }

  int kind = KIND_NONE, apply = APPLY_NONE;
  if (converged) {
    apply = which == KIND_AVG ? APPLY_TAKE_AVG : APPLY_NONE;
  } else if (st->restarts_on && st->restart_scheme == 1) {
    // the cuPDLP+ scheme (readings): PDLP's three rules on the fixed-point
    // residual of the current point; a restart moves to its PDHG step T(z)
    // (the iterate and the anchor) and takes a PID step of the primal weight
    // on the moves of the restart point
    const double rc = fixed_residual(st->cur, st->tau, st->sigma);
    const bool restart = (rc <= st->beta_suff * st->r_restart) ||
                         (rc <= st->beta_nec * st->r_restart && rc > st->r_prev) ||
                         ((double)st->t >= st->beta_art * (double)st->k);
    if (restart) {
      kind = KIND_STEP;
      if (st->primal_weight_on) pid_primal_weight(st, sqrt(st->cur.q[Q_FXR2]), sqrt(st->cur.q[Q_FYR2]));
      apply = APPLY_RESTART_STEP;
      st->r_restart = rc;
      st->t = 0;
      st->restarts += 1;
    }
    st->r_prev = rc;
  } else if (st->restarts_on) {
    const double om = st->omega;
    const double kc = weighted_kkt(cp, cd, cg, om);
    const double kr = weighted_kkt(st->rs_p, st->rs_d, st->rs_g, om);
    const double kp = weighted_kkt(st->pc_p, st->pc_d, st->pc_g, om);
    const bool restart = (kc <= st->beta_suff * kr) || (kc <= st->beta_nec * kr && kc > kp) ||
                         ((double)st->t >= st->beta_art * (double)st->k);
    if (restart) {
      kind = which;
      if (st->primal_weight_on) {
        const double dx = sqrt(e.q[Q_DX2]), dy = sqrt(e.q[Q_DY2]);
        if (dx > 1e-10 && dy > 1e-10) st->omega = exp(st->theta * log(dy / dx) + (1.0 - st->theta) * log(om));
      }
      apply = which == KIND_AVG ? APPLY_RESTART_AVG : APPLY_RESTART_CUR;
      st->rs_p = cp;
      st->rs_d = cd;
      st->rs_g = cg;
      st->t = 0;
      st->restarts += 1;
    }
    st->pc_p = cp;
    st->pc_d = cd;
    st->pc_g = cg;
  }
  st->kind = kind;
  st->apply_mode = apply;
  st->converged = converged;
  st->tau = st->eta / st->omega;
  st->sigma = st->eta * st->omega;
  if (trace && st->evals < TRACE_CAP) {
    TraceRec& r = trace[st->evals];
    r.iteration = st->k;
    r.kind = kind;
    r.candidate = which;
    r.omega = st->omega;
    r.rel_kkt = rel;
  }
  st->evals += 1;
}

}  // namespace pdhg
