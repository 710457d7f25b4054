// CUDA kernels of the PDHG engine (sm_103a).
//
// The iteration is bandwidth bound: each half-step streams one copy of the
// scaled matrix (CSR of Ahat for the dual step, CSR of Ahat^T for the primal
// step) exactly once, gathers one vector, and fuses the vector update of the
// step into the epilogue of the row reduction, so the step's vectors are read
// and written once. Tensor cores play no part: SpMV is not a dense
// contraction.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace pdhg {

namespace {

constexpr int TPB = 256;

__device__ __forceinline__ double relu(double v) { return v < 0.0 ? 0.0 : v; }  // NaN passes through

template <int W>
__device__ __forceinline__ double group_max(double v) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off, W));
  return v;
}

// Every group of LPR lanes owns one row per pass; a warp handles 32/LPR rows
// per pass and all lanes of a warp make the same number of passes, so the
// group shuffles always run with the full warp.
template <int LPR, class Fn>
__device__ __forceinline__ void for_each_row(int nrows, Fn&& fn) {
  constexpr int RPW = 32 / LPR;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR, gl = lane % LPR;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = warp * RPW; base < nrows; base += nwarps * RPW) {
    const long long row = base + sub;
    fn((int)row, row < nrows, gl);
  }
}

// Row dot product sum_k M_rk vec[col_k]; result valid in group lane 0.
template <int LPR>
__device__ __forceinline__ double row_dot(const Csr& M, int row, bool valid, int gl, const double* __restrict__ vec) {
  double acc = 0.0;
  if (valid) {
    const int beg = __ldg(M.rp + row), end = __ldg(M.rp + row + 1);
    for (int k = beg + gl; k < end; k += LPR) acc += __ldg(M.v + k) * __ldg(vec + __ldg(M.ci + k));
  }
  return group_sum<LPR>(acc);
}

// ---------------------------------------------------------------------------
// setup kernels
// ---------------------------------------------------------------------------
template <int LPR>
__global__ void __launch_bounds__(TPB) k_row_absmax(Csr M, double* __restrict__ out) {
  for_each_row<LPR>(M.rows, [&](int r, bool valid, int gl) {
    double mx = 0.0;
    if (valid)
      for (int k = M.rp[r] + gl; k < M.rp[r + 1]; k += LPR) mx = fmax(mx, fabs(M.v[k]));
    mx = group_max<LPR>(mx);
    if (valid && gl == 0) out[r] = mx;
  });
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_row_abspow_sum(Csr M, double alpha, double* __restrict__ out) {
  for_each_row<LPR>(M.rows, [&](int r, bool valid, int gl) {
    double acc = 0.0;
    if (valid)
      for (int k = M.rp[r] + gl; k < M.rp[r + 1]; k += LPR) {
        const double a = fabs(M.v[k]);
        acc += alpha == 1.0 ? a : pow(a, alpha);
      }
    acc = group_sum<LPR>(acc);
    if (valid && gl == 0) out[r] = acc;
  });
}

__global__ void k_inv_sqrt_or_one(const double* __restrict__ in, double* __restrict__ out, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    const double v = in[i];
    out[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  }
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_scale_csr(Csr M, const double* __restrict__ r, const double* __restrict__ s,
                                                   int transposed) {
  for_each_row<LPR>(M.rows, [&](int row, bool valid, int gl) {
    if (!valid) return;
    for (int k = M.rp[row] + gl; k < M.rp[row + 1]; k += LPR) {
      const int col = M.ci[k];
      const double ri = transposed ? r[col] : r[row];
      const double sj = transposed ? s[row] : s[col];
      M.v[k] = (ri * M.v[k]) * sj;
    }
  });
}

__global__ void k_mul_inplace(double* __restrict__ d, const double* __restrict__ f, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    d[i] *= f[i];
}

__global__ void k_mul(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] * b[i];
}

__global__ void k_div(double* __restrict__ out, const double* __restrict__ a, const double* __restrict__ b, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] / b[i];
}

__global__ void k_fill(double* __restrict__ v, double val, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    v[i] = val;
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_spmv(Csr M, const double* __restrict__ x, double* __restrict__ y) {
  for_each_row<LPR>(M.rows, [&](int r, bool valid, int gl) {
    const double acc = row_dot<LPR>(M, r, valid, gl, x);
    if (valid && gl == 0) y[r] = acc;
  });
}

__global__ void __launch_bounds__(TPB) k_sumsq_partials(const double* __restrict__ v, int len, double* __restrict__ partials) {
  double vals[1] = {0.0};
  const bool mx[1] = {false};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    vals[0] += v[i] * v[i];
  block_reduce<1>(vals, mx);
  if (threadIdx.x == 0) partials[blockIdx.x] = vals[0];
}

// one warp sums nb partials in a fixed order
__global__ void k_sum_partials(const double* __restrict__ partials, int nb, double* __restrict__ out) {
  double acc = 0.0;
  for (int b = threadIdx.x; b < nb; b += 32) acc += partials[b];
  acc = warp_sum(acc);
  if (threadIdx.x == 0) *out = acc;
}

__global__ void k_div_by_norm(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ s2, int len) {
  const double s = sqrt(*s2);
  if (!(s > 0.0)) return;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] / s;
}

// scal: [0] = ||Ahat v||^2 of the last power iteration, [1] = ||chat||^2,
// [2] = ||bhat||^2, [3] = ||b||^2, [4] = ||c||^2
__global__ void k_finish_setup(DevState* st, const double* __restrict__ scal, double step_factor, int primal_weight) {
  const double est = sqrt(scal[0]);
  st->norm_est = est;
  st->eta = est > 0.0 ? step_factor / est : 1.0;
  double omega = 1.0;
  if (primal_weight) {
    const double cn = sqrt(scal[1]), bn = sqrt(scal[2]);
    if (cn > 1e-10 && bn > 1e-10) omega = cn / bn;
  }
  st->omega = omega;
  st->tau = st->eta / omega;
  st->sigma = st->eta * omega;
  st->b_norm = sqrt(scal[3]);
  st->c_norm = sqrt(scal[4]);
}

// ---------------------------------------------------------------------------
// the two fused half-steps of one PDHG iteration
// ---------------------------------------------------------------------------
template <int LPR>
__global__ void __launch_bounds__(TPB) k_primal_step(Csr At, const double* __restrict__ y, const double* __restrict__ ch,
                                                     double* __restrict__ x, double* __restrict__ xbar,
                                                     double* __restrict__ xsum, const DevState* __restrict__ st,
                                                     int accumulate) {
  const double tau = st->tau;
  for_each_row<LPR>(At.rows, [&](int j, bool valid, int gl) {
    const double g = row_dot<LPR>(At, j, valid, gl, y);
    if (valid && gl == 0) {
      const double xj = x[j];
      const double xn = relu(xj - tau * (ch[j] - g));
      xbar[j] = 2.0 * xn - xj;
      x[j] = xn;
      if (accumulate) xsum[j] += xn;
    }
  });
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_dual_step(Csr A, const double* __restrict__ xbar, const double* __restrict__ bh,
                                                   double* __restrict__ y, double* __restrict__ ysum,
                                                   const DevState* __restrict__ st, int accumulate) {
  const double sigma = st->sigma;
  for_each_row<LPR>(A.rows, [&](int i, bool valid, int gl) {
    const double h = row_dot<LPR>(A, i, valid, gl, xbar);
    if (valid && gl == 0) {
      const double yn = y[i] + sigma * (bh[i] - h);
      y[i] = yn;
      if (accumulate) ysum[i] += yn;
    }
  });
}

__global__ void k_add_counters(DevState* st, long long dk) {
  st->k += dk;
  st->t += dk;
}

// ---------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------
__global__ void k_make_average(const double* __restrict__ xs, const double* __restrict__ ys, const double* __restrict__ x,
                               const double* __restrict__ y, double* __restrict__ xa, double* __restrict__ ya, int n,
                               int m, const DevState* __restrict__ st) {
  const long long t = st->t;
  const double td = (double)t;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) xa[i] = t > 0 ? xs[i] / td : x[i];
    if (i < m) ya[i] = t > 0 ? ys[i] / td : y[i];
  }
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_eval_dual(Csr At, const double* __restrict__ py, const double* __restrict__ ch,
                                                   const double* __restrict__ dc, const double* __restrict__ px,
                                                   const double* __restrict__ xr, double* __restrict__ partials) {
  double v[6] = {0, 0, 0, 0, 0, 0};
  const bool mx[6] = {false, false, true, false, false, false};
  for_each_row<LPR>(At.rows, [&](int j, bool valid, int gl) {
    const double g = row_dot<LPR>(At, j, valid, gl, py);
    if (valid && gl == 0) {
      const double c = ch[j];
      const double rd = relu(g - c);
      const double zh = relu(c - g);
      const double rdu = rd / dc[j];
      const double xj = px[j];
      v[0] += rd * rd;
      v[1] += rdu * rdu;
      v[2] = fmax(v[2], fabs(rdu));
      v[3] += c * xj;
      v[4] += xj * zh;
      if (xr) {
        const double d = xj - xr[j];
        v[5] += d * d;
      }
    }
  });
  block_reduce<6>(v, mx);
  if (threadIdx.x == 0) {
    double* p = partials + (size_t)blockIdx.x * NQ;
    p[Q_RD2S] = v[0];
    p[Q_RD2U] = v[1];
    p[Q_RDINF] = v[2];
    p[Q_CX] = v[3];
    p[Q_XZ] = v[4];
    p[Q_DX2] = v[5];
  }
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_eval_primal(Csr A, const double* __restrict__ px, const double* __restrict__ bh,
                                                     const double* __restrict__ dr, const double* __restrict__ py,
                                                     const double* __restrict__ yr, double* __restrict__ partials) {
  double v[5] = {0, 0, 0, 0, 0};
  const bool mx[5] = {false, false, true, false, false};
  for_each_row<LPR>(A.rows, [&](int i, bool valid, int gl) {
    const double h = row_dot<LPR>(A, i, valid, gl, px);
    if (valid && gl == 0) {
      const double b = bh[i];
      const double rp = b - h;
      const double rpu = rp / dr[i];
      const double yi = py[i];
      v[0] += rp * rp;
      v[1] += rpu * rpu;
      v[2] = fmax(v[2], fabs(rpu));
      v[3] += b * yi;
      if (yr) {
        const double d = yi - yr[i];
        v[4] += d * d;
      }
    }
  });
  block_reduce<5>(v, mx);
  if (threadIdx.x == 0) {
    double* p = partials + (size_t)blockIdx.x * NQ;
    p[Q_RP2S] = v[0];
    p[Q_RP2U] = v[1];
    p[Q_RPINF] = v[2];
    p[Q_BY] = v[3];
    p[Q_DY2] = v[4];
  }
}

// warp q sums quantity q over the blocks in a fixed order
__global__ void k_eval_finalize(const double* __restrict__ partials, int nb, EvalSums* __restrict__ out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= NQ) return;
  const bool is_max = (q == Q_RDINF || q == Q_RPINF);
  double acc = 0.0;
  for (int b = lane; b < nb; b += 32) {
    const double v = partials[(size_t)b * NQ + q];
    acc = is_max ? fmax(acc, v) : acc + v;
  }
  acc = is_max ? warp_max(acc) : warp_sum(acc);
  if (lane == 0) out->q[q] = acc;
}

__device__ __forceinline__ void scaled_norms(const EvalSums& e, double& p, double& d, double& g) {
  p = sqrt(e.q[Q_RP2S]);
  d = sqrt(e.q[Q_RD2S]);
  g = fabs(e.q[Q_CX] - e.q[Q_BY]);
}

__device__ __forceinline__ double weighted_kkt(double p, double d, double g, double omega) {
  return sqrt(omega * p * p + d * d / omega + g * g);
}

__global__ void k_init_restart_ref(DevState* st) {
  double p, d, g;
  scaled_norms(st->cur, p, d, g);
  st->rs_p = st->pc_p = p;
  st->rs_d = st->pc_d = d;
  st->rs_g = st->pc_g = g;
}

// One evaluation's decisions (single thread): candidate, termination,
// snapshot schedule (Algorithm 1), restart test, primal-weight update.
__global__ void k_decide(DevState* st, TraceRec* trace) {
  double cp, cd, cg;
  scaled_norms(st->cur, cp, cd, cg);
  int which = KIND_CUR;
  if (st->restarts_on && st->t > 0) {
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
  const double rel = fmax(rel_p, fmax(rel_d, rel_g));
  st->numeric = !(isfinite(rel_p) && isfinite(rel_d) && isfinite(rel_g) && isfinite(cp) && isfinite(cd));
  st->candidate = which;
  st->cand_rel_kkt = rel;

  const int converged = st->tol > 0.0 && rel <= st->tol;
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
  if (snap) st->snapshots += 1;

  int kind = KIND_NONE, apply = APPLY_NONE;
  if (converged) {
    apply = which == KIND_AVG ? APPLY_TAKE_AVG : APPLY_NONE;
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
  if (st->evals < TRACE_CAP) {
    TraceRec& r = trace[st->evals];
    r.iteration = st->k;
    r.kind = kind;
    r.candidate = which;
    r.omega = st->omega;
    r.rel_kkt = rel;
  }
  st->evals += 1;
}

__global__ void k_apply(const DevState* __restrict__ st, double* __restrict__ x, double* __restrict__ y,
                        const double* __restrict__ xa, const double* __restrict__ ya, double* __restrict__ xr,
                        double* __restrict__ yr, double* __restrict__ xs, double* __restrict__ ys, int n, int m) {
  const int mode = st->apply_mode;
  if (mode == APPLY_NONE) return;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) {
      if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG) x[i] = xa[i];
      if (mode != APPLY_TAKE_AVG) {
        xr[i] = x[i];
        xs[i] = 0.0;
      }
    }
    if (i < m) {
      if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG) y[i] = ya[i];
      if (mode != APPLY_TAKE_AVG) {
        yr[i] = y[i];
        ys[i] = 0.0;
      }
    }
  }
}

template <int LPR>
__global__ void __launch_bounds__(TPB) k_pack_dual(Csr At, const double* __restrict__ px, const double* __restrict__ py,
                                                   const double* __restrict__ ch, const double* __restrict__ dc,
                                                   double* __restrict__ ox, double* __restrict__ oz) {
  for_each_row<LPR>(At.rows, [&](int j, bool valid, int gl) {
    const double g = oz ? row_dot<LPR>(At, j, valid, gl, py) : 0.0;
    if (valid && gl == 0) {
      if (ox) ox[j] = dc[j] * px[j];
      if (oz) oz[j] = relu(ch[j] - g) / dc[j];
    }
  });
}

__global__ void k_pack_y(const double* __restrict__ py, const double* __restrict__ dr, double* __restrict__ oy, int m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    oy[i] = dr[i] * py[i];
}

// dispatch on lanes-per-row
#define PDHG_DISPATCH_LPR(lpr, KERNEL, GRID, STREAM, ...)                         \
  switch (lpr) {                                                                 \
    case 1: KERNEL<1><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;             \
    case 2: KERNEL<2><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;             \
    case 4: KERNEL<4><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;             \
    case 8: KERNEL<8><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;             \
    case 16: KERNEL<16><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;           \
    default: KERNEL<32><<<GRID, TPB, 0, STREAM>>>(__VA_ARGS__); break;           \
  }

}  // namespace

int pick_lanes_per_row(double mean_row_len) {
  int l = 1;
  while (l < 32 && l * 1.5 < mean_row_len) l *= 2;
  return l;
}

void launch_row_absmax(const Csr& M, int lpr, double* out, int grid, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lpr, k_row_absmax, grid, s, M, out);
}
void launch_row_abspow_sum(const Csr& M, int lpr, double alpha, double* out, int grid, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lpr, k_row_abspow_sum, grid, s, M, alpha, out);
}
void launch_inv_sqrt_or_one(const double* in, double* out, int len, int grid, cudaStream_t s) {
  k_inv_sqrt_or_one<<<grid, TPB, 0, s>>>(in, out, len);
}
void launch_scale_csr(const Csr& M, int lpr, const double* r, const double* s, int transposed, int grid,
                      cudaStream_t st) {
  PDHG_DISPATCH_LPR(lpr, k_scale_csr, grid, st, M, r, s, transposed);
}
void launch_mul_inplace(double* d, const double* f, int len, int grid, cudaStream_t s) {
  k_mul_inplace<<<grid, TPB, 0, s>>>(d, f, len);
}
void launch_mul(double* out, const double* a, const double* b, int len, int grid, cudaStream_t s) {
  k_mul<<<grid, TPB, 0, s>>>(out, a, b, len);
}
void launch_div(double* out, const double* a, const double* b, int len, int grid, cudaStream_t s) {
  k_div<<<grid, TPB, 0, s>>>(out, a, b, len);
}
void launch_fill(double* v, double val, long long len, int grid, cudaStream_t s) {
  k_fill<<<grid, TPB, 0, s>>>(v, val, len);
}
void launch_spmv(const Csr& M, int lpr, const double* x, double* y, int grid, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lpr, k_spmv, grid, s, M, x, y);
}
void launch_sumsq(const double* v, int len, double* partials, int nb, double* out, cudaStream_t s) {
  k_sumsq_partials<<<nb, TPB, 0, s>>>(v, len, partials);
  k_sum_partials<<<1, 32, 0, s>>>(partials, nb, out);
}
void launch_div_by_norm(double* v, const double* w, const double* s2, int len, int grid, cudaStream_t s) {
  k_div_by_norm<<<grid, TPB, 0, s>>>(v, w, s2, len);
}
void launch_finish_setup(DevState* st, const double* scal, double step_factor, int primal_weight, cudaStream_t s) {
  k_finish_setup<<<1, 1, 0, s>>>(st, scal, step_factor, primal_weight);
}
void launch_primal_step(const Csr& At, int lpr, const double* y, const double* ch, double* x, double* xbar,
                        double* xsum, const DevState* st, int accumulate, int grid, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lpr, k_primal_step, grid, s, At, y, ch, x, xbar, xsum, st, accumulate);
}
void launch_dual_step(const Csr& A, int lpr, const double* xbar, const double* bh, double* y, double* ysum,
                      const DevState* st, int accumulate, int grid, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lpr, k_dual_step, grid, s, A, xbar, bh, y, ysum, st, accumulate);
}
void launch_add_counters(DevState* st, long long dk, cudaStream_t s) { k_add_counters<<<1, 1, 0, s>>>(st, dk); }
void launch_make_average(const double* xs, const double* ys, const double* x, const double* y, double* xa,
                         double* ya, int n, int m, const DevState* st, int grid, cudaStream_t s) {
  k_make_average<<<grid, TPB, 0, s>>>(xs, ys, x, y, xa, ya, n, m, st);
}
void launch_eval_point(const Csr& A, int lprA, const Csr& At, int lprAt, const double* px, const double* py,
                       const double* bh, const double* ch, const double* dr, const double* dc, const double* xr,
                       const double* yr, double* partials, int nb, cudaStream_t s) {
  PDHG_DISPATCH_LPR(lprAt, k_eval_dual, nb, s, At, py, ch, dc, px, xr, partials);
  PDHG_DISPATCH_LPR(lprA, k_eval_primal, nb, s, A, px, bh, dr, py, yr, partials);
}
void launch_eval_finalize(const double* partials, int nb, EvalSums* out, cudaStream_t s) {
  k_eval_finalize<<<1, 32 * NQ, 0, s>>>(partials, nb, out);
}
void launch_init_restart_ref(DevState* st, cudaStream_t s) { k_init_restart_ref<<<1, 1, 0, s>>>(st); }
void launch_decide(DevState* st, TraceRec* trace, cudaStream_t s) { k_decide<<<1, 1, 0, s>>>(st, trace); }
void launch_apply(const DevState* st, double* x, double* y, const double* xa, const double* ya, double* xr,
                  double* yr, double* xs, double* ys, int n, int m, int grid, cudaStream_t s) {
  k_apply<<<grid, TPB, 0, s>>>(st, x, y, xa, ya, xr, yr, xs, ys, n, m);
}
void launch_pack_solution(const Csr& At, int lprAt, const double* px, const double* py, const double* ch,
                          const double* dc, const double* dr, double* ox, double* oy, double* oz, int grid,
                          cudaStream_t s) {
  if (ox || oz) PDHG_DISPATCH_LPR(lprAt, k_pack_dual, grid, s, At, px, py, ch, dc, ox, oz);
  if (oy) k_pack_y<<<grid, TPB, 0, s>>>(py, dr, oy, At.cols);
}

}  // namespace pdhg
