// The whole solve loop of a small LP in one thread block (option
// `persistent`): Algorithm 1's PDHG loop (Section 3.1) without its crossover
// threads, in one launch; the single-block form has no counterpart in the
// paper. One launch runs PDHG iterations, the evaluation of the
// current and average points every eval_every iterations, the restart and
// primal-weight decisions and the termination test, with every vector of the
// LP held in shared memory and the two half-steps separated by block
// barriers only. A batch of small LPs runs one block per LP in the same
// launch; the blocks never wait on one another.
//
// It computes exactly the multi-launch engine's sequence (same layouts, same
// per-row summation order in the half-steps, same decisions); only the order
// in which the evaluation's block partial sums are combined differs, so the
// two agree to rounding. The matrix is read through L1 (__ldg): at these
// sizes both layouts stay in the SM's L1 after the first iteration.
//
// The launch returns when the iteration budget is spent or at an evaluation
// that converged, found a NaN/Inf, or scheduled a snapshot (the host takes
// the snapshot from the vectors written back here and launches again).
#include <cuda_runtime.h>

#include "common.cuh"
#include "decide.cuh"
#include "kernels.cuh"

namespace pdhg {
namespace {

constexpr int PT_NW = PERSIST_TPB / 32;

// Dot products of the rows of units [u0, u1) of H with a vector held in
// shared memory at local indices (global column - base, length len; padding
// entries, whose column index is 0, read 0). op.finish(row, acc) is called
// once per valid row, by the lane that owns it.
struct SharedGather {
  const double* s;
  int base, len;
  __device__ __forceinline__ double operator()(int c) const {
    const unsigned l = (unsigned)(c - base);
    return l < (unsigned)len ? s[l] : 0.0;
  }
};

template <class Op>
__device__ __forceinline__ void cta_dot(const Hyb& H, int u0, int u1, const SharedGather& g, Op& op) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int u = u0 + warp; u < u1; u += PT_NW) {
    const int4 info = __ldg(H.uinfo + u);
    const long long beg = __ldg(H.uoff + u), end = __ldg(H.uoff + u + 1);
    if (info.y == 0) {
      // the step kernels' order: lane L takes entries 2L, 2L+1 of each
      // 64-entry half of a 128-entry step (rows are padded to 4 entries)
      double acc = 0.0;
      for (long long k = beg + 2 * lane; k < end; k += 128) {
        acc += __ldg(H.v + k) * g(__ldg(H.ci + k));
        acc += __ldg(H.v + k + 1) * g(__ldg(H.ci + k + 1));
        if (k + 64 < end) {
          acc += __ldg(H.v + k + 64) * g(__ldg(H.ci + k + 64));
          acc += __ldg(H.v + k + 65) * g(__ldg(H.ci + k + 65));
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) op.finish(info.x, acc);
    } else {
      const int R = info.y;
      const int Lp = (int)((end - beg) / (32 * R));
      for (int q = 0; q < R; ++q) {
        if (32 * q + lane >= info.z) continue;
        double acc = 0.0;
        if (Lp == 1) {
          const long long k = beg + 32 * q + lane;
          acc += __ldg(H.v + k) * g(__ldg(H.ci + k));
        } else {
          // entries 2p, 2p+1 sit side by side: one 8-byte index load and one
          // 16-byte value load per pair, in the step kernels' order
          const long long k0 = beg + 64 * q + 2 * lane;
#pragma unroll 4
          for (int e2 = 0; e2 < (Lp >> 1); ++e2) {
            const long long k = k0 + (long long)e2 * 64 * R;
            const int2 c = __ldg(reinterpret_cast<const int2*>(H.ci + k));
            const double2 a = __ldg(reinterpret_cast<const double2*>(H.v + k));
            acc += a.x * g(c.x);
            acc += a.y * g(c.y);
          }
        }
        op.finish(info.x + 32 * q + lane, acc);
      }
    }
  }
}

// shared-memory vectors of the block's LP, indexed locally
struct Vecs {
  double *x, *xbar, *xsum, *xr, *ch, *idc, *xa;  // n each (idc = 1 / D_c)
  double *y, *ysum, *yr, *bh, *idr, *ya;         // m each (idr = 1 / D_r)
  int x0, n, y0, m;
};

struct PrimalStep {
  Vecs v;
  double tau;
  int accumulate;
  __device__ __forceinline__ void finish(int row, double g) {
    const int j = row - v.x0;
    const double xj = v.x[j];
    const double xn = relu(xj - tau * (v.ch[j] - g));
    v.xbar[j] = 2.0 * xn - xj;
    v.x[j] = xn;
    if (accumulate) v.xsum[j] += xn;
  }
};

struct DualStep {
  Vecs v;
  double sigma;
  int accumulate;
  __device__ __forceinline__ void finish(int row, double h) {
    const int i = row - v.y0;
    const double yn = v.y[i] + sigma * (v.bh[i] - h);
    v.y[i] = yn;
    if (accumulate) v.ysum[i] += yn;
  }
};

// evaluation sums of one point (px, py), in the order of EvalSums
struct EvalDual {
  Vecs v;
  const double* px;
  double* acc;  // [NQ], this thread's partial sums
  __device__ __forceinline__ void finish(int row, double g) {
    const int j = row - v.x0;
    const double c = v.ch[j];
    const double rd = relu(g - c);
    const double zh = relu(c - g);
    const double rdu = rd * v.idc[j];
    const double xj = px[j];
    const double d = xj - v.xr[j];
    acc[Q_RD2S] += rd * rd;
    acc[Q_RD2U] += rdu * rdu;
    acc[Q_RDINF] = fmax(acc[Q_RDINF], fabs(rdu));
    acc[Q_CX] += c * xj;
    acc[Q_XZ] += xj * zh;
    acc[Q_DX2] += d * d;
  }
};

struct EvalPrimal {
  Vecs v;
  const double* py;
  double* acc;
  __device__ __forceinline__ void finish(int row, double h) {
    const int i = row - v.y0;
    const double b = v.bh[i];
    const double rp = b - h;
    const double rpu = rp * v.idr[i];
    const double yi = py[i];
    const double d = yi - v.yr[i];
    acc[Q_RP2S] += rp * rp;
    acc[Q_RP2U] += rpu * rpu;
    acc[Q_RPINF] = fmax(acc[Q_RPINF], fabs(rpu));
    acc[Q_BY] += b * yi;
    acc[Q_DY2] += d * d;
  }
};

__device__ void eval_point(const Hyb& A, const Hyb& At, int ua0, int ua1, int ut0, int ut1, const Vecs& v,
                           const double* px, const double* py, EvalSums* out) {
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  EvalDual od{v, px, acc};
  cta_dot(At, ut0, ut1, SharedGather{py, v.y0, v.m}, od);
  EvalPrimal op{v, py, acc};
  cta_dot(A, ua0, ua1, SharedGather{px, v.x0, v.n}, op);
  bool mx[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) mx[q] = (q == Q_RDINF || q == Q_RPINF);
  block_reduce<NQ>(acc, mx);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) out->q[q] = acc[q];
  }
}

__global__ void __launch_bounds__(PERSIST_TPB, 1)
    k_solve_block(Hyb A, Hyb At, PersistentArgs a, DevState* __restrict__ sts, TraceRec* __restrict__ trace) {
  const int inst = blockIdx.x;
  DevState* st = sts + inst;
  if (st->frozen) return;
  extern __shared__ double sh[];
  Vecs v;
  v.x0 = a.xoff ? a.xoff[inst] : 0;
  v.y0 = a.yoff ? a.yoff[inst] : 0;
  v.n = (a.xoff ? a.xoff[inst + 1] : a.n) - v.x0;
  v.m = (a.yoff ? a.yoff[inst + 1] : a.m) - v.y0;
  const int ua0 = a.ustart ? a.ustart[inst] : 0, ua1 = a.ustart ? a.ustart[inst + 1] : A.n_units;
  const int ut0 = a.ustart ? a.ustart[inst] : 0, ut1 = a.ustart ? a.ustart[inst + 1] : At.n_units;
  // direct offsets into the shared array, so that the compiler keeps shared
  // (not generic) addressing for every vector access
  v.x = sh;
  v.xbar = sh + v.n;
  v.xsum = sh + 2 * v.n;
  v.xr = sh + 3 * v.n;
  v.ch = sh + 4 * v.n;
  v.idc = sh + 5 * v.n;
  v.xa = sh + 6 * v.n;
  v.y = sh + 7 * v.n;
  v.ysum = v.y + v.m;
  v.yr = v.y + 2 * v.m;
  v.bh = v.y + 3 * v.m;
  v.idr = v.y + 4 * v.m;
  v.ya = v.y + 5 * v.m;
  for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
    const int g = v.x0 + j;
    v.x[j] = a.x[g];
    v.xbar[j] = a.xbar[g];
    v.xsum[j] = a.xsum[g];
    v.xr[j] = a.xr[g];
    v.ch[j] = a.ch[g];
    v.idc[j] = a.idc[g];
    v.xa[j] = a.xavg[g];
  }
  for (int i = threadIdx.x; i < v.m; i += blockDim.x) {
    const int g = v.y0 + i;
    v.y[i] = a.y[g];
    v.ysum[i] = a.ysum[g];
    v.yr[i] = a.yr[g];
    v.bh[i] = a.bh[g];
    v.idr[i] = a.idr[g];
    v.ya[i] = a.yavg[g];
  }
  long long k = st->k, t = st->t;
  double tau = st->tau, sigma = st->sigma;
  const int E = a.eval_every;
  __syncthreads();
  if (threadIdx.x == 0) st->snapshot_flag = 0;  // a flag the host has served

  long long done = 0;
  while (done < a.max_iters) {
    const long long nb = a.evaluating ? min((long long)(E - k % E), a.max_iters - done) : a.max_iters - done;
    PrimalStep ps{v, tau, a.restarts};
    DualStep ds{v, sigma, a.restarts};
    for (long long it = 0; it < nb; ++it) {
      cta_dot(At, ut0, ut1, SharedGather{v.y, v.y0, v.m}, ps);
      __syncthreads();
      cta_dot(A, ua0, ua1, SharedGather{v.xbar, v.x0, v.n}, ds);
      __syncthreads();
    }
    k += nb;
    t += nb;
    done += nb;
    if (!(a.evaluating && k % E == 0)) continue;

    // evaluation: the average (restarts on) and the current point
    if (a.restarts) {
      const double it = t > 0 ? 1.0 / (double)t : 0.0;
      for (int j = threadIdx.x; j < v.n; j += blockDim.x) v.xa[j] = t > 0 ? v.xsum[j] * it : v.x[j];
      for (int i = threadIdx.x; i < v.m; i += blockDim.x) v.ya[i] = t > 0 ? v.ysum[i] * it : v.y[i];
      __syncthreads();
      eval_point(A, At, ua0, ua1, ut0, ut1, v, v.xa, v.ya, &st->avg);
    }
    eval_point(A, At, ua0, ua1, ut0, ut1, v, v.x, v.y, &st->cur);
    if (threadIdx.x == 0) {
      st->k = k;
      st->t = t;
      decide_one(st, trace);
      if (a.batch && st->converged) st->frozen = 1;
    }
    __syncthreads();
    const int mode = st->apply_mode;
    if (mode != APPLY_NONE) {
      const bool take_avg = mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG;
      const bool restart = mode != APPLY_TAKE_AVG;
      for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
        if (take_avg) v.x[j] = v.xa[j];
        if (restart) {
          v.xr[j] = v.x[j];
          v.xsum[j] = 0.0;
        }
      }
      for (int i = threadIdx.x; i < v.m; i += blockDim.x) {
        if (take_avg) v.y[i] = v.ya[i];
        if (restart) {
          v.yr[i] = v.y[i];
          v.ysum[i] = 0.0;
        }
      }
    }
    t = st->t;
    tau = st->tau;
    sigma = st->sigma;
    const bool stop = st->converged || st->numeric || st->snapshot_flag;
    __syncthreads();
    if (stop) break;
  }
  if (threadIdx.x == 0) {
    st->k = k;
    st->t = t;
  }
  for (int j = threadIdx.x; j < v.n; j += blockDim.x) {
    const int g = v.x0 + j;
    a.x[g] = v.x[j];
    a.xbar[g] = v.xbar[j];
    a.xsum[g] = v.xsum[j];
    a.xr[g] = v.xr[j];
    a.xavg[g] = v.xa[j];
  }
  for (int i = threadIdx.x; i < v.m; i += blockDim.x) {
    const int g = v.y0 + i;
    a.y[g] = v.y[i];
    a.ysum[g] = v.ysum[i];
    a.yr[g] = v.yr[i];
    a.yavg[g] = v.ya[i];
  }
}

}  // namespace

size_t persistent_smem_bytes(long long n, long long m) { return sizeof(double) * (size_t)(7 * n + 6 * m); }

cudaError_t launch_solve_block(const Hyb& A, const Hyb& At, const PersistentArgs& a, int blocks, size_t smem,
                               DevState* sts, TraceRec* trace, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(k_solve_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_solve_block<<<blocks, PERSIST_TPB, smem, s>>>(A, At, a, sts, trace);
  return cudaGetLastError();
}

}  // namespace pdhg
