// CUDA kernels of the PDHG engine (sm_103a).
//
// They run the "Perform PDHG iteration" step of Algorithm 1 (Section 3.1) on
// the LP pair of Section 2, in the PDLP form the paper's solver follows
// (Section 1, Section 4.1; the paper gives no formula, so the iteration, the
// scaling and the restart scheme are readings), and compute Section 2's
// residuals and relative termination test. The paper notes that PDHG is
// memory-bandwidth bound (Section 5).
//
// The iteration is bandwidth bound: each half-step streams one copy of the
// scaled matrix (Ahat for the dual step, Ahat^T for the primal step) exactly
// once, gathers one vector, and fuses the vector update of the step into the
// epilogue of the row reduction, so the step's vectors are read and written
// once. Tensor cores play no part: SpMV is not a dense contraction.
//
// Cache policy: the matrix is read with no L1 allocation and the L2
// evict-first policy; the step's own vectors are read and written with the
// streaming policy. The vector the next half-step gathers (xbar, written by
// the primal step; y, written by the dual step) is written with the default
// policy, so it stays resident in the 126 MB L2, and the gathers go through
// L1 (which then holds the most frequently gathered entries, numbered first).
#include <math.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "common.cuh"
#include "kernels.cuh"
#include "decide.cuh"
#include "step_ops.cuh"

// Minimum resident blocks per SM requested for the two step kernels. The
// kernels are latency bound, so occupancy matters more than registers: with
// 6 blocks of 256 threads (<= 40 registers; the bound is written for the
// largest block, 512 threads x 3) they ran ~1.9x faster on the
// large LP than with the compiler's free choice (80 registers, 3 blocks).
// The epilogue loads are issued when a row finishes (not prefetched) so the
// 40 registers suffice without spills.
#ifndef PDHG_STEP_MIN_BLOCKS
#define PDHG_STEP_MIN_BLOCKS 6
#endif

namespace pdhg {

namespace {


// ---- cache-policy loads ----------------------------------------------------
__device__ __forceinline__ unsigned long long stream_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ int ld_stream(const int* p, unsigned long long pol) {
  int r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double ld_stream(const double* p, unsigned long long pol) {
  double r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ int2 ld_stream2(const int* p, unsigned long long pol) {
  int2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.s32 {%0, %1}, [%2], %3;"
      : "=r"(r.x), "=r"(r.y)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double2 ld_stream2(const double* p, unsigned long long pol) {
  double2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
      : "=d"(r.x), "=d"(r.y)
      : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_stream(const float* p, unsigned long long pol) {
  float r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float2 ld_stream2(const float* p, unsigned long long pol) {
  float2 r;
  asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
      : "=f"(r.x), "=f"(r.y)
      : "l"(p), "l"(pol));
  return r;
}

// How the row kernels read a layout's column indices: 32-bit (every layout),
// or 16-bit (the panel layout's indices relative to a panel of at most 65536
// rows, half the index bytes). pair(k) reads entries k, k+1 (k even) with one
// load; one(k) reads entry k.
struct IdxI32 {
  const int* __restrict__ p;
  __device__ __forceinline__ int2 pair(long long k, unsigned long long pol) const { return ld_stream2(p + k, pol); }
  __device__ __forceinline__ int one(long long k, unsigned long long pol) const { return ld_stream(p + k, pol); }
};
struct IdxU16 {
  const unsigned short* __restrict__ p;
  __device__ __forceinline__ int2 pair(long long k, unsigned long long pol) const {
    unsigned v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b32 %0, [%1], %2;"
        : "=r"(v)
        : "l"(p + k), "l"(pol));
    return make_int2((int)(v & 0xffffu), (int)(v >> 16));  // entry k in the low half
  }
  __device__ __forceinline__ int one(long long k, unsigned long long pol) const {
    unsigned short v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(p + k), "l"(pol));
    return (int)v;
  }
};
// Scalar visitor (setup kernels): every warp takes units in a grid-stride
// loop; op.entry(acc, k, r) sees every slot k of row r (padding included:
// value 0, column 0), op.finish(r, acc) the combined result (max or sum).
// For long rows only lane 0 calls finish.
// Checked build (PDHG_CHECKED): unit u's entry range lies within the layout's
// slots, its slice shape divides the range, and its rows lie within the
// layout's rows; otherwise the unit is skipped and CHECK_UNIT set. (Padding
// units of a batch have no valid rows and pass.)
__device__ __forceinline__ bool unit_ok(const Hyb& H, int u) {
#ifdef PDHG_CHECKED
  const int4 info = H.uinfo[u];
  const long long b = H.uoff[u], e = H.uoff[u + 1];
  bool ok = 0 <= b && b <= e && e <= H.slots;
  if (info.y == 0)
    ok = ok && info.x >= 0 && info.x < H.rows;
  else
    ok = ok && (info.y == 1 || info.y == 2 || info.y == 4) && (e - b) % (32 * info.y) == 0 && info.z >= 0 &&
         info.z <= 32 * info.y && (info.z == 0 || (info.x >= 0 && (long long)info.x + info.z <= H.rows));
  if (!ok && H.check) atomicOr(H.check, (unsigned)CHECK_UNIT);
  return ok;
#else
  return true;
#endif
}

template <bool MAX, class Op>
__device__ __forceinline__ void hyb_rows(const Hyb& H, Op& op) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((gridDim.x * (unsigned)blockDim.x) >> 5);
  for (int u = gwarp; u < H.n_units; u += nwarps) {
    if (!unit_ok(H, u)) continue;
    const int4 info = H.uinfo[u];
    const long long base = H.uoff[u], end = H.uoff[u + 1];
    if (info.y == 0) {
      double acc = 0.0;
      for (long long k = base + lane; k < end; k += 32) acc = op.entry(acc, k, info.x);
      acc = MAX ? warp_max(acc) : warp_sum(acc);
      if (lane == 0) op.finish(info.x, acc);
    } else {
      const int Lp = (int)((end - base) / (32 * info.y));
      for (int q = 0; q < info.y; ++q) {
        const bool valid = 32 * q + lane < info.z;
        const int r = valid ? info.x + 32 * q + lane : -1;  // -1: padding row
        double acc = 0.0;
        for (int e = 0; e < Lp; ++e) acc = op.entry(acc, slice_slot(base, Lp, info.y, q, e, lane), r);
        if (valid) op.finish(r, acc);
      }
    }
  }
}

// How the dot-product visitor reads the gathered vector: through L1 from
// global memory (GlobalGather), or, for the first `hot` entries, from a
// shared-memory copy (HotGatherT, below).
template <class T>
struct GlobalGather {
  const T* __restrict__ vec;
  __device__ __forceinline__ T operator()(int c) const { return __ldg(vec + c); }
};

// Dot-product visitor (hot path): acc_r = sum over row r of a_rk vec[col_k].
// `op` supplies State begin(r) (its epilogue loads, issued before the row's
// entries) and finish(r, acc, state). Long rows: a warp per row, 4 entries per
// lane per step (two pairs from two contiguous halves). Slices: R rows per thread, 2 entries per load, so a thread
// has 2R independent gathers in flight per step.
// The values have type V and the gathered vector, the products and the sums
// type T (the type the gather returns): V = T, or FP32 values with FP64
// arithmetic (every FP32 value is exactly an FP64 value).
template <class G>
using GatherT = typename std::decay<decltype(std::declval<const G&>()(0))>::type;

template <int R, int UN, class V, class Op, class G, class IX>
__device__ __forceinline__ void slice_dot(const IX& ix, const V* __restrict__ vals, int row0, int nvalid,
                                          long long base, int Lp, const G& gather, Op& op, unsigned long long pol,
                                          int lane) {
  using T = GatherT<G>;
  typename Op::State st[R];
  T acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = row0 + 32 * q + lane;
    if (32 * q + lane < nvalid) st[q] = op.begin(r);
    acc[q] = T(0);
  }
  if (Lp == 1) {
#pragma unroll
    for (int q = 0; q < R; ++q) {
      const long long k = base + 32 * q + lane;
      const int c = ix.one(k, pol);
      acc[q] += as_acc<T>(ld_stream(vals + k, pol)) * gather(c);
    }
  } else {
    const int L2 = Lp >> 1;
    long long k = base + 2 * lane;
#pragma unroll UN
    for (int e2 = 0; e2 < L2; ++e2) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int2 c = ix.pair(k + 64 * q, pol);
        const typename Pair<V>::type a = ld_stream2(vals + k + 64 * q, pol);
        const T g0 = gather(c.x), g1 = gather(c.y);
        acc[q] += as_acc<T>(a.x) * g0;
        acc[q] += as_acc<T>(a.y) * g1;
      }
      k += 64 * R;
    }
  }
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int r = row0 + 32 * q + lane;
    if (32 * q + lane < nvalid) op.finish(r, acc[q], st[q]);
  }
}

// Checked build: a gathered column index outside [0, cols) sets CHECK_COLUMN
// and reads nothing (the product uses 0)
template <class T, class G>
struct CheckedGather {
  G g;
  int cols;
  unsigned* word;
  __device__ __forceinline__ T operator()(int c) const {
    if ((unsigned)c >= (unsigned)cols) {
      if (word) atomicOr(word, (unsigned)CHECK_COLUMN);
      return T(0);
    }
    return g(c);
  }
};

// One unit of H (a long row, or a slice of 32*R rows) for the dot-product
// visitor below.
template <int UN = 2, class V, class Op, class G, class IX>
__device__ __forceinline__ void unit_dot_ix(const Hyb& H, const IX& ix, const V* __restrict__ vals, int u,
                                            const G& gather_in, Op& op, unsigned long long pol, int lane) {
  using T = GatherT<G>;
#ifdef PDHG_CHECKED
  if (!unit_ok(H, u)) return;
  const CheckedGather<T, G> gather{gather_in, H.cols, H.check};
#else
  const G& gather = gather_in;
#endif
  const int4 info = H.uinfo[u];
  const long long beg = H.uoff[u], end = H.uoff[u + 1];
  if (info.y == 0) {
    const int row = info.x;
    typename Op::State st{};
    if (lane == 0) st = op.begin(row);
    T acc = T(0);
    // a step covers 128 entries as two contiguous 64-entry halves; lane L
    // takes entries 2L, 2L+1 of each half, so every load instruction of the
    // warp reads whole sectors (256 B of indices, 512 B of values)
#pragma unroll 2
    for (long long k = beg + 2 * lane; k < end; k += 128) {
      const int2 c0 = ix.pair(k, pol);
      const typename Pair<V>::type a = ld_stream2(vals + k, pol);
      const bool second = k + 64 < end;
      const int2 c1 = second ? ix.pair(k + 64, pol) : make_int2(0, 0);
      typename Pair<V>::type b;
      b.x = V(0);
      b.y = V(0);
      if (second) b = ld_stream2(vals + k + 64, pol);
      const T g0 = gather(c0.x), g1 = gather(c0.y);
      const T g2 = gather(c1.x), g3 = gather(c1.y);
      acc += as_acc<T>(a.x) * g0;
      acc += as_acc<T>(a.y) * g1;
      acc += as_acc<T>(b.x) * g2;
      acc += as_acc<T>(b.y) * g3;
    }
    acc = warp_sum(acc);
    if (lane == 0) op.finish(row, acc, st);
  } else {
    const int Lp = (int)((end - beg) / (32 * info.y));
    if (info.y == 4)
      slice_dot<4, UN>(ix, vals, info.x, info.z, beg, Lp, gather, op, pol, lane);
    else if (info.y == 2)
      slice_dot<2, UN>(ix, vals, info.x, info.z, beg, Lp, gather, op, pol, lane);
    else
      slice_dot<1, UN>(ix, vals, info.x, info.z, beg, Lp, gather, op, pol, lane);
  }
}

// unit u with the layout's 32-bit column indices
template <class V, class Op, class G>
__device__ __forceinline__ void unit_dot(const Hyb& H, const V* __restrict__ vals, int u, const G& gather, Op& op,
                                         unsigned long long pol, int lane) {
  unit_dot_ix(H, IdxI32{H.ci}, vals, u, gather, op, pol, lane);
}

// every unit of H from unit u_begin on, one warp per unit in a grid-stride loop
// over a grid of nblk blocks, of which this block is block bid (by default the
// launch's own grid; the persistent batch solve passes the virtual block it
// stands in for)
template <class V, class Op, class G>
__device__ __forceinline__ void hyb_dot(const Hyb& H, const V* __restrict__ vals, const G& gather, Op& op,
                                        int u_begin = 0, int bid = -1, int nblk = 0) {
  if (bid < 0) {
    bid = (int)blockIdx.x;
    nblk = (int)gridDim.x;
  }
  const unsigned long long pol = stream_policy();
  const int lane = threadIdx.x & 31;
  const int gwarp = (int)(((unsigned)bid * blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)(((unsigned)nblk * blockDim.x) >> 5);
  for (int u = u_begin + gwarp; u < H.n_units; u += nwarps) unit_dot(H, vals, u, gather, op, pol, lane);
}

struct NoState {};

// ---------------------------------------------------------------------------
// setup kernels: Ruiz and Pock-Chambolle scaling, the power iteration for
// ||Ahat||_2 and the step sizes (readings: the paper names its solver's line
// of work, Section 4.1, but not its set-up)
// ---------------------------------------------------------------------------
struct AbsMaxOp {
  const double* __restrict__ v;
  double* __restrict__ out;
  __device__ __forceinline__ double entry(double acc, long long k, int) const { return fmax(acc, fabs(v[k])); }
  __device__ __forceinline__ void finish(int r, double acc) { out[r] = acc; }
};

__global__ void __launch_bounds__(TPB) k_row_absmax(Hyb M, double* __restrict__ out) {
  AbsMaxOp op{M.v, out};
  hyb_rows<true>(M, op);
}

struct AbsPowSumOp {
  const double* __restrict__ v;
  double alpha;
  double* __restrict__ out;
  __device__ __forceinline__ double entry(double acc, long long k, int) const {
    const double a = fabs(v[k]);
    return acc + (alpha == 1.0 ? a : (a > 0.0 ? pow(a, alpha) : 0.0));
  }
  __device__ __forceinline__ void finish(int r, double acc) { out[r] = acc; }
};

__global__ void __launch_bounds__(TPB) k_row_abspow_sum(Hyb M, double alpha, double* __restrict__ out) {
  AbsPowSumOp op{M.v, alpha, out};
  hyb_rows<false>(M, op);
}

struct ScaleOp {
  const int* __restrict__ ci;
  double* __restrict__ v;
  const double* __restrict__ rf;  // row factors of A (length m)
  const double* __restrict__ sf;  // column factors of A (length n)
  int transposed;                 // 0: M is A; 1: M is A^T; 2: M is the panel layout of A^T
  const int* __restrict__ pcol;   // panel layout: column of A of every segment row
  const int* __restrict__ pbase;  // panel layout: first row of A of the segment row's panel
  __device__ __forceinline__ double entry(double acc, long long k, int r) const {
    if (r >= 0) {  // not a padding row
      const int c = ci[k];
      double ri, sj;
      if (transposed == 0) {
        ri = rf[r];
        sj = sf[c];
      } else if (transposed == 1) {
        ri = rf[c];
        sj = sf[r];
      } else {
        ri = rf[pbase[r] + c];
        sj = sf[pcol[r]];
      }
      v[k] = (ri * v[k]) * sj;
    }
    return acc;
  }
  __device__ __forceinline__ void finish(int, double) {}
};

__global__ void __launch_bounds__(TPB) k_scale(Hyb M, const double* __restrict__ r, const double* __restrict__ s,
                                               int transposed, const int* __restrict__ pcol,
                                               const int* __restrict__ pbase) {
  ScaleOp op{M.ci, M.v, r, s, transposed, pcol, pbase};
  hyb_rows<false>(M, op);
}

__global__ void k_inv_sqrt_or_one(const double* __restrict__ in, double* __restrict__ out, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    const double v = in[i];
    out[i] = v > 0.0 ? 1.0 / sqrt(v) : 1.0;
  }
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

__global__ void k_reciprocal(double* __restrict__ out, const double* __restrict__ in, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    out[i] = 1.0 / in[i];
}

__global__ void k_fill(double* __restrict__ v, double val, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    v[i] = val;
}

struct SpmvOp {
  using State = NoState;
  double* __restrict__ out;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int r, double acc, const State&) { out[r] = acc; }
};

__global__ void __launch_bounds__(TPB) k_spmv(Hyb M, const double* __restrict__ x, double* __restrict__ y) {
  SpmvOp op{y};
  hyb_dot(M, M.v, GlobalGather<double>{x}, op);
}

__global__ void __launch_bounds__(TPB) k_sumsq_partials(const double* __restrict__ v, int len,
                                                        double* __restrict__ partials) {
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

__global__ void k_div_by_norm(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ s2,
                              int len) {
  const double s = sqrt(*s2);
  if (!(s > 0.0)) return;
  const double is = 1.0 / s;  // one division per thread: FP64 division is costly on this GPU
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    v[i] = w[i] * is;
}

// scal: [0] = ||Ahat v||^2 of the last power iteration, [1] = ||chat||^2,
// [2] = ||bhat||^2, [3] = ||b||^2, [4] = ||c||^2
__device__ void k_finish_setup_body(DevState* st, const double* __restrict__ scal, double step_factor,
                                    int primal_weight) {
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

__global__ void k_finish_setup(DevState* st, const double* __restrict__ scal, double step_factor, int primal_weight) {
  k_finish_setup_body(st, scal, step_factor, primal_weight);
}

// ---------------------------------------------------------------------------
// the two fused half-steps of one PDHG iteration (Algorithm 1, Section 3.1):
// x' = max(0, x - tau (chat - Ahat^T y)), xbar = 2x' - x, then
// y' = y + sigma (bhat - Ahat xbar)
// ---------------------------------------------------------------------------
// Unscaled values (SC = true; FP32 copies of A's values, FP64 arithmetic):
// the step kernels then gather D_c xbar and D_r y in place of xbar and y,
// since Ahat xbar = D_r (A (D_c xbar)) and Ahat^T y = D_c (A^T (D_r y)); the
// primal step scales its row sums by D_c and writes D_c xbar, the dual step
// scales its row sums by D_r and writes D_r y' beside y'. SC = false: the
// scaled values, and dsc / yg are unused.
template <class T, bool SC>
struct ColScale {
  const T* __restrict__ d;
  __device__ __forceinline__ T load(int j) const { return SC ? __ldcs(d + j) : T(1); }
  __device__ __forceinline__ T apply(T d_j, T v) const { return SC ? d_j * v : v; }
};

// The primal projection max(0, v), or with option refine32 (FP32 phases on
// corrections to an FP64 restart point x_r) max(lo_j, v), lo = -x_r rounded
// toward zero, so that x_r + v stays >= 0. NaN passes through either way.
template <class T>
__device__ __forceinline__ T project(const T* __restrict__, int, T v) {
  return relu(v);
}
template <>
__device__ __forceinline__ float project<float>(const float* __restrict__ lo, int j, float v) {
  if (!lo) return relu(v);
  const float l = __ldcs(lo + j);
  return v < l ? l : v;
}

template <class T, bool SC = false>
struct PrimalOp {
  using State = NoState;
  const T* __restrict__ ch;
  T* __restrict__ x;
  T* __restrict__ xbar;
  T* __restrict__ xsum;
  T tau;
  int accumulate;
  ColScale<T, SC> dc;
  const T* __restrict__ lo;  // option refine32 (FP32): lower bounds of the corrections; nullptr: 0
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, T g, const State&) {
    const T d = dc.load(j);
    const T xj = __ldcs(x + j);
    // every load before the first store: the compiler keeps loads after
    // stores to other arrays (it cannot tell that they do not overlap), so a
    // load placed after a store waits for it; the order measured 1.5-2.6%
    // faster
    const T cj = __ldcs(ch + j);
    const T sj = accumulate ? __ldcs(xsum + j) : T(0);
    const T xn = project(lo, j, xj - tau * (cj - dc.apply(d, g)));
    xbar[j] = dc.apply(d, T(2) * xn - xj);  // default policy: gathered by the dual step next
    __stcs(x + j, xn);
    if (accumulate) __stcs(xsum + j, sj + xn);
  }
};

// State of the problem a block works on: a batch maps every block to one
// instance (binst); a single problem has binst == nullptr.
__device__ __forceinline__ const DevState* block_state(const DevState* sts, const int* binst) {
  return binst ? sts + binst[blockIdx.x] : sts;
}

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_primal_step(Hyb At, const V* __restrict__ vals, const T* __restrict__ y, const T* __restrict__ ch,
                  T* __restrict__ x, T* __restrict__ xbar, T* __restrict__ xsum, const DevState* __restrict__ sts,
                  const int* __restrict__ binst, int accumulate, int u_begin, const T* __restrict__ dsc,
                  const T* __restrict__ lo) {
  const DevState* st = block_state(sts, binst);
  if (st->frozen) return;
  PrimalOp<T, !std::is_same<T, V>::value> op{ch, x, xbar, xsum, (T)st->tau, accumulate, {dsc}, lo};
  hyb_dot(At, vals, GlobalGather<T>{y}, op, u_begin);
}

// The same, computed by one thread of the block and shared: an FP64 division
// in every thread of a step kernel would cost the FP64 pipe more than a
// hundred of the step's multiply-adds per row. Every thread of the block
// must call it.
__device__ __forceinline__ double block_halpern_weight(const DevState* st, int it) {
  __shared__ double w_shared;
  if (threadIdx.x == 0) w_shared = halpern_weight(st, it);
  __syncthreads();
  return w_shared;
}

// ---- panel-tiled primal half-step (option primal_panels) --------------------
// The rows of A^T are cut into segments by panels of panel_rows consecutive
// entries of y. Pass 1: every block stages one panel of y in shared memory and
// reduces its panel's segments (Hyb layout Pn, local row indices) with the
// gathers served from shared memory, writing one partial sum per segment at
// its column-major position. Pass 2: one thread per column adds its partial
// sums in panel order and applies the primal update. The random gathers of y
// that bound k_primal_step (one L2 request each) become shared-memory reads,
// and the L2 traffic left is the partial sums' writes and coalesced reads.
template <class T>
struct SmemGather {
  const T* s;
  __device__ __forceinline__ T operator()(int c) const { return s[c]; }
};

// the output position of a segment row is loaded when the row starts, so its
// latency overlaps the entries' loads
template <class T>
struct PartialOp {
  struct State {
    int pos;
  };
  T* __restrict__ partial;
  const int* __restrict__ segout;
  __device__ __forceinline__ State begin(int r) { return {__ldg(segout + r)}; }
  __device__ __forceinline__ void finish(int, T acc, const State& st) { partial[st.pos] = acc; }
};

// FP32 panels take half the shared memory, so two blocks could share an SM
template <class T, class V = T, bool I16 = false>
__global__ void __launch_bounds__(PANEL_TPB, sizeof(T) == 4 ? PANEL_MINB32 : 1)
    k_primal_panels(Hyb Pn, const V* __restrict__ vals, const T* __restrict__ y, const int* __restrict__ pfirst,
                    const int4* __restrict__ binfo, const int* __restrict__ ustart, const int* __restrict__ segout,
                    T* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T* ys = reinterpret_cast<T*>(panel_smem);
  // the short-column step launched after this pass may start on SMs as their
  // panel blocks finish (programmatic dependent launch; see short_and_combine)
  asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
  // panels get blocks in proportion to their stored entries (the first panels,
  // holding the longest rows of A, have the most)
  const int4 bi = binfo[blockIdx.x];
  const int p = bi.x, sub = bi.y, kpp = bi.z;
  const int i0 = pfirst[p], len = pfirst[p + 1] - i0;
  // the panel of y into shared memory with asynchronous 16-byte copies, all in
  // flight at once, when the panel starts on a 16-byte boundary (the default
  // panel height is a multiple of 16 entries); the rest with plain loads
  {
    constexpr int PER = 16 / (int)sizeof(T);
    const T* src = y + i0;
    const int nv = (reinterpret_cast<unsigned long long>(src) & 15ull) == 0 ? len / PER : 0;
    const unsigned dst0 = (unsigned)__cvta_generic_to_shared(ys);
    for (int v = threadIdx.x; v < nv; v += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst0 + 16u * (unsigned)v), "l"(src + v * PER)
                   : "memory");
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    for (int t = nv * PER + threadIdx.x; t < len; t += blockDim.x) ys[t] = src[t];
    asm volatile("cp.async.wait_all;\n" ::: "memory");
  }
  __syncthreads();
  const unsigned long long pol = stream_policy();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  PartialOp<T> op{partial, segout};
  // the panel's units (sorted by decreasing length) are dealt to its blocks'
  // warps in rounds of W, alternately forwards and backwards, so that no warp
  // (and no block) gets the longest unit of every round
  const int ub = ustart[p], cnt = ustart[p + 1] - ub, W = kpp * nw, g = sub * nw + (threadIdx.x >> 5);
  for (int r0 = 0, fwd = 1; r0 < cnt; r0 += W, fwd ^= 1) {
    const int o = r0 + (fwd ? g : W - 1 - g);
    if (o >= cnt) continue;
    if (I16)
      unit_dot_ix<sizeof(T) == 4 ? PANEL_UNROLL32 : PANEL_UNROLL64>(Pn, IdxU16{Pn.ci16}, vals, ub + o,
                                                                    SmemGather<T>{ys}, op, pol, lane);
    else
      unit_dot(Pn, vals, ub + o, SmemGather<T>{ys}, op, pol, lane);
  }
}

// ---- reflected Halpern form of the two half-steps (option halpern) ----------
// (the cuPDLP+ line the paper's solver follows, Section 4.1; a reading, as the
// paper gives no formula)
// With (x~, y~) the PDHG map's output, w = (t + 1) / (t + 2) (t = iterations
// since the last restart, before this step) and the last restart point
// (xr, yr) as anchor: x <- w ((1 + rho) x~ - rho x) + (1 - w) xr, likewise y;
// the dual step still gathers xbar = 2 x~ - x.
template <class T, bool SC = false, bool R1 = false>
struct PrimalHalpernOp {
  using State = NoState;
  const T* __restrict__ ch;
  T* __restrict__ x;
  T* __restrict__ xbar;
  const T* __restrict__ xr;
  T tau, w, rho;
  ColScale<T, SC> dc;
  const T* __restrict__ lo;  // option refine32 (FP32): lower bounds of the corrections; nullptr: 0
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, T g, const State&) {
    const T d = dc.load(j);
    const T xj = __ldcs(x + j);
    // (the loads stay in this order: placed before the stores, as in
    // PrimalOp, they changed the compiler's FP32 contractions here, and with
    // them the bit-identity with the streamed kernels, for no measured gain)
    const T xt = project(lo, j, xj - tau * (__ldcs(ch + j) - dc.apply(d, g)));
    const T xb = T(2) * xt - xj;
    xbar[j] = dc.apply(d, xb);
    __stcs(x + j, halpern_mix_r<R1>(xt, xj, xb, __ldcs(xr + j), w, T(1) - w, rho));
  }
};

template <class T, bool SC = false, bool R1 = false>
struct DualHalpernOp {
  using State = NoState;
  const T* __restrict__ bh;
  T* __restrict__ y;
  const T* __restrict__ yr;
  T sigma, w, rho;
  ColScale<T, SC> dr;
  T* __restrict__ yg;  // SC: D_r y', gathered by the primal step next
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int i, T h, const State&) {
    const T d = dr.load(i);
    const T yi = y[i];
    const T yt = yi + sigma * (__ldcs(bh + i) - dr.apply(d, h));
    const T yn = halpern_mix_r<R1>(yt, yi, T(2) * yt - yi, __ldcs(yr + i), w, T(1) - w, rho);
    y[i] = yn;
    if (SC) yg[i] = d * yn;
  }
};

// ---- the short columns' direct step fused with the long columns' combine ---
// Pass 2 of the panel-tiled primal half-step: blocks [0, cblocks) add each long
// column's panel-major partial sums (panel p of column j at p * ncols + j,
// zero where the column has no entry in the panel; added in panel order with
// eight loads in flight) and apply the update through the same op as the
// direct step; the other blocks run the direct step over the short columns
// (the units of At from u_begin on). One launch instead of two, so the
// combine's latency-bound work overlaps the direct step.
template <class T, class V, class Op>
__device__ __forceinline__ void short_and_combine(const Hyb& At, const V* __restrict__ vals, const T* __restrict__ y,
                                                  Op& op, int u_begin, int cblocks, int panels,
                                                  const T* __restrict__ partial, int ncols, int cfirst) {
  // blocks [cfirst, cfirst + cblocks) combine the long columns, the others
  // step the short columns; cfirst is about one wave of blocks, so that the
  // combine (latency bound) overlaps short-column work and, when this launch
  // overlaps the panel pass (programmatic dependent launch), is scheduled
  // once the panel pass has (nearly) finished
  const int sblocks = (int)gridDim.x - cblocks;
  const int bx = (int)blockIdx.x;
  if (bx >= cfirst && bx < cfirst + cblocks) {
    // the partial sums of the panel pass: wait for it (returns at once when
    // the launch is not a programmatic dependent one)
    asm volatile("griddepcontrol.wait;\n" ::: "memory");
    const int cb = bx - cfirst;
    for (int j = cb * blockDim.x + threadIdx.x; j < ncols; j += cblocks * blockDim.x) {
      const typename Op::State sj = op.begin(j);
      const T* pj = partial + j;
      T g = T(0);
      int p = 0;
      for (; p + 8 <= panels; p += 8) {
        T a[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) a[e] = __ldcs(pj + (long long)(p + e) * ncols);
#pragma unroll
        for (int e = 0; e < 8; ++e) g += a[e];
      }
      for (; p < panels; ++p) g += __ldcs(pj + (long long)p * ncols);
      op.finish(j, g, sj);
    }
    return;
  }
  // the short columns: they read y (the dual step's, complete before the
  // panel pass began) and write only their own columns, so they may run
  // beside the panel pass's last blocks
  const unsigned long long pol = stream_policy();
  const int lane = threadIdx.x & 31;
  const int sb = bx < cfirst ? bx : bx - cblocks;  // index among the short-column blocks
  const int gwarp = (int)((sb * (unsigned)blockDim.x + threadIdx.x) >> 5);
  const int nwarps = (int)((sblocks * (unsigned)blockDim.x) >> 5);
  for (int u = u_begin + gwarp; u < At.n_units; u += nwarps) unit_dot(At, vals, u, GlobalGather<T>{y}, op, pol, lane);
}

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_primal_short_combine(Hyb At, const V* __restrict__ vals, const T* __restrict__ y, const T* __restrict__ ch,
                           T* __restrict__ x, T* __restrict__ xbar, T* __restrict__ xsum,
                           const DevState* __restrict__ st, int accumulate, int u_begin, int cblocks, int panels,
                           const T* __restrict__ partial, int ncols, int cfirst, const T* __restrict__ dsc,
                           const T* __restrict__ lo) {
  PrimalOp<T, !std::is_same<T, V>::value> op{ch, x, xbar, xsum, (T)st->tau, accumulate, {dsc}, lo};
  short_and_combine(At, vals, y, op, u_begin, cblocks, panels, partial, ncols, cfirst);
}

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_primal_step_halpern(Hyb At, const V* __restrict__ vals, const T* __restrict__ y, const T* __restrict__ ch,
                          T* __restrict__ x, T* __restrict__ xbar, const T* __restrict__ xr,
                          const DevState* __restrict__ sts, const int* __restrict__ binst, int it, int u_begin,
                          const T* __restrict__ dsc, const T* __restrict__ lo) {
  const DevState* st = block_state(sts, binst);
  if (st->frozen) return;
  constexpr bool SC = !std::is_same<T, V>::value;
  const T w = (T)block_halpern_weight(st, it), rho = (T)st->rho;
  if (rho == T(1)) {  // the reflection of the default form, known to every entry's update
    PrimalHalpernOp<T, SC, true> op{ch, x, xbar, xr, (T)st->tau, w, rho, {dsc}, lo};
    hyb_dot(At, vals, GlobalGather<T>{y}, op, u_begin);
  } else {
    PrimalHalpernOp<T, SC, false> op{ch, x, xbar, xr, (T)st->tau, w, rho, {dsc}, lo};
    hyb_dot(At, vals, GlobalGather<T>{y}, op, u_begin);
  }
}

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_primal_short_combine_halpern(Hyb At, const V* __restrict__ vals, const T* __restrict__ y,
                                   const T* __restrict__ ch, T* __restrict__ x, T* __restrict__ xbar,
                                   const T* __restrict__ xr, const DevState* __restrict__ st, int it, int u_begin,
                                   int cblocks, int panels, const T* __restrict__ partial, int ncols, int cfirst,
                                   const T* __restrict__ dsc, const T* __restrict__ lo) {
  constexpr bool SC = !std::is_same<T, V>::value;
  const T w = (T)block_halpern_weight(st, it), rho = (T)st->rho;
  if (rho == T(1)) {
    PrimalHalpernOp<T, SC, true> op{ch, x, xbar, xr, (T)st->tau, w, rho, {dsc}, lo};
    short_and_combine(At, vals, y, op, u_begin, cblocks, panels, partial, ncols, cfirst);
  } else {
    PrimalHalpernOp<T, SC, false> op{ch, x, xbar, xr, (T)st->tau, w, rho, {dsc}, lo};
    short_and_combine(At, vals, y, op, u_begin, cblocks, panels, partial, ncols, cfirst);
  }
}

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_dual_step_halpern(Hyb A, const V* __restrict__ vals, const T* __restrict__ xbar, const T* __restrict__ bh,
                        T* __restrict__ y, const T* __restrict__ yr, const DevState* __restrict__ sts,
                        const int* __restrict__ binst, int it, const T* __restrict__ dsc, T* __restrict__ yg) {
  const DevState* st = block_state(sts, binst);
  if (st->frozen) return;
  constexpr bool SC = !std::is_same<T, V>::value;
  const T w = (T)block_halpern_weight(st, it), rho = (T)st->rho;
  if (rho == T(1)) {
    DualHalpernOp<T, SC, true> op{bh, y, yr, (T)st->sigma, w, rho, {dsc}, yg};
    hyb_dot(A, vals, GlobalGather<T>{xbar}, op);
  } else {
    DualHalpernOp<T, SC, false> op{bh, y, yr, (T)st->sigma, w, rho, {dsc}, yg};
    hyb_dot(A, vals, GlobalGather<T>{xbar}, op);
  }
}

template <class T, bool SC = false>
struct DualOp {
  using State = NoState;
  const T* __restrict__ bh;
  T* __restrict__ y;
  T* __restrict__ ysum;
  T sigma;
  int accumulate;
  ColScale<T, SC> dr;
  T* __restrict__ yg;  // SC: D_r y', gathered by the primal step next
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int i, T h, const State&) {
    const T d = dr.load(i);
    const T yi = y[i], bi = __ldcs(bh + i);  // every load before the first store (see PrimalOp)
    const T si = accumulate ? __ldcs(ysum + i) : T(0);
    const T yn = yi + sigma * (bi - dr.apply(d, h));
    y[i] = yn;  // default policy: gathered by the primal step next (SC: yg is)
    if (SC) yg[i] = d * yn;
    if (accumulate) __stcs(ysum + i, si + yn);
  }
};

template <class T, class V = T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_dual_step(Hyb A, const V* __restrict__ vals, const T* __restrict__ xbar, const T* __restrict__ bh,
                T* __restrict__ y, T* __restrict__ ysum, const DevState* __restrict__ sts,
                const int* __restrict__ binst, int accumulate, const T* __restrict__ dsc, T* __restrict__ yg) {
  const DevState* st = block_state(sts, binst);
  if (st->frozen) return;
  DualOp<T, !std::is_same<T, V>::value> op{bh, y, ysum, (T)st->sigma, accumulate, {dsc}, yg};
  hyb_dot(A, vals, GlobalGather<T>{xbar}, op);
}

// The dual step as a persistent kernel (one HOT_TPB-thread block per SM) that
// first copies xbar[0, hot) into shared memory. With the variables numbered by
// decreasing column length, these are the most frequently gathered entries
// (on the large Zipf LP the first 27,648 columns hold 55% of A's entries, the
// first 56,320 hold 75%), and their gathers then stay off the L1-to-L2
// request path that bounds the random gathers; the others go through L1.
// The copy is issued as 16-byte cp.async transfers, all in flight at once.
template <class T>
struct HotGatherT {
  const T* __restrict__ vec;
  const T* hot_vals;  // shared memory copy of vec[0, hot)
  int hot;
  __device__ __forceinline__ T operator()(int c) const { return c < hot ? hot_vals[c] : __ldg(vec + c); }
};

template <class T>
__device__ __forceinline__ const T* stage_hot(const T* __restrict__ xbar, int hot) {
  extern __shared__ __align__(16) unsigned char hot_smem[];
  T* sh = reinterpret_cast<T*>(hot_smem);
  constexpr int PER = 16 / (int)sizeof(T);
  const int nv = (reinterpret_cast<unsigned long long>(xbar) & 15ull) == 0 ? hot / PER : 0;
  const unsigned dst0 = (unsigned)__cvta_generic_to_shared(sh);
  for (int v = threadIdx.x; v < nv; v += blockDim.x)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst0 + 16u * (unsigned)v), "l"(xbar + v * PER)
                 : "memory");
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int t = nv * PER + threadIdx.x; t < hot; t += blockDim.x) sh[t] = xbar[t];
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  __syncthreads();
  return sh;
}

template <class T>
__global__ void __launch_bounds__(HOT_TPB, 1)
    k_dual_step_hot(Hyb A, const T* __restrict__ vals, const T* __restrict__ xbar, int hot,
                    const T* __restrict__ bh, T* __restrict__ y, T* __restrict__ ysum,
                    const DevState* __restrict__ st, int accumulate) {
  const T* sh = stage_hot(xbar, hot);
  DualOp<T> op{bh, y, ysum, (T)st->sigma, accumulate};
  hyb_dot(A, vals, HotGatherT<T>{xbar, sh, hot}, op);
}

template <class T>
__global__ void __launch_bounds__(HOT_TPB, 1)
    k_dual_step_hot_halpern(Hyb A, const T* __restrict__ vals, const T* __restrict__ xbar, int hot,
                            const T* __restrict__ bh, T* __restrict__ y, const T* __restrict__ yr,
                            const DevState* __restrict__ st, int it) {
  const T* sh = stage_hot(xbar, hot);
  const T w = (T)block_halpern_weight(st, it), rho = (T)st->rho;
  if (rho == T(1)) {  // as k_dual_step_halpern: the reflection known at compile time
    DualHalpernOp<T, false, true> op{bh, y, yr, (T)st->sigma, w, rho};
    hyb_dot(A, vals, HotGatherT<T>{xbar, sh, hot}, op);
  } else {
    DualHalpernOp<T, false, false> op{bh, y, yr, (T)st->sigma, w, rho};
    hyb_dot(A, vals, HotGatherT<T>{xbar, sh, hot}, op);
  }
}

__global__ void k_add_counters(DevState* st, long long dk) {
  st->k += dk;
  st->t += dk;
}

// ---------------------------------------------------------------------------
// evaluation: Section 2's residuals r_P = b - A x and r_D = A^T y + z - c with
// z = max(0, c - A^T y), the objectives, the gap and x^T z, for the current
// point and the average, on the problem as given; Algorithm 1's "maxresid" is
// the largest of the three relative measures (Section 3.1)
// ---------------------------------------------------------------------------
__global__ void k_make_average(const double* __restrict__ xs, const double* __restrict__ ys,
                               const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ xa,
                               double* __restrict__ ya, int n, int m, const DevState* __restrict__ st) {
  const long long t = st->t;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;  // one division; FP64 division is costly on this GPU
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) xa[i] = t > 0 ? xs[i] * it : x[i];
    if (i < m) ya[i] = t > 0 ? ys[i] * it : y[i];
  }
}

struct EvalDualOp {
  using State = NoState;
  const double* __restrict__ ch;
  const double* __restrict__ idc;  // 1 / D_c
  const double* __restrict__ px;
  const double* __restrict__ xr;
  // fixed-point residual scheme (xt != null): the primal part of the PDHG step
  // from this point, x~ = max(0, x - tau (chat - g)), is written to xt
  double tau = 0.0;
  double* __restrict__ xt = nullptr;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, double g, const State&) {
    const double c = ch[j];
    const double rd = relu(g - c);
    const double zh = relu(c - g);
    const double rdu = rd * idc[j];
    const double xj = px[j];
    acc[0] += rd * rd;
    acc[1] += rdu * rdu;
    acc[2] = fmax(acc[2], fabs(rdu));
    acc[3] += c * xj;
    acc[4] += xj * zh;
    if (xr) {
      const double d = xj - xr[j];
      acc[5] += d * d;
    }
    if (xt) {
      const double x1 = relu(xj - tau * (c - g));
      xt[j] = x1;
      const double d = x1 - xj, dr = x1 - xr[j];
      acc[6] += d * d;
      acc[7] += dr * dr;
    }
  }
};

// the evaluation partial sums of the rows of At in block bid of nblk (one
// row of partials per block; blocks of a frozen batch instance write zeros)
template <class G>
__device__ __forceinline__ void eval_dual_block(const Hyb& At, const G& gather_py, const double* __restrict__ ch,
                                                const double* __restrict__ idc, const double* __restrict__ px,
                                                const double* __restrict__ xr, double* __restrict__ partials,
                                                bool frozen, int bid, int nblk, double tau = 0.0,
                                                double* __restrict__ xt = nullptr) {
  if (frozen) {
    if (threadIdx.x < 6) partials[(size_t)bid * NQ + Q_RD2S + threadIdx.x] = 0.0;
    if (threadIdx.x < 2) partials[(size_t)bid * NQ + Q_FX2 + threadIdx.x] = 0.0;
    return;
  }
  EvalDualOp op;
  op.ch = ch;
  op.idc = idc;
  op.px = px;
  op.xr = xr;
  op.tau = tau;
  op.xt = xt;
  hyb_dot(At, At.v, gather_py, op, 0, bid, nblk);
  const bool mx[8] = {false, false, true, false, false, false, false, false};
  block_reduce<8>(op.acc, mx);
  if (threadIdx.x == 0) {
    double* p = partials + (size_t)bid * NQ;
    p[Q_RD2S] = op.acc[0];
    p[Q_RD2U] = op.acc[1];
    p[Q_RDINF] = op.acc[2];
    p[Q_CX] = op.acc[3];
    p[Q_XZ] = op.acc[4];
    p[Q_DX2] = op.acc[5];
    p[Q_FX2] = op.acc[6];
    p[Q_FXR2] = op.acc[7];
  }
}

__global__ void __launch_bounds__(STEP_TPB_MAX) k_eval_dual(Hyb At, const double* __restrict__ py,
                                                   const double* __restrict__ ch, const double* __restrict__ idc,
                                                   const double* __restrict__ px, const double* __restrict__ xr,
                                                   double* __restrict__ partials, const DevState* __restrict__ sts,
                                                   const int* __restrict__ binst) {
  eval_dual_block(At, GlobalGather<double>{py}, ch, idc, px, xr, partials, binst && sts[binst[blockIdx.x]].frozen,
                  (int)blockIdx.x, (int)gridDim.x);
}

struct EvalPrimalOp {
  using State = NoState;
  const double* __restrict__ bh;
  const double* __restrict__ idr;  // 1 / D_r
  const double* __restrict__ py;
  const double* __restrict__ yr;
  // fixed-point residual scheme (ht != null): ht = Ahat x~; the dual part of
  // the PDHG step, y~ = y + sigma (bhat - (2 Ahat x~ - Ahat x)), is written to yt
  double sigma = 0.0;
  const double* __restrict__ ht = nullptr;
  double* __restrict__ yt = nullptr;
  double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int i, double h, const State&) {
    const double b = bh[i];
    const double rp = b - h;
    const double rpu = rp * idr[i];
    const double yi = py[i];
    acc[0] += rp * rp;
    acc[1] += rpu * rpu;
    acc[2] = fmax(acc[2], fabs(rpu));
    acc[3] += b * yi;
    if (yr) {
      const double d = yi - yr[i];
      acc[4] += d * d;
    }
    if (ht) {
      const double h1 = ht[i];
      const double y1 = yi + sigma * (b - (2.0 * h1 - h));
      yt[i] = y1;
      const double d = y1 - yi, dr = y1 - yr[i];
      acc[5] += d * d;
      acc[6] += d * (h1 - h);
      acc[7] += dr * dr;
    }
  }
};

template <class G>
__device__ __forceinline__ void eval_primal_block(const Hyb& A, const G& gather_px, const double* __restrict__ bh,
                                                  const double* __restrict__ idr, const double* __restrict__ py,
                                                  const double* __restrict__ yr, double* __restrict__ partials,
                                                  bool frozen, int bid, int nblk, double sigma = 0.0,
                                                  const double* __restrict__ ht = nullptr,
                                                  double* __restrict__ yt = nullptr) {
  if (frozen) {
    if (threadIdx.x < 5) partials[(size_t)bid * NQ + Q_RP2S + threadIdx.x] = 0.0;
    if (threadIdx.x < 3) partials[(size_t)bid * NQ + Q_FY2 + threadIdx.x] = 0.0;
    return;
  }
  EvalPrimalOp op;
  op.bh = bh;
  op.idr = idr;
  op.py = py;
  op.yr = yr;
  op.sigma = sigma;
  op.ht = ht;
  op.yt = yt;
  hyb_dot(A, A.v, gather_px, op, 0, bid, nblk);
  const bool mx[8] = {false, false, true, false, false, false, false, false};
  block_reduce<8>(op.acc, mx);
  if (threadIdx.x == 0) {
    double* p = partials + (size_t)bid * NQ;
    p[Q_RP2S] = op.acc[0];
    p[Q_RP2U] = op.acc[1];
    p[Q_RPINF] = op.acc[2];
    p[Q_BY] = op.acc[3];
    p[Q_DY2] = op.acc[4];
    p[Q_FY2] = op.acc[5];
    p[Q_FXY] = op.acc[6];
    p[Q_FYR2] = op.acc[7];
  }
}

__global__ void __launch_bounds__(STEP_TPB_MAX) k_eval_primal(Hyb A, const double* __restrict__ px,
                                                     const double* __restrict__ bh, const double* __restrict__ idr,
                                                     const double* __restrict__ py, const double* __restrict__ yr,
                                                     double* __restrict__ partials, const DevState* __restrict__ sts,
                                                     const int* __restrict__ binst) {
  eval_primal_block(A, GlobalGather<double>{px}, bh, idr, py, yr, partials,
                    binst && sts[binst[blockIdx.x]].frozen, (int)blockIdx.x, (int)gridDim.x);
}

// the evaluation of the current point with the fixed-point residual's parts
// (restart_scheme = 1, single LPs): the dual pass also writes x~, the primal
// pass (after ht = Ahat x~) also writes y~
__global__ void __launch_bounds__(STEP_TPB_MAX) k_eval_dual_fp(Hyb At, const double* __restrict__ py,
                                                      const double* __restrict__ ch, const double* __restrict__ idc,
                                                      const double* __restrict__ px, const double* __restrict__ xr,
                                                      double* __restrict__ partials, const DevState* __restrict__ st,
                                                      double* __restrict__ xt) {
  eval_dual_block(At, GlobalGather<double>{py}, ch, idc, px, xr, partials, false, (int)blockIdx.x, (int)gridDim.x,
                  st->tau, xt);
}
__global__ void __launch_bounds__(STEP_TPB_MAX) k_eval_primal_fp(Hyb A, const double* __restrict__ px,
                                                        const double* __restrict__ bh,
                                                        const double* __restrict__ idr,
                                                        const double* __restrict__ py, const double* __restrict__ yr,
                                                        double* __restrict__ partials,
                                                        const DevState* __restrict__ st,
                                                        const double* __restrict__ ht, double* __restrict__ yt) {
  eval_primal_block(A, GlobalGather<double>{px}, bh, idr, py, yr, partials, false, (int)blockIdx.x, (int)gridDim.x,
                    st->sigma, ht, yt);
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

__global__ void k_init_restart_ref(DevState* st) {
  double p, d, g;
  scaled_norms(st->cur, p, d, g);
  st->rs_p = st->pc_p = p;
  st->rs_d = st->pc_d = d;
  st->rs_g = st->pc_g = g;
  st->r_restart = st->r_prev = fixed_residual(st->cur, st->tau, st->sigma);  // 0 unless evaluated with it
}

__global__ void k_decide(DevState* st, TraceRec* trace) { decide_one(st, trace); }

// ---------------------------------------------------------------------------
// batch: per-instance counterparts (instance = blockIdx.y for vector kernels,
// one thread per instance for scalar kernels); many independent LPs at once,
// each following the single-LP method (no counterpart in the paper)
// ---------------------------------------------------------------------------
__global__ void k_decide_b(DevState* sts, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  if (sts[i].frozen) {
    sts[i].snapshot_flag = 0;  // an instance that stopped schedules no snapshot
    return;
  }
  decide_one(sts + i, nullptr);
  if (sts[i].converged) sts[i].frozen = 1;
}

__global__ void k_add_counters_b(DevState* sts, int count, long long dk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count || sts[i].frozen) return;
  sts[i].k += dk;
  sts[i].t += dk;
}

__global__ void k_init_restart_ref_b(DevState* sts, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  double p, d, g;
  scaled_norms(sts[i].cur, p, d, g);
  sts[i].rs_p = sts[i].pc_p = p;
  sts[i].rs_d = sts[i].pc_d = d;
  sts[i].rs_g = sts[i].pc_g = g;
}

// per-instance sums of the per-block partials (blocks [bstart[i], bstart[i+1]))
// into *(EvalSums*)((char*)out + i * stride)
__global__ void k_eval_finalize_b(const double* __restrict__ partials, const int* __restrict__ bstart, char* out,
                                  size_t stride) {
  const int i = blockIdx.x;
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= NQ) return;
  const bool is_max = (q == Q_RDINF || q == Q_RPINF);
  double acc = 0.0;
  for (int b = bstart[i] + lane; b < bstart[i + 1]; b += 32) {
    const double v = partials[(size_t)b * NQ + q];
    acc = is_max ? fmax(acc, v) : acc + v;
  }
  acc = is_max ? warp_max(acc) : warp_sum(acc);
  if (lane == 0) reinterpret_cast<EvalSums*>(out + (size_t)i * stride)->q[q] = acc;
}

__global__ void k_make_average_b(const double* __restrict__ xs, const double* __restrict__ ys,
                                 const double* __restrict__ x, const double* __restrict__ y, double* __restrict__ xa,
                                 double* __restrict__ ya, const int* __restrict__ xoff, const int* __restrict__ yoff,
                                 const DevState* __restrict__ sts) {
  const int i = blockIdx.y;
  if (sts[i].frozen) return;
  const long long t = sts[i].t;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  for (int j = xoff[i] + blockIdx.x * blockDim.x + threadIdx.x; j < xoff[i + 1]; j += gridDim.x * blockDim.x)
    xa[j] = t > 0 ? xs[j] * it : x[j];
  for (int r = yoff[i] + blockIdx.x * blockDim.x + threadIdx.x; r < yoff[i + 1]; r += gridDim.x * blockDim.x)
    ya[r] = t > 0 ? ys[r] * it : y[r];
}

__global__ void k_apply_b(const DevState* __restrict__ sts, double* __restrict__ x, double* __restrict__ y,
                          const double* __restrict__ xa, const double* __restrict__ ya, double* __restrict__ xr,
                          double* __restrict__ yr, double* __restrict__ xs, double* __restrict__ ys,
                          const int* __restrict__ xoff, const int* __restrict__ yoff) {
  const int i = blockIdx.y;
  const int mode = sts[i].apply_mode;
  if (mode == APPLY_NONE) return;
  for (int j = xoff[i] + blockIdx.x * blockDim.x + threadIdx.x; j < xoff[i + 1]; j += gridDim.x * blockDim.x) {
    if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG) x[j] = xa[j];
    if (mode != APPLY_TAKE_AVG) {
      xr[j] = x[j];
      xs[j] = 0.0;
    }
  }
  for (int r = yoff[i] + blockIdx.x * blockDim.x + threadIdx.x; r < yoff[i + 1]; r += gridDim.x * blockDim.x) {
    if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG) y[r] = ya[r];
    if (mode != APPLY_TAKE_AVG) {
      yr[r] = y[r];
      ys[r] = 0.0;
    }
  }
}

// per-instance sum of squares of v over [off[i], off[i+1]) into out[i * ostride]
// (one block per instance; deterministic)
__global__ void __launch_bounds__(TPB) k_sumsq_b(const double* __restrict__ v, const int* __restrict__ off,
                                                 double* __restrict__ out, int ostride) {
  const int i = blockIdx.x;
  double vals[1] = {0.0};
  const bool mx[1] = {false};
  for (int j = off[i] + threadIdx.x; j < off[i + 1]; j += blockDim.x) vals[0] += v[j] * v[j];
  block_reduce<1>(vals, mx);
  if (threadIdx.x == 0) out[(size_t)i * ostride] = vals[0];
}

// v = w / sqrt(s2[i * sstride]) on instance i's range when positive
__global__ void k_div_by_norm_b(double* __restrict__ v, const double* __restrict__ w, const double* __restrict__ s2,
                                int sstride, const int* __restrict__ off) {
  const int i = blockIdx.y;
  const double s = sqrt(s2[(size_t)i * sstride]);
  if (!(s > 0.0)) return;
  const double is = 1.0 / s;
  for (int j = off[i] + blockIdx.x * blockDim.x + threadIdx.x; j < off[i + 1]; j += gridDim.x * blockDim.x)
    v[j] = w[j] * is;
}

// v = 1 / sqrt(count of instance i) on instance i's range (power-iteration start)
// Start vector of the power iteration, before normalization: 0.5 + u with u
// the top 53 bits of SplitMix64 (Steele, Lea and Flood 2014; finalizer
// constants of Vigna's reference splitmix64.c) at counter j + 1, j the caller's
// column (local to the instance). A fixed pseudo-random vector, since the
// all-ones vector is mapped to zero by matrices such as [1, -1].
__device__ __forceinline__ double power_start_value(unsigned long long j) {
  unsigned long long z = (j + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return 0.5 + (double)(z >> 11) * 0x1.0p-53;
}

// instance blockIdx.y owns internal columns [off[i], off[i+1]) (off == nullptr:
// one problem of n columns); perm_x maps internal to the caller's columns
__global__ void k_power_start(double* __restrict__ v, const int* __restrict__ perm_x, const int* __restrict__ off,
                              int n) {
  const int i = blockIdx.y;
  const int a = off ? off[i] : 0, e = off ? off[i + 1] : n;
  for (int j = a + blockIdx.x * blockDim.x + threadIdx.x; j < e; j += gridDim.x * blockDim.x)
    v[j] = power_start_value((unsigned long long)(perm_x[j] - a));
}

__global__ void k_finish_setup_b(DevState* sts, int count, const double* __restrict__ scal, int sstride,
                                 double step_factor, int primal_weight) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  k_finish_setup_body(sts + i, scal + (size_t)i * sstride, step_factor, primal_weight);
}

__global__ void k_apply(const DevState* __restrict__ st, double* __restrict__ x, double* __restrict__ y,
                        const double* __restrict__ xa, const double* __restrict__ ya, double* __restrict__ xr,
                        double* __restrict__ yr, double* __restrict__ xs, double* __restrict__ ys, int n, int m) {
  const int mode = st->apply_mode;
  if (mode == APPLY_NONE) return;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    // APPLY_RESTART_STEP: xa, ya hold the PDHG step T(z) of the current point
    if (i < n) {
      if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG || mode == APPLY_RESTART_STEP) x[i] = xa[i];
      if (mode != APPLY_TAKE_AVG) {
        xr[i] = x[i];
        xs[i] = 0.0;
      }
    }
    if (i < m) {
      if (mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG || mode == APPLY_RESTART_STEP) y[i] = ya[i];
      if (mode != APPLY_TAKE_AVG) {
        yr[i] = y[i];
        ys[i] = 0.0;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// mixed precision: FP32 iteration state, FP64 evaluation and restarts (no
// counterpart in the paper, whose PDHG runs in FP64)
// ---------------------------------------------------------------------------
// values32 admits zeros and normal FP32 numbers (the step kernels rebuild
// their FP64 bit patterns with integer operations, which subnormals defeat)
__global__ void k_fp32_inexact(const double* __restrict__ v, long long len, int* __restrict__ flag) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    const double a = v[i];
    bad |= (double)(float)a != a || (a != 0.0 && fabs(a) < 1.1754943508222875e-38);  // FP32's smallest normal
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(flag, 1);
}

__global__ void k_narrow_index(unsigned short* __restrict__ dst, const int* __restrict__ src, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (unsigned short)src[i];
}

__global__ void k_narrow(float* __restrict__ dst, const double* __restrict__ src, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

__global__ void k_widen(double* __restrict__ dst, const float* __restrict__ src, long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = (double)src[i];
}

// FP64 averages from FP32 running sums
__global__ void k_make_average32(const float* __restrict__ xs, const float* __restrict__ ys,
                                 const float* __restrict__ x, const float* __restrict__ y, double* __restrict__ xa,
                                 double* __restrict__ ya, int n, int m, const DevState* __restrict__ st) {
  const long long t = st->t;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) xa[i] = t > 0 ? (double)xs[i] * it : (double)x[i];
    if (i < m) ya[i] = t > 0 ? (double)ys[i] * it : (double)y[i];
  }
}

// The decision of k_decide applied to an FP32 iteration: the FP32 state takes
// the candidate (rounded), the FP64 copies (x, y = evaluation point, xr, yr =
// restart reference) follow the FP32 state exactly, the FP32 sums restart.
__global__ void k_apply32(const DevState* __restrict__ st, float* __restrict__ x32, float* __restrict__ y32,
                          double* __restrict__ x, double* __restrict__ y, const double* __restrict__ xa,
                          const double* __restrict__ ya, double* __restrict__ xr, double* __restrict__ yr,
                          float* __restrict__ xs, float* __restrict__ ys, int n, int m) {
  const int mode = st->apply_mode;
  if (mode == APPLY_NONE) return;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) {
      if (mode == APPLY_TAKE_AVG) {
        x[i] = xa[i];
        x32[i] = (float)xa[i];
      } else {
        if (mode == APPLY_RESTART_AVG || mode == APPLY_RESTART_STEP) {
          const float v = (float)xa[i];
          x32[i] = v;
          x[i] = (double)v;
        }
        xr[i] = x[i];
        xs[i] = st->halpern ? x32[i] : 0.0f;  // Halpern: the FP32 anchor
      }
    }
    if (i < m) {
      if (mode == APPLY_TAKE_AVG) {
        y[i] = ya[i];
        y32[i] = (float)ya[i];
      } else {
        if (mode == APPLY_RESTART_AVG || mode == APPLY_RESTART_STEP) {
          const float v = (float)ya[i];
          y32[i] = v;
          y[i] = (double)v;
        }
        yr[i] = y[i];
        ys[i] = st->halpern ? y32[i] : 0.0f;
      }
    }
  }
}

// ---- option refine32: FP32 phases on corrections to an FP64 restart point ----
// (reading: the paper names no precision scheme; FP64 holds the restart
// point, the KKT residuals and the restart test, FP32 the iteration)
__global__ void k_widen_delta(double* __restrict__ dst, const double* __restrict__ ref, const float* __restrict__ d,
                              long long len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = ref[i] + (double)d[i];
}

__global__ void k_widen_sum_delta(double* __restrict__ dst, const double* __restrict__ ref,
                                  const float* __restrict__ s32, long long len, const DevState* __restrict__ st) {
  const double t = (double)st->t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    dst[i] = t * ref[i] + (double)s32[i];
}

__global__ void k_make_average32_delta(const float* __restrict__ xs, const float* __restrict__ ys,
                                       const float* __restrict__ x, const float* __restrict__ y,
                                       const double* __restrict__ xr, const double* __restrict__ yr,
                                       double* __restrict__ xa, double* __restrict__ ya, int n, int m,
                                       const DevState* __restrict__ st) {
  const long long t = st->t;
  const double it = t > 0 ? 1.0 / (double)t : 0.0;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) xa[i] = xr[i] + (t > 0 ? (double)xs[i] * it : (double)x[i]);
    if (i < m) ya[i] = yr[i] + (t > 0 ? (double)ys[i] * it : (double)y[i]);
  }
}

__global__ void k_apply32_delta(const DevState* __restrict__ st, float* __restrict__ x32, float* __restrict__ y32,
                                double* __restrict__ x, double* __restrict__ y, const double* __restrict__ xa,
                                const double* __restrict__ ya, double* __restrict__ xr, double* __restrict__ yr,
                                float* __restrict__ xs, float* __restrict__ ys, int n, int m) {
  const int mode = st->apply_mode;
  if (mode == APPLY_NONE) return;
  const bool from_a = mode == APPLY_RESTART_AVG || mode == APPLY_RESTART_STEP;
  const int len = n > m ? n : m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x) {
    if (i < n) {
      if (mode == APPLY_TAKE_AVG) {
        x[i] = xa[i];
        x32[i] = (float)(xa[i] - xr[i]);
      } else {
        const double v = from_a ? xa[i] : x[i];
        x[i] = v;
        xr[i] = v;
        x32[i] = 0.0f;
        xs[i] = 0.0f;  // the sums restart; the Halpern anchor is the reference itself
      }
    }
    if (i < m) {
      if (mode == APPLY_TAKE_AVG) {
        y[i] = ya[i];
        y32[i] = (float)(ya[i] - yr[i]);
      } else {
        const double v = from_a ? ya[i] : y[i];
        y[i] = v;
        yr[i] = v;
        y32[i] = 0.0f;
        ys[i] = 0.0f;
      }
    }
  }
}

__device__ __forceinline__ bool restarted(const DevState* st) {
  const int mode = st->apply_mode;
  return mode == APPLY_RESTART_CUR || mode == APPLY_RESTART_AVG || mode == APPLY_RESTART_STEP;
}

// rows j of Ahat^T: ch32_j = chat_j - (Ahat^T yr)_j, lo32_j = -xr_j rounded up
struct RecenterDualOp {
  using State = NoState;
  const double* __restrict__ ch;
  const double* __restrict__ xr;
  float* __restrict__ ch32;
  float* __restrict__ lo32;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, double g, const State&) {
    ch32[j] = (float)(ch[j] - g);
    lo32[j] = __double2float_ru(-xr[j]);
  }
};

// rows i of Ahat: bh32_i = bhat_i - (Ahat xr)_i
struct RecenterPrimalOp {
  using State = NoState;
  const double* __restrict__ bh;
  float* __restrict__ bh32;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int i, double h, const State&) { bh32[i] = (float)(bh[i] - h); }
};

__global__ void __launch_bounds__(STEP_TPB_MAX) k_recenter_dual(Hyb At, const double* __restrict__ yr,
                                                                const double* __restrict__ ch,
                                                                const double* __restrict__ xr, float* __restrict__ ch32,
                                                                float* __restrict__ lo32,
                                                                const DevState* __restrict__ st, int force) {
  if (!force && !restarted(st)) return;
  RecenterDualOp op{ch, xr, ch32, lo32};
  hyb_dot(At, At.v, GlobalGather<double>{yr}, op);
}

__global__ void __launch_bounds__(STEP_TPB_MAX) k_recenter_primal(Hyb A, const double* __restrict__ xr,
                                                                  const double* __restrict__ bh,
                                                                  float* __restrict__ bh32,
                                                                  const DevState* __restrict__ st, int force) {
  if (!force && !restarted(st)) return;
  RecenterPrimalOp op{bh, bh32};
  hyb_dot(A, A.v, GlobalGather<double>{xr}, op);
}

// Start of the FP64 phase: the point just evaluated into st->cur becomes the
// restart reference and the count since the last restart starts over.
// Start of a feasibility polishing phase (Section 5; the phases are readings).
// st->cur holds the start point's evaluation on the phase's problem: the start
// is the restart reference and the previous candidate, counters at zero, no
// snapshots, the phase's test.
__global__ void k_polish_begin(DevState* st, int term_mode) {
  double p, d, g;
  scaled_norms(st->cur, p, d, g);
  st->rs_p = st->pc_p = p;
  st->rs_d = st->pc_d = d;
  st->rs_g = st->pc_g = g;
  st->t = 0;
  st->k = 0;
  st->term_mode = term_mode;
  st->eps_target = 0.0;
  st->snapshot_every = 0;
  st->next_snapshot = 0;
  st->converged = 0;
  st->snapshot_flag = 0;
}

__global__ void k_promote_state(DevState* st) {
  double p, d, g;
  scaled_norms(st->cur, p, d, g);
  st->rs_p = st->pc_p = p;
  st->rs_d = st->pc_d = d;
  st->rs_g = st->pc_g = g;
  st->r_restart = st->r_prev = fixed_residual(st->cur, st->tau, st->sigma);  // restart_scheme = 1
  st->t = 0;
}

// ---------------------------------------------------------------------------
// adjoint of one PDHG iteration (fixed step, no restarts; differentiation has
// no counterpart in the paper)
//   forward: u = x - tau (chat - Ahat^T y), x' = max(u, 0), v = 2x' - x,
//            y' = y + sigma (bhat - Ahat v)
//   reverse: g_v = -sigma Ahat^T g_y',  g_u = [x' > 0] (g_x' + 2 g_v),
//            g_x = -g_v + g_u,  g_chat -= tau g_u,
//            g_y = g_y' + tau Ahat g_u,  g_bhat += sigma g_y'
// ([x' > 0] is [u > 0]; the derivative of max(u, 0) at u = 0 is taken as 0)
// ---------------------------------------------------------------------------
template <class T>
struct AdjPrimalOp {
  using State = NoState;
  const T* __restrict__ xnext;  // x_{k+1} of the recomputed forward pass
  T* __restrict__ gx;           // in: adjoint of x_{k+1}; out: adjoint of x_k
  T* __restrict__ gu;           // out: adjoint of u_k
  T* __restrict__ gch;          // accumulated adjoint of chat
  T sigma, tau;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, T acc, const State&) {
    const T gv = -sigma * acc;
    const T g = xnext[j] > T(0) ? gx[j] + T(2) * gv : T(0);
    gu[j] = g;
    gx[j] = g - gv;
    gch[j] -= tau * g;
  }
};

template <class T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_adj_primal(Hyb At, const T* __restrict__ vals, const T* __restrict__ gy, const T* __restrict__ xnext,
                 T* __restrict__ gx, T* __restrict__ gu, T* __restrict__ gch, const DevState* __restrict__ st) {
  AdjPrimalOp<T> op{xnext, gx, gu, gch, (T)st->sigma, (T)st->tau};
  hyb_dot(At, vals, GlobalGather<T>{gy}, op);
}

template <class T>
struct AdjDualOp {
  using State = NoState;
  T* __restrict__ gy;   // in: adjoint of y_{k+1}; out: adjoint of y_k
  T* __restrict__ gbh;  // accumulated adjoint of bhat
  T sigma, tau;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int i, T acc, const State&) {
    const T g = gy[i];
    gbh[i] += sigma * g;
    gy[i] = g + tau * acc;
  }
};

template <class T>
__global__ void __launch_bounds__(STEP_TPB_MAX, PDHG_STEP_MIN_BLOCKS * TPB / STEP_TPB_MAX)
    k_adj_dual(Hyb A, const T* __restrict__ vals, const T* __restrict__ gu, T* __restrict__ gy, T* __restrict__ gbh,
               const DevState* __restrict__ st) {
  AdjDualOp<T> op{gy, gbh, (T)st->sigma, (T)st->tau};
  hyb_dot(A, vals, GlobalGather<T>{gu}, op);
}

// g[j] = d[j] * in[perm[j]] (caller numbering -> internal, scaled); 0 if in is null
template <class T>
__global__ void k_adj_seed(T* __restrict__ g, const double* __restrict__ in, const int* __restrict__ perm,
                           const double* __restrict__ d, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    g[i] = in ? (T)(d[i] * in[perm[i]]) : T(0);
}

// out[perm[j]] = d[j] * g[j] (internal, scaled -> caller numbering)
template <class T>
__global__ void k_adj_unseed(double* __restrict__ out, const T* __restrict__ g, const int* __restrict__ perm,
                             const double* __restrict__ d, int len) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
    out[perm[i]] = d[i] * (double)g[i];
}

// Snapshot packing: the candidate (x, y) unscaled, with z = max(0, c - A^T y),
// in the caller's numbering: the copy (x_k, y_k, z_k) Algorithm 1 hands to a
// crossover thread (Section 3.1).
struct PackDualOp {
  using State = NoState;
  const int* __restrict__ perm;
  const double* __restrict__ px;
  const double* __restrict__ ch;
  const double* __restrict__ dc;
  double* __restrict__ ox;
  double* __restrict__ oz;
  __device__ __forceinline__ State begin(int) { return {}; }
  __device__ __forceinline__ void finish(int j, double g, const State&) {
    const int o = perm[j];
    if (ox) ox[o] = dc[j] * px[j];
    if (oz) oz[o] = relu(ch[j] - g) / dc[j];
  }
};

__global__ void __launch_bounds__(TPB) k_pack_dual(Hyb At, const int* __restrict__ perm,
                                                   const double* __restrict__ px, const double* __restrict__ py,
                                                   const double* __restrict__ ch, const double* __restrict__ dc,
                                                   double* __restrict__ ox, double* __restrict__ oz) {
  PackDualOp op{perm, px, ch, dc, ox, oz};
  hyb_dot(At, At.v, GlobalGather<double>{py}, op);
}

__global__ void k_pack_y(const int* __restrict__ perm, const double* __restrict__ py, const double* __restrict__ dr,
                         double* __restrict__ oy, int m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m; i += (long long)gridDim.x * blockDim.x)
    oy[perm[i]] = dr[i] * py[i];
}

// Batch snapshots (Algorithm 1's hand-off for every LP of a batch): the
// candidate (x, y, z) of each instance whose evaluation scheduled a snapshot,
// on its problem as given, into the stacked output in the caller's numbering
template <class G>
__device__ __forceinline__ void snap_dual_block(const Hyb& At, const DevState& st, const int* __restrict__ perm,
                                                const double* x, const double* xa, const G& gy, const G& gya,
                                                const double* __restrict__ ch, const double* __restrict__ dc,
                                                double* ox, double* oz, int bid, int nblk) {
  if (st.candidate == KIND_AVG) {
    PackDualOp op{perm, xa, ch, dc, ox, oz};
    hyb_dot(At, At.v, gya, op, 0, bid, nblk);
  } else {
    PackDualOp op{perm, x, ch, dc, ox, oz};
    hyb_dot(At, At.v, gy, op, 0, bid, nblk);
  }
}

__global__ void __launch_bounds__(STEP_TPB_MAX) k_snap_dual_b(Hyb At, const DevState* __restrict__ sts,
                                                     const int* __restrict__ binst, const int* __restrict__ perm,
                                                     const double* __restrict__ x, const double* __restrict__ y,
                                                     const double* __restrict__ xa, const double* __restrict__ ya,
                                                     const double* __restrict__ ch, const double* __restrict__ dc,
                                                     double* __restrict__ ox, double* __restrict__ oz) {
  const DevState& st = sts[binst[blockIdx.x]];
  if (!st.snapshot_flag) return;
  snap_dual_block(At, st, perm, x, xa, GlobalGather<double>{y}, GlobalGather<double>{ya}, ch, dc, ox, oz,
                  (int)blockIdx.x, (int)gridDim.x);
}

__global__ void k_snap_y_b(const DevState* __restrict__ sts, const int* __restrict__ perm, const double* y,
                           const double* ya, const double* __restrict__ dr, double* __restrict__ oy,
                           const int* __restrict__ yoff) {
  const int i = blockIdx.y;
  if (!sts[i].snapshot_flag) return;
  const double* py = sts[i].candidate == KIND_AVG ? ya : y;
  for (int r = yoff[i] + blockIdx.x * blockDim.x + threadIdx.x; r < yoff[i + 1]; r += gridDim.x * blockDim.x)
    oy[perm[r]] = dr[r] * py[r];
}

// ---------------------------------------------------------------------------
// A whole batch in one cooperative launch (option persistent = 2; no
// counterpart in the paper): every instance's iterations, evaluations,
// restart and primal-weight decisions and termination test, with grid-wide
// barriers between the phases instead of kernel boundaries. The grid's blocks
// take the batch's blocks (the unit-grid blocks of the multi-launch engine,
// each belonging to one instance) in turn, and every block runs the same
// per-block code as the multi-launch kernels, so the two forms compute the
// same numbers in the same order. Vectors written during the launch are
// gathered with coherent loads (not the read-only path the separate kernels
// use).
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_acquire_s32(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier. Thread 0 of each block arrives on a counter; the last to
// arrive resets it and advances the generation; the others wait for the
// generation to change, for at most `budget` clock cycles and only while no
// block has reported an error. Every block of a cooperative launch is
// resident, so the wait ends unless a block has stopped early. Returns false
// in every thread of the block when the wait gave up (the first block to give
// up records BATCH_ERR_TIMEOUT and the barrier's tag) or an error is set: the
// caller then returns, and so does every other block at its next barrier.
__device__ bool grid_barrier(BatchCtl* c, long long budget, int tag) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = ld_acquire_u32(&c->gen);
    __threadfence();
    if (atomicAdd(&c->arrive, 1u) == gridDim.x - 1) {
      atomicExch(&c->arrive, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (ld_acquire_u32(&c->gen) == g) {
        if (ld_acquire_s32(&c->error) != BATCH_ERR_NONE) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > budget) {
          if (atomicCAS(&c->error, BATCH_ERR_NONE, BATCH_ERR_TIMEOUT) == BATCH_ERR_NONE) c->where = tag;
          ok = 0;
          break;
        }
        __nanosleep(128);
      }
    }
    if (ok && ld_acquire_s32(&c->error) != BATCH_ERR_NONE) ok = 0;
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// a vector written by other blocks of the same launch: plain (coherent) loads
template <class T>
struct CoherentGather {
  const T* vec;
  __device__ __forceinline__ T operator()(int c) const { return vec[c]; }
};

__global__ void __launch_bounds__(STEP_TPB_MAX, 2) k_batch_solve(BatchArgs a) {
  BatchCtl* ctl = a.ctl;
  const long long budget = ctl->budget, k0 = ctl->k0, max_iters = ctl->max_iters;
  const int G = (int)gridDim.x, nvb = a.nvb, E = a.eval_every;
  const int tid = (int)threadIdx.x, tpb = (int)blockDim.x;
  int tag = 0;
  long long done = 0;
  while (done < max_iters) {
    const long long nb = min((long long)E - (k0 + done) % E, max_iters - done);
    for (long long it = 0; it < nb; ++it) {
      // primal half-step over every block of an active instance
      for (int vb = blockIdx.x; vb < nvb; vb += G) {
        const DevState* st = a.sts + a.binst[vb];
        if (st->frozen) continue;
        if (a.halpern && st->rho == 1.0) {  // as the multi-launch kernels: reflection 1 at compile time
          PrimalHalpernOp<double, false, true> op{a.ch, a.x, a.xbar, a.xr, st->tau, halpern_weight(st, (int)it),
                                                  st->rho};
          hyb_dot(a.At, a.At.v, CoherentGather<double>{a.y}, op, 0, vb, nvb);
        } else if (a.halpern) {
          PrimalHalpernOp<double> op{a.ch, a.x, a.xbar, a.xr, st->tau, halpern_weight(st, (int)it), st->rho};
          hyb_dot(a.At, a.At.v, CoherentGather<double>{a.y}, op, 0, vb, nvb);
        } else {
          PrimalOp<double> op{a.ch, a.x, a.xbar, a.xsum, st->tau, a.restarts};
          hyb_dot(a.At, a.At.v, CoherentGather<double>{a.y}, op, 0, vb, nvb);
        }
      }
      if (!grid_barrier(ctl, budget, ++tag)) return;
      // dual half-step
      for (int vb = blockIdx.x; vb < nvb; vb += G) {
        const DevState* st = a.sts + a.binst[vb];
        if (st->frozen) continue;
        if (a.halpern && st->rho == 1.0) {
          DualHalpernOp<double, false, true> op{a.bh, a.y, a.yr, st->sigma, halpern_weight(st, (int)it), st->rho};
          hyb_dot(a.A, a.A.v, CoherentGather<double>{a.xbar}, op, 0, vb, nvb);
        } else if (a.halpern) {
          DualHalpernOp<double> op{a.bh, a.y, a.yr, st->sigma, halpern_weight(st, (int)it), st->rho};
          hyb_dot(a.A, a.A.v, CoherentGather<double>{a.xbar}, op, 0, vb, nvb);
        } else {
          DualOp<double> op{a.bh, a.y, a.ysum, st->sigma, a.restarts};
          hyb_dot(a.A, a.A.v, CoherentGather<double>{a.xbar}, op, 0, vb, nvb);
        }
      }
      if (!grid_barrier(ctl, budget, ++tag)) return;
    }
    done += nb;
    if ((k0 + done) % E != 0) {
      // a launch that ends inside an evaluation period: only the counters
      for (int i = blockIdx.x * tpb + tid; i < a.count; i += G * tpb) {
        DevState* st = a.sts + i;
        if (st->frozen) continue;
        st->k += nb;
        st->t += nb;
      }
      break;
    }
    // evaluation 1: the averages since the last restart (t after this period)
    if (a.restarts && !a.halpern) {
      for (int i = 0; i < a.count; ++i) {
        const DevState* st = a.sts + i;
        if (st->frozen) continue;
        const long long t = st->t + nb;
        const double inv = t > 0 ? 1.0 / (double)t : 0.0;
        for (int j = a.xoff[i] + blockIdx.x * tpb + tid; j < a.xoff[i + 1]; j += G * tpb)
          a.xavg[j] = t > 0 ? a.xsum[j] * inv : a.x[j];
        for (int r = a.yoff[i] + blockIdx.x * tpb + tid; r < a.yoff[i + 1]; r += G * tpb)
          a.yavg[r] = t > 0 ? a.ysum[r] * inv : a.y[r];
      }
      if (!grid_barrier(ctl, budget, ++tag)) return;
    }
    // evaluation 2: per-block partial sums of the average and the current point
    for (int vb = blockIdx.x; vb < nvb; vb += G) {
      const bool frozen = a.sts[a.binst[vb]].frozen != 0;
      if (a.restarts && !a.halpern) {
        eval_dual_block(a.At, CoherentGather<double>{a.yavg}, a.ch, a.idc, a.xavg, a.xr, a.part_avg, frozen, vb, nvb);
        eval_primal_block(a.A, CoherentGather<double>{a.xavg}, a.bh, a.idr, a.yavg, a.yr, a.part_avg, frozen, vb,
                          nvb);
      }
      eval_dual_block(a.At, CoherentGather<double>{a.y}, a.ch, a.idc, a.x, a.xr, a.part_cur, frozen, vb, nvb);
      eval_primal_block(a.A, CoherentGather<double>{a.x}, a.bh, a.idr, a.y, a.yr, a.part_cur, frozen, vb, nvb);
    }
    if (!grid_barrier(ctl, budget, ++tag)) return;
    // evaluation 3: per-instance sums (warp q sums quantity q over the
    // instance's blocks in a fixed order), then the decisions
    for (int i = blockIdx.x; i < a.count; i += G) {
      DevState* st = a.sts + i;
      if (st->frozen) {
        if (tid == 0) st->snapshot_flag = 0;  // an instance that stopped schedules no snapshot
        continue;
      }
      const int warp = tid >> 5, lane = tid & 31;
      for (int q2 = warp; q2 < 2 * NQ; q2 += tpb >> 5) {
        const bool avg = q2 >= NQ;
        if (avg && !(a.restarts && !a.halpern)) continue;
        const int q = avg ? q2 - NQ : q2;
        const double* part = avg ? a.part_avg : a.part_cur;
        const bool is_max = (q == Q_RDINF || q == Q_RPINF);
        double acc = 0.0;
        for (int b = a.bstart[i] + lane; b < a.bstart[i + 1]; b += 32) {
          const double v = part[(size_t)b * NQ + q];
          acc = is_max ? fmax(acc, v) : acc + v;
        }
        acc = is_max ? warp_max(acc) : warp_sum(acc);
        if (lane == 0) (avg ? st->avg : st->cur).q[q] = acc;
      }
      __syncthreads();
      if (tid == 0) {
        st->k += nb;
        st->t += nb;
        decide_one(st, nullptr);
        if (st->converged) {
          st->frozen = 1;
          atomicSub(&ctl->active, 1);
        } else if (st->numeric) {
          atomicCAS(&ctl->error, BATCH_ERR_NONE, BATCH_ERR_NUMERIC);
        }
      }
      __syncthreads();
    }
    if (!grid_barrier(ctl, budget, ++tag)) return;
    // evaluation 4: scheduled snapshots (reading the candidate, which the
    // restarts below leave in place), restarts and the average taken at
    // convergence
    if (a.snap_x) {
      for (int vb = blockIdx.x; vb < nvb; vb += G) {
        const DevState& st = a.sts[a.binst[vb]];
        if (!st.snapshot_flag) continue;
        snap_dual_block(a.At, st, a.perm_x, a.x, a.xavg, CoherentGather<double>{a.y},
                        CoherentGather<double>{a.yavg}, a.ch, a.dc, a.snap_x, a.snap_z, vb, nvb);
      }
      for (int i = 0; i < a.count; ++i) {
        const DevState& st = a.sts[i];
        if (!st.snapshot_flag) continue;
        const double* py = st.candidate == KIND_AVG ? a.yavg : a.y;
        for (int r = a.yoff[i] + blockIdx.x * tpb + tid; r < a.yoff[i + 1]; r += G * tpb)
          a.snap_y[a.perm_y[r]] = a.dr[r] * py[r];
      }
    }
    for (int i = 0; i < a.count; ++i) {
      const int mode = a.sts[i].apply_mode;
      if (mode == APPLY_NONE) continue;
      const bool take_avg = mode == APPLY_RESTART_AVG || mode == APPLY_TAKE_AVG, restart = mode != APPLY_TAKE_AVG;
      for (int j = a.xoff[i] + blockIdx.x * tpb + tid; j < a.xoff[i + 1]; j += G * tpb) {
        if (take_avg) a.x[j] = a.xavg[j];
        if (restart) {
          a.xr[j] = a.x[j];
          a.xsum[j] = 0.0;
        }
      }
      for (int r = a.yoff[i] + blockIdx.x * tpb + tid; r < a.yoff[i + 1]; r += G * tpb) {
        if (take_avg) a.y[r] = a.yavg[r];
        if (restart) {
          a.yr[r] = a.y[r];
          a.ysum[r] = 0.0;
        }
      }
    }
    if (!grid_barrier(ctl, budget, ++tag)) return;
    if (ld_acquire_s32(&ctl->active) == 0) break;
  }
  if (blockIdx.x == 0 && tid == 0) ctl->done = done;
}

}  // namespace

void launch_row_absmax(const Hyb& M, double* out, int grid, cudaStream_t s) {
  k_row_absmax<<<grid, TPB, 0, s>>>(M, out);
}
void launch_row_abspow_sum(const Hyb& M, double alpha, double* out, int grid, cudaStream_t s) {
  k_row_abspow_sum<<<grid, TPB, 0, s>>>(M, alpha, out);
}
void launch_inv_sqrt_or_one(const double* in, double* out, int len, int grid, cudaStream_t s) {
  k_inv_sqrt_or_one<<<grid, TPB, 0, s>>>(in, out, len);
}
void launch_scale(const Hyb& M, const double* r, const double* s, int transposed, int grid, cudaStream_t st,
                  const int* pcol, const int* pbase) {
  k_scale<<<grid, TPB, 0, st>>>(M, r, s, transposed, pcol, pbase);
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
void launch_reciprocal(double* out, const double* in, int len, int grid, cudaStream_t s) {
  k_reciprocal<<<grid, TPB, 0, s>>>(out, in, len);
}
void launch_fill(double* v, double val, long long len, int grid, cudaStream_t s) {
  k_fill<<<grid, TPB, 0, s>>>(v, val, len);
}
void launch_spmv(const Hyb& M, const double* x, double* y, int grid, cudaStream_t s) {
  k_spmv<<<grid, TPB, 0, s>>>(M, x, y);
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
void launch_primal_step(const Hyb& At, const double* y, const double* ch, double* x, double* xbar, double* xsum,
                        const DevState* st, int accumulate, int grid, cudaStream_t s, const int* binst, int tpb,
                        int u_begin) {
  k_primal_step<double><<<grid, tpb, 0, s>>>(At, At.v, y, ch, x, xbar, xsum, st, binst, accumulate, u_begin, nullptr,
                                              nullptr);
}
void launch_dual_step(const Hyb& A, const double* xbar, const double* bh, double* y, double* ysum,
                      const DevState* st, int accumulate, int grid, cudaStream_t s, const int* binst, int tpb) {
  k_dual_step<double><<<grid, tpb, 0, s>>>(A, A.v, xbar, bh, y, ysum, st, binst, accumulate, nullptr, nullptr);
}
void launch_primal_step32(const Hyb& At, const float* y, const float* ch, float* x, float* xbar, float* xsum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb, int u_begin,
                          const float* lo) {
  k_primal_step<float><<<grid, tpb, 0, s>>>(At, At.v32, y, ch, x, xbar, xsum, st, nullptr, accumulate, u_begin,
                                              nullptr, lo);
}
void launch_dual_step32(const Hyb& A, const float* xbar, const float* bh, float* y, float* ysum, const DevState* st,
                        int accumulate, int grid, cudaStream_t s, int tpb) {
  k_dual_step<float><<<grid, tpb, 0, s>>>(A, A.v32, xbar, bh, y, ysum, st, nullptr, accumulate, nullptr, nullptr);
}
void launch_primal_step_u(const Hyb& At, const double* yg, const double* ch, double* x, double* xbar, double* xsum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb, int u_begin,
                          const double* dc) {
  k_primal_step<double, float><<<grid, tpb, 0, s>>>(At, At.u32, yg, ch, x, xbar, xsum, st, nullptr, accumulate,
                                                     u_begin, dc, nullptr);
}
void launch_dual_step_u(const Hyb& A, const double* xbar, const double* bh, double* y, double* ysum,
                        const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb, const double* dr,
                        double* yg) {
  k_dual_step<double, float><<<grid, tpb, 0, s>>>(A, A.u32, xbar, bh, y, ysum, st, nullptr, accumulate, dr, yg);
}
cudaError_t configure_primal_panels() {
  cudaError_t e = cudaSuccess;
  auto allow = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, PANEL_SMEM_MAX);
  };
  allow((const void*)k_primal_panels<double, double, false>);
  allow((const void*)k_primal_panels<float, float, false>);
  allow((const void*)k_primal_panels<double, float, false>);
  allow((const void*)k_primal_panels<double, double, true>);
  allow((const void*)k_primal_panels<float, float, true>);
  allow((const void*)k_primal_panels<double, float, true>);
  return e;
}
template <class T, class V>
void launch_panel_pass(const Hyb& Pn, const V* vals, const PanelLayout& L, const T* y, T* partial, cudaStream_t s) {
  if (L.ncols == 0) return;
  const size_t smem = sizeof(T) * (size_t)L.rows;
  if (Pn.ci16)  // 16-bit panel-relative row indices
    k_primal_panels<T, V, true><<<L.blocks, PANEL_TPB, smem, s>>>(Pn, vals, y, L.pfirst, L.binfo, L.ustart,
                                                                  L.segout, partial);
  else
    k_primal_panels<T, V, false><<<L.blocks, PANEL_TPB, smem, s>>>(Pn, vals, y, L.pfirst, L.binfo, L.ustart,
                                                                   L.segout, partial);
}
template void launch_panel_pass<double, double>(const Hyb&, const double*, const PanelLayout&, const double*, double*,
                                                cudaStream_t);
template void launch_panel_pass<float, float>(const Hyb&, const float*, const PanelLayout&, const float*, float*,
                                              cudaStream_t);
template void launch_panel_pass<double, float>(const Hyb&, const float*, const PanelLayout&, const double*, double*,
                                               cudaStream_t);
template <class T, class V>
void launch_primal_short_combine(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, T* xsum,
                                 const DevState* st, int accumulate, int short_grid, const PanelLayout& L,
                                 const T* partial, int tpb, cudaStream_t s, int halpern_it, const T* dc,
                                 const T* lo, int overlap, int wave_blocks) {
  const int cblocks = (L.ncols + tpb - 1) / tpb;
  const int grid = cblocks + short_grid;
  const int cfirst = std::min(short_grid, wave_blocks);
  // overlap (and a panel pass just launched): a programmatic dependent launch,
  // whose short-column blocks start as the panel blocks finish
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3((unsigned)tpb);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = overlap && L.ncols > 0 ? 1 : 0;
  if (halpern_it >= 0)
    cudaLaunchKernelEx(&cfg, k_primal_short_combine_halpern<T, V>, At, vals, y, ch, x, xbar, (const T*)xsum,
                       (const DevState*)st, halpern_it, L.ulong, cblocks, L.panels, partial, L.ncols, cfirst, dc, lo);
  else
    cudaLaunchKernelEx(&cfg, k_primal_short_combine<T, V>, At, vals, y, ch, x, xbar, xsum, (const DevState*)st,
                       accumulate, L.ulong, cblocks, L.panels, partial, L.ncols, cfirst, dc, lo);
}
template void launch_primal_short_combine<double, double>(const Hyb&, const double*, const double*, const double*,
                                                          double*, double*, double*, const DevState*, int, int,
                                                          const PanelLayout&, const double*, int, cudaStream_t, int,
                                                          const double*, const double*, int, int);
template void launch_primal_short_combine<float, float>(const Hyb&, const float*, const float*, const float*, float*,
                                                        float*, float*, const DevState*, int, int,
                                                        const PanelLayout&, const float*, int, cudaStream_t, int,
                                                        const float*, const float*, int, int);
template void launch_primal_short_combine<double, float>(const Hyb&, const float*, const double*, const double*,
                                                         double*, double*, double*, const DevState*, int, int,
                                                         const PanelLayout&, const double*, int, cudaStream_t, int,
                                                         const double*, const double*, int, int);
template <class T, class V>
void launch_primal_step_halpern(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, const T* xr,
                                const DevState* st, int it, int grid, cudaStream_t s, int tpb, const int* binst,
                                int u_begin, const T* dc, const T* lo) {
  k_primal_step_halpern<T, V><<<grid, tpb, 0, s>>>(At, vals, y, ch, x, xbar, xr, st, binst, it, u_begin, dc, lo);
}
template <class T, class V>
void launch_dual_step_halpern(const Hyb& A, const V* vals, const T* xbar, const T* bh, T* y, const T* yr,
                              const DevState* st, int it, int grid, cudaStream_t s, int tpb, const int* binst,
                              const T* dr, T* yg) {
  k_dual_step_halpern<T, V><<<grid, tpb, 0, s>>>(A, vals, xbar, bh, y, yr, st, binst, it, dr, yg);
}
template void launch_primal_step_halpern<double, double>(const Hyb&, const double*, const double*, const double*,
                                                         double*, double*, const double*, const DevState*, int, int,
                                                         cudaStream_t, int, const int*, int, const double*,
                                                         const double*);
template void launch_primal_step_halpern<float, float>(const Hyb&, const float*, const float*, const float*, float*,
                                                       float*, const float*, const DevState*, int, int, cudaStream_t,
                                                       int, const int*, int, const float*, const float*);
template void launch_primal_step_halpern<double, float>(const Hyb&, const float*, const double*, const double*,
                                                        double*, double*, const double*, const DevState*, int, int,
                                                        cudaStream_t, int, const int*, int, const double*,
                                                        const double*);
template void launch_dual_step_halpern<double, double>(const Hyb&, const double*, const double*, const double*,
                                                       double*, const double*, const DevState*, int, int,
                                                       cudaStream_t, int, const int*, const double*, double*);
template void launch_dual_step_halpern<float, float>(const Hyb&, const float*, const float*, const float*, float*,
                                                     const float*, const DevState*, int, int, cudaStream_t, int,
                                                     const int*, const float*, float*);
template void launch_dual_step_halpern<double, float>(const Hyb&, const float*, const double*, const double*, double*,
                                                      const double*, const DevState*, int, int, cudaStream_t, int,
                                                      const int*, const double*, double*);
template <class T>
void launch_dual_step_hot(const Hyb& A, const T* vals, const T* xbar, int hot, const T* bh, T* y, T* ysum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int halpern_it) {
  const size_t smem = (size_t)hot * sizeof(T);
  if (halpern_it >= 0)
    k_dual_step_hot_halpern<T><<<grid, HOT_TPB, smem, s>>>(A, vals, xbar, hot, bh, y, ysum, st, halpern_it);
  else
    k_dual_step_hot<T><<<grid, HOT_TPB, smem, s>>>(A, vals, xbar, hot, bh, y, ysum, st, accumulate);
}
template void launch_dual_step_hot<double>(const Hyb&, const double*, const double*, int, const double*, double*,
                                           double*, const DevState*, int, int, cudaStream_t, int);
template void launch_dual_step_hot<float>(const Hyb&, const float*, const float*, int, const float*, float*, float*,
                                          const DevState*, int, int, cudaStream_t, int);
void launch_add_counters(DevState* st, long long dk, cudaStream_t s) { k_add_counters<<<1, 1, 0, s>>>(st, dk); }
void launch_make_average(const double* xs, const double* ys, const double* x, const double* y, double* xa,
                         double* ya, int n, int m, const DevState* st, int grid, cudaStream_t s) {
  k_make_average<<<grid, TPB, 0, s>>>(xs, ys, x, y, xa, ya, n, m, st);
}
void launch_eval_point(const Hyb& A, const Hyb& At, const double* px, const double* py, const double* bh,
                       const double* ch, const double* idr, const double* idc, const double* xr, const double* yr,
                       double* partials, int nb, cudaStream_t s, const DevState* sts, const int* binst, int tpb) {
  k_eval_dual<<<nb, tpb, 0, s>>>(At, py, ch, idc, px, xr, partials, sts, binst);
  k_eval_primal<<<nb, tpb, 0, s>>>(A, px, bh, idr, py, yr, partials, sts, binst);
}
void launch_eval_point_fp(const Hyb& A, const Hyb& At, const double* px, const double* py, const double* bh,
                          const double* ch, const double* idr, const double* idc, const double* xr, const double* yr,
                          double* partials, int nb, const DevState* st, double* xt, double* ht, double* yt,
                          int spmv_grid, cudaStream_t s, int tpb) {
  k_eval_dual_fp<<<nb, tpb, 0, s>>>(At, py, ch, idc, px, xr, partials, st, xt);
  k_spmv<<<spmv_grid, TPB, 0, s>>>(A, xt, ht);
  k_eval_primal_fp<<<nb, tpb, 0, s>>>(A, px, bh, idr, py, yr, partials, st, ht, yt);
}
void launch_decide_b(DevState* sts, int count, cudaStream_t s) { k_decide_b<<<(count + 127) / 128, 128, 0, s>>>(sts, count); }
void launch_add_counters_b(DevState* sts, int count, long long dk, cudaStream_t s) {
  k_add_counters_b<<<(count + 127) / 128, 128, 0, s>>>(sts, count, dk);
}
void launch_init_restart_ref_b(DevState* sts, int count, cudaStream_t s) {
  k_init_restart_ref_b<<<(count + 127) / 128, 128, 0, s>>>(sts, count);
}
void launch_eval_finalize_b(const double* partials, const int* bstart, int count, EvalSums* out0, size_t stride,
                            cudaStream_t s) {
  k_eval_finalize_b<<<count, 32 * NQ, 0, s>>>(partials, bstart, reinterpret_cast<char*>(out0), stride);
}
void launch_make_average_b(const double* xs, const double* ys, const double* x, const double* y, double* xa,
                           double* ya, const int* xoff, const int* yoff, const DevState* sts, int count, int gx,
                           cudaStream_t s) {
  k_make_average_b<<<dim3(gx, count), TPB, 0, s>>>(xs, ys, x, y, xa, ya, xoff, yoff, sts);
}
void launch_apply_b(const DevState* sts, double* x, double* y, const double* xa, const double* ya, double* xr,
                    double* yr, double* xs, double* ys, const int* xoff, const int* yoff, int count, int gx,
                    cudaStream_t s) {
  k_apply_b<<<dim3(gx, count), TPB, 0, s>>>(sts, x, y, xa, ya, xr, yr, xs, ys, xoff, yoff);
}
void launch_snap_b(const Hyb& At, const DevState* sts, const int* binst, int nblocks, const int* perm_x,
                   const int* perm_y, const double* x, const double* y, const double* xa, const double* ya,
                   const double* ch, const double* dc, const double* dr, double* ox, double* oy, double* oz,
                   const int* yoff, int count, int gx, int tpb, cudaStream_t s) {
  k_snap_dual_b<<<nblocks, tpb, 0, s>>>(At, sts, binst, perm_x, x, y, xa, ya, ch, dc, ox, oz);
  k_snap_y_b<<<dim3(gx, count), TPB, 0, s>>>(sts, perm_y, y, ya, dr, oy, yoff);
}
cudaError_t batch_solve_grid(int tpb, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_solve, tpb, 0);
  if (e != cudaSuccess) return e;
  *grid = sms * std::max(per_sm, 1);
  return cudaSuccess;
}
cudaError_t launch_batch_solve(const BatchArgs& a, int grid, int tpb, cudaStream_t s) {
  BatchArgs args = a;
  void* params[] = {&args};
  return cudaLaunchCooperativeKernel((const void*)k_batch_solve, dim3(grid), dim3(tpb), params, 0, s);
}
void launch_sumsq_b(const double* v, const int* off, int count, double* out, int ostride, cudaStream_t s) {
  k_sumsq_b<<<count, TPB, 0, s>>>(v, off, out, ostride);
}
void launch_div_by_norm_b(double* v, const double* w, const double* s2, int sstride, const int* off, int count,
                          int gx, cudaStream_t s) {
  k_div_by_norm_b<<<dim3(gx, count), TPB, 0, s>>>(v, w, s2, sstride, off);
}
void launch_power_start(double* v, const int* perm_x, const int* off, int count, int n, int gx, cudaStream_t s) {
  k_power_start<<<dim3(gx, count), TPB, 0, s>>>(v, perm_x, off, n);
}
void launch_finish_setup_b(DevState* sts, int count, const double* scal, int sstride, double step_factor,
                           int primal_weight, cudaStream_t s) {
  k_finish_setup_b<<<(count + 127) / 128, 128, 0, s>>>(sts, count, scal, sstride, step_factor, primal_weight);
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
void launch_pack_solution(const Hyb& At, const int* perm_x, const int* perm_y, const double* px, const double* py,
                          const double* ch, const double* dc, const double* dr, double* ox, double* oy, double* oz,
                          int grid, cudaStream_t s) {
  if (ox || oz) k_pack_dual<<<grid, TPB, 0, s>>>(At, perm_x, px, py, ch, dc, ox, oz);
  if (oy) k_pack_y<<<grid, TPB, 0, s>>>(perm_y, py, dr, oy, At.cols);
}

void launch_narrow(float* dst, const double* src, long long len, int grid, cudaStream_t s) {
  k_narrow<<<grid, TPB, 0, s>>>(dst, src, len);
}
void launch_widen(double* dst, const float* src, long long len, int grid, cudaStream_t s) {
  k_widen<<<grid, TPB, 0, s>>>(dst, src, len);
}
void launch_make_average32(const float* xs, const float* ys, const float* x, const float* y, double* xa, double* ya,
                           int n, int m, const DevState* st, int grid, cudaStream_t s) {
  k_make_average32<<<grid, TPB, 0, s>>>(xs, ys, x, y, xa, ya, n, m, st);
}
void launch_apply32(const DevState* st, float* x32, float* y32, double* x, double* y, const double* xa,
                    const double* ya, double* xr, double* yr, float* xs, float* ys, int n, int m, int grid,
                    cudaStream_t s) {
  k_apply32<<<grid, TPB, 0, s>>>(st, x32, y32, x, y, xa, ya, xr, yr, xs, ys, n, m);
}
void launch_narrow_index(unsigned short* dst, const int* src, long long len, int grid, cudaStream_t s) {
  if (len > 0) k_narrow_index<<<grid, TPB, 0, s>>>(dst, src, len);
}
void launch_widen_delta(double* dst, const double* ref, const float* d, long long len, int grid, cudaStream_t s) {
  k_widen_delta<<<grid, TPB, 0, s>>>(dst, ref, d, len);
}
void launch_widen_sum_delta(double* dst, const double* ref, const float* sum32, long long len, const DevState* st,
                            int grid, cudaStream_t s) {
  k_widen_sum_delta<<<grid, TPB, 0, s>>>(dst, ref, sum32, len, st);
}
void launch_make_average32_delta(const float* xs, const float* ys, const float* x, const float* y, const double* xr,
                                 const double* yr, double* xa, double* ya, int n, int m, const DevState* st, int grid,
                                 cudaStream_t s) {
  k_make_average32_delta<<<grid, TPB, 0, s>>>(xs, ys, x, y, xr, yr, xa, ya, n, m, st);
}
void launch_apply32_delta(const DevState* st, float* x32, float* y32, double* x, double* y, const double* xa,
                          const double* ya, double* xr, double* yr, float* xs, float* ys, int n, int m, int grid,
                          cudaStream_t s) {
  k_apply32_delta<<<grid, TPB, 0, s>>>(st, x32, y32, x, y, xa, ya, xr, yr, xs, ys, n, m);
}
void launch_recenter(const Hyb& A, const Hyb& At, const double* xr, const double* yr, const double* bh,
                     const double* ch, float* bh32, float* ch32, float* lo32, const DevState* st, int force, int grA,
                     int grT, cudaStream_t s) {
  k_recenter_dual<<<grT, TPB, 0, s>>>(At, yr, ch, xr, ch32, lo32, st, force);
  k_recenter_primal<<<grA, TPB, 0, s>>>(A, xr, bh, bh32, st, force);
}
void launch_fp32_inexact(const double* v, long long len, int* flag, cudaStream_t s) {
  if (len > 0) k_fp32_inexact<<<(int)std::min<long long>(4096, (len + TPB - 1) / TPB), TPB, 0, s>>>(v, len, flag);
}
void launch_promote_state(DevState* st, cudaStream_t s) { k_promote_state<<<1, 1, 0, s>>>(st); }
void launch_polish_begin(DevState* st, int term_mode, cudaStream_t s) { k_polish_begin<<<1, 1, 0, s>>>(st, term_mode); }

template <class T>
void launch_adj_step(const Hyb& A, const Hyb& At, const T* valsA, const T* valsAt, const T* xnext, T* gx, T* gy,
                     T* gu, T* gch, T* gbh, const DevState* st, cudaStream_t s) {
  k_adj_primal<T><<<std::max(1, (At.units() + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK), TPB, 0, s>>>(
      At, valsAt, gy, xnext, gx, gu, gch, st);
  k_adj_dual<T><<<std::max(1, (A.units() + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK), TPB, 0, s>>>(A, valsA, gu, gy,
                                                                                                    gbh, st);
}
template void launch_adj_step<double>(const Hyb&, const Hyb&, const double*, const double*, const double*, double*,
                                      double*, double*, double*, double*, const DevState*, cudaStream_t);
template void launch_adj_step<float>(const Hyb&, const Hyb&, const float*, const float*, const float*, float*, float*,
                                     float*, float*, float*, const DevState*, cudaStream_t);

template <class T>
void launch_adj_seed(T* g, const double* in, const int* perm, const double* d, int len, int grid, cudaStream_t s) {
  k_adj_seed<T><<<grid, TPB, 0, s>>>(g, in, perm, d, len);
}
template void launch_adj_seed<double>(double*, const double*, const int*, const double*, int, int, cudaStream_t);
template void launch_adj_seed<float>(float*, const double*, const int*, const double*, int, int, cudaStream_t);

template <class T>
void launch_adj_unseed(double* out, const T* g, const int* perm, const double* d, int len, int grid,
                       cudaStream_t s) {
  k_adj_unseed<T><<<grid, TPB, 0, s>>>(out, g, perm, d, len);
}
template void launch_adj_unseed<double>(double*, const double*, const int*, const double*, int, int, cudaStream_t);
template void launch_adj_unseed<float>(double*, const float*, const int*, const double*, int, int, cudaStream_t);

void prefer_l1_for_step_kernels() {
  // the step kernels use no shared memory: give the on-chip memory to L1,
  // which caches the gathered vector
  cudaFuncSetAttribute(k_primal_step<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_dual_step<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_step<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_dual_step<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_step<double, float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_dual_step<double, float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_short_combine<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_short_combine<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_short_combine_halpern<double>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_primal_short_combine_halpern<float>, cudaFuncAttributePreferredSharedMemoryCarveout, 0);
  cudaFuncSetAttribute(k_dual_step_hot<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, HOT_SMEM_MAX);
  cudaFuncSetAttribute(k_dual_step_hot<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, HOT_SMEM_MAX);
  cudaFuncSetAttribute(k_dual_step_hot_halpern<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, HOT_SMEM_MAX);
  cudaFuncSetAttribute(k_dual_step_hot_halpern<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, HOT_SMEM_MAX);
}

}  // namespace pdhg
