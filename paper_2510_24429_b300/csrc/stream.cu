// Streamed step kernels (option stream_steps): the PDHG half-steps of
// Algorithm 1's "Perform PDHG iteration" (Section 3.1), in the PDLP form and
// the reflected Halpern form the paper's solver follows (Section 1,
// Section 4.1; readings, as the paper gives no formula), with the matrix and
// the step's own vectors moved into shared memory by bulk copies (TMA)
// instead of register loads.
//
// Why: the direct step kernels (kernels.cu) issue their matrix loads, their
// gathers and their epilogue loads from registers, so the bytes a warp keeps
// in flight are bounded by its registers, and a warp waits for the epilogue
// loads of a row only once the row is summed. Here every warp owns a ring of
// `depth` slots in shared memory. One lane keeps depth - 1 jobs ahead in
// flight: a job is a piece of at most STREAM_PIECE matrix slots of one unit
// (indices and values, two cp.async.bulk copies) plus, with the unit's last
// piece, the unit's rows of the step's vectors (x, chat, x_sum, D_c for the
// primal step; y, bhat, y_sum, D_r for the dual step; the anchor in place of
// the sums in the Halpern form), each one bulk copy, all completing on the
// slot's mbarrier. The warp then reads the piece from shared memory and
// issues only the gathers of the other half-step's vector from registers.
//
// The arithmetic per row is that of k_primal_step, k_primal_short_combine and
// k_dual_step (and their Halpern forms), in the same order: a long row is
// summed by lanes over the same entry sequence (pieces are multiples of 128
// entries), then reduced by warp_sum; a slice row sums its entries in order;
// the long columns' panel partial sums are added in panel order. So the
// results are bit-identical to the direct kernels', which the tests check.
//
// Every mbarrier wait is bounded (about a second of clock64 cycles). A wait
// that runs out sets DevState::wait_err, waits (bounded again) for the warp's
// copies still in flight, and the warp returns; the host reports
// PDHG_ERR_TIMEOUT. Vectors are read up to 16 bytes past their ends (the
// alignment of a bulk copy); the engine allocates every device buffer with
// that much slack.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"
#include "step_ops.cuh"

namespace pdhg {

namespace {

constexpr long long WAIT_CYCLES = 1LL << 31;  // ~1 s at 2 GHz
constexpr int CAP = STREAM_PRE_CAP;

__device__ __forceinline__ unsigned long long evict_first_policy() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}

__device__ __forceinline__ void mbar_init(unsigned bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}

// Bounded wait for the phase of parity `parity` of the mbarrier at `bar`;
// false when WAIT_CYCLES passed first. Warp-uniform: true only when every
// lane saw the phase complete.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  bool ok = mbar_try_wait(bar, parity);
  if (!ok) {
    const long long t0 = clock64();
    while (!(ok = mbar_try_wait(bar, parity)))
      if (clock64() - t0 > WAIT_CYCLES) break;
  }
  return __all_sync(0xffffffffu, ok);
}

// global -> shared bulk copy completing on the mbarrier at `bar` (16-byte
// aligned addresses, a multiple of 16 bytes)
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar,
                                          unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar), "l"(pol)
      : "memory");
}

// The epilogues, reading the step's vectors from the staged copies: for row
// r, vector k of the job sits at p[k * CAP + r] (p already offset by the first
// staged row). Each performs the arithmetic of its counterpart in kernels.cu
// in the same order.

// The primal projection: max(0, v), or (FP32 with option refine32) max(lo_j,
// v) with lo staged as the fourth vector (the FP32 steps stage no D_c), as
// project() of the direct kernels
template <class T>
__device__ __forceinline__ T sproject(int, const T*, int, T v) {
  return relu(v);
}
template <>
__device__ __forceinline__ float sproject<float>(int use_lo, const float* lo, int j, float v) {
  if (!use_lo) return relu(v);
  const float l = lo[j];
  return v < l ? l : v;
}

// PrimalOp: staged x, chat, x_sum (accumulate), D_c (SC) or the bounds (lo)
template <class T, bool SC>
struct SPrimalOp {
  T* __restrict__ x;
  T* __restrict__ xbar;
  T* __restrict__ xsum;
  T tau;
  int accumulate, use_lo;
  __device__ __forceinline__ void finish(int j, T g, const T* p) const {
    const T d = SC ? p[3 * CAP + j] : T(1);
    const T xj = p[j];
    const T xn = sproject(use_lo, p + 3 * CAP, j, xj - tau * (p[CAP + j] - (SC ? d * g : g)));
    xbar[j] = SC ? d * (T(2) * xn - xj) : T(2) * xn - xj;  // default policy: gathered by the dual step next
    __stcs(x + j, xn);
    if (accumulate) __stcs(xsum + j, p[2 * CAP + j] + xn);
  }
};

// PrimalHalpernOp: staged x, chat, anchor x_r, D_c (SC) or the bounds (lo)
template <class T, bool SC, bool R1>
struct SPrimalHalpernOp {
  T* __restrict__ x;
  T* __restrict__ xbar;
  T tau, w, rho;
  int use_lo;
  __device__ __forceinline__ void finish(int j, T g, const T* p) const {
    const T d = SC ? p[3 * CAP + j] : T(1);
    const T xj = p[j];
    const T xt = sproject(use_lo, p + 3 * CAP, j, xj - tau * (p[CAP + j] - (SC ? d * g : g)));
    const T xb = T(2) * xt - xj;
    xbar[j] = SC ? d * xb : xb;
    __stcs(x + j, halpern_mix_r<R1>(xt, xj, xb, p[2 * CAP + j], w, T(1) - w, rho));
  }
};

// DualOp: staged y, bhat, y_sum (accumulate), D_r (SC)
template <class T, bool SC>
struct SDualOp {
  T* __restrict__ y;
  T* __restrict__ ysum;
  T* __restrict__ yg;
  T sigma;
  int accumulate;
  __device__ __forceinline__ void finish(int i, T h, const T* p) const {
    const T d = SC ? p[3 * CAP + i] : T(1);
    const T yn = p[i] + sigma * (p[CAP + i] - (SC ? d * h : h));
    y[i] = yn;  // default policy: gathered by the primal step next (SC: yg is)
    if (SC) yg[i] = d * yn;
    if (accumulate) __stcs(ysum + i, p[2 * CAP + i] + yn);
  }
};

// DualHalpernOp: staged y, bhat, anchor y_r, D_r (SC)
template <class T, bool SC, bool R1>
struct SDualHalpernOp {
  T* __restrict__ y;
  T* __restrict__ yg;
  T sigma, w, rho;
  __device__ __forceinline__ void finish(int i, T h, const T* p) const {
    const T d = SC ? p[3 * CAP + i] : T(1);
    const T yi = p[i];
    const T yt = yi + sigma * (p[CAP + i] - (SC ? d * h : h));
    const T yn = halpern_mix_r<R1>(yt, yi, T(2) * yt - yi, p[2 * CAP + i], w, T(1) - w, rho);
    y[i] = yn;
    if (SC) yg[i] = d * yn;
  }
};

// One warp's ring of `depth` slots and its job sequence. Jobs are numbered by
// a virtual unit index v = gw, gw + GW, ... below nvirt = ncomb + (n_units -
// u_begin): v < ncomb is the combine job of long columns [32 v, 32 v + 32)
// (the panel-tiled primal step's partial sums), any other v is unit
// u_begin + v - ncomb of the layout, cut into pieces of STREAM_PIECE slots
// (at least one piece: the last one also stages the unit's rows). Every lane
// runs the issue cursor (uniform control flow); lane 0 issues the copies.
template <class T, class V>
struct Ring {
  static constexpr int A = 16 / (int)sizeof(T);  // entries per 16 bytes (bulk-copy alignment)
  const Hyb& H;
  const V* __restrict__ vals;
  const T* pre_src[STREAM_NPRE];  // staged vectors (nullptr: not staged)
  int npre;
  int ncols, ncomb, u_begin;
  long long nvirt, GW;
  unsigned char* ring;  // this warp's slots
  unsigned ring_s;      // its shared-memory address
  unsigned bar0;        // shared-memory address of its first mbarrier
  int depth;
  unsigned slot_bytes;
  unsigned long long pol;
  int lane;
  long long iv;  // issue cursor: job v, piece ij of inj
  int ij, inj;
  long long issued = 0, cons = 0;

  __device__ __forceinline__ int pieces_of(long long v) const {
    if (v < ncomb) return 1;
    const int u = u_begin + (int)(v - ncomb);
    const long long len = H.uoff[u + 1] - H.uoff[u];
    return (int)max(1LL, (len + STREAM_PIECE - 1) / STREAM_PIECE);
  }
  __device__ __forceinline__ int slot() const { return (int)(cons % depth); }
  __device__ __forceinline__ const int* ci(int s) const {
    return reinterpret_cast<const int*>(ring + (size_t)s * slot_bytes);
  }
  __device__ __forceinline__ const V* val(int s) const {
    return reinterpret_cast<const V*>(ring + (size_t)s * slot_bytes + STREAM_PIECE * 4);
  }
  // staged vectors of slot s, indexed by row: vector k of row r at p[k * CAP + r]
  __device__ __forceinline__ const T* pre(int s, int r0) const {
    return reinterpret_cast<const T*>(ring + (size_t)s * slot_bytes + STREAM_PIECE * (4 + sizeof(V))) -
           (r0 & ~(A - 1));
  }
  __device__ __forceinline__ void start(long long v0) {
    iv = v0;
    ij = 0;
    inj = v0 < nvirt ? pieces_of(v0) : 0;
  }

  // put the next job of the sequence in flight in the next free slot
  __device__ __forceinline__ void issue() {
    if (iv >= nvirt) return;
    const int s = (int)(issued % depth);
    const unsigned bar = bar0 + 8u * (unsigned)s;
    long long sb = 0;
    int cnt = 0, r0 = 0, nr = 0;
    if (iv < ncomb) {
      r0 = 32 * (int)iv;
      nr = min(32, ncols - r0);
    } else {
      const int u = u_begin + (int)(iv - ncomb);
      const long long beg = H.uoff[u], end = H.uoff[u + 1];
      sb = beg + (long long)ij * STREAM_PIECE;
      cnt = (int)max(0LL, min((long long)STREAM_PIECE, end - sb));
      if (ij == inj - 1) {
        const int4 info = H.uinfo[u];
        r0 = info.x;
        nr = info.y == 0 ? 1 : info.z;
      }
    }
    if (lane == 0) {
      int a0 = 0, a1 = 0;
      if (nr > 0) {
        a0 = r0 & ~(A - 1);
        a1 = (r0 + nr + A - 1) & ~(A - 1);
      }
      const unsigned pre_bytes = (unsigned)(a1 - a0) * (unsigned)sizeof(T);
      mbar_expect_tx(bar, (unsigned)cnt * (unsigned)(4 + sizeof(V)) + (unsigned)npre * pre_bytes);
      const unsigned dst = ring_s + (unsigned)s * slot_bytes;
      if (cnt > 0) {
        bulk_load(dst, H.ci + sb, (unsigned)cnt * 4u, bar, pol);
        bulk_load(dst + STREAM_PIECE * 4, vals + sb, (unsigned)cnt * (unsigned)sizeof(V), bar, pol);
      }
      if (pre_bytes) {
        const unsigned pdst = dst + STREAM_PIECE * (4 + (unsigned)sizeof(V));
#pragma unroll
        for (int k = 0; k < STREAM_NPRE; ++k)
          if (pre_src[k]) bulk_load(pdst + (unsigned)(k * CAP * sizeof(T)), pre_src[k] + a0, pre_bytes, bar, pol);
      }
    }
    if (++ij == inj) {
      iv += GW;
      ij = 0;
      inj = iv < nvirt ? pieces_of(iv) : 0;
    }
    ++issued;
  }
  // wait for the job in the consumer's slot (bounded; warp-uniform result)
  __device__ __forceinline__ bool wait() const {
    return mbar_wait(bar0 + 8u * (unsigned)slot(), (unsigned)((cons / depth) & 1));
  }
  // the warp is done with the consumer's slot: refill it with the next job
  __device__ __forceinline__ void release() {
    __syncwarp();
    if (lane == 0) asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    ++cons;
    issue();
  }
  // after a failed wait: wait (bounded) for the copies still in flight
  __device__ __forceinline__ void drain() {
    while (cons < issued) {
      mbar_wait(bar0 + 8u * (unsigned)slot(), (unsigned)((cons / depth) & 1));
      ++cons;
    }
  }
};

// a long row (one warp): lane L sums entries 2L, 2L + 1 and 2L + 64, 2L + 65
// of every 128, over pieces that start at multiples of 128 entries, in the
// order of unit_dot's long-row loop; then the warp sum
template <class T, class V, class Op>
__device__ __forceinline__ bool long_unit(Ring<T, V>& S, int row, long long beg, long long end,
                                          const T* __restrict__ gvec, const Op& op) {
  using PV = typename Pair<V>::type;
  const int nj = (int)max(1LL, (end - beg + STREAM_PIECE - 1) / STREAM_PIECE);
  T acc = T(0);
  for (int j = 0; j < nj; ++j) {
    if (!S.wait()) return false;
    const int s = S.slot();
    const int cnt = (int)min((long long)STREAM_PIECE, end - beg - (long long)j * STREAM_PIECE);
    const int* ci = S.ci(s);
    const V* vv = S.val(s);
    for (int kk = 2 * S.lane; kk < cnt; kk += 128) {
      const int2 c0 = *reinterpret_cast<const int2*>(ci + kk);
      const PV a = *reinterpret_cast<const PV*>(vv + kk);
      const bool second = kk + 64 < cnt;
      int2 c1 = make_int2(0, 0);
      PV b;
      b.x = V(0);
      b.y = V(0);
      if (second) {
        c1 = *reinterpret_cast<const int2*>(ci + kk + 64);
        b = *reinterpret_cast<const PV*>(vv + kk + 64);
      }
      const T g0 = __ldg(gvec + c0.x), g1 = __ldg(gvec + c0.y);
      const T g2 = __ldg(gvec + c1.x), g3 = __ldg(gvec + c1.y);
      acc += as_acc<T>(a.x) * g0;
      acc += as_acc<T>(a.y) * g1;
      acc += as_acc<T>(b.x) * g2;
      acc += as_acc<T>(b.y) * g3;
    }
    if (j == nj - 1) {
      acc = warp_sum(acc);
      if (S.lane == 0) op.finish(row, acc, S.pre(s, row));
    }
    S.release();
  }
  return true;
}

// a slice of 32 R rows (entries in pairs, see Hyb): each lane sums its R rows'
// entries in order, all gathers of a piece issued before its multiply-adds
template <int R, class T, class V, class Op>
__device__ __forceinline__ bool slice_unit(Ring<T, V>& S, int4 info, long long beg, long long end,
                                           const T* __restrict__ gvec, const Op& op) {
  using PV = typename Pair<V>::type;
  constexpr int G = STREAM_PIECE / 64;          // pair groups per full piece (a multiple of R)
  constexpr int GB = sizeof(T) == 8 ? 4 : 8;    // groups whose gathers are in flight together
  const long long len = end - beg;
  const int Lp = (int)(len / (32 * R));
  const int nj = (int)max(1LL, (len + STREAM_PIECE - 1) / STREAM_PIECE);
  const int lane = S.lane;
  T acc[R];
#pragma unroll
  for (int q = 0; q < R; ++q) acc[q] = T(0);
  for (int j = 0; j < nj; ++j) {
    if (!S.wait()) return false;
    const int s = S.slot();
    const int* ci = S.ci(s);
    const V* vv = S.val(s);
    if (Lp == 1) {
#pragma unroll
      for (int q = 0; q < R; ++q) {
        const int k = 32 * q + lane;
        acc[q] += as_acc<T>(vv[k]) * __ldg(gvec + ci[k]);
      }
    } else if (Lp >= 2) {
      const int ng = (int)(min((long long)STREAM_PIECE, len - (long long)j * STREAM_PIECE) >> 6);
      // the gathers of GB pair groups first (the values are read from shared
      // memory after they land); GB groups are a multiple of R
#pragma unroll
      for (int b = 0; b < G; b += GB) {
        T g0[GB], g1[GB];
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          if (b + g < ng) {
            const int2 c = *reinterpret_cast<const int2*>(ci + 64 * (b + g) + 2 * lane);
            g0[g] = __ldg(gvec + c.x);
            g1[g] = __ldg(gvec + c.y);
          }
        }
#pragma unroll
        for (int g = 0; g < GB; ++g) {
          if (b + g < ng) {
            const PV a = *reinterpret_cast<const PV*>(vv + 64 * (b + g) + 2 * lane);
            acc[g % R] += as_acc<T>(a.x) * g0[g];
            acc[g % R] += as_acc<T>(a.y) * g1[g];
          }
        }
      }
    }
    if (j == nj - 1) {
      const T* p = S.pre(s, info.x);
#pragma unroll
      for (int q = 0; q < R; ++q)
        if (32 * q + lane < info.z) op.finish(info.x + 32 * q + lane, acc[q], p);
    }
    S.release();
  }
  return true;
}

// combine job: 32 long columns, each lane adding its column's panel partial
// sums in panel order with eight loads in flight (short_and_combine's loop)
template <class T, class V, class Op>
__device__ __forceinline__ bool combine_job(Ring<T, V>& S, long long v, const T* __restrict__ partial, int panels,
                                            const Op& op) {
  if (!S.wait()) return false;
  const int j0 = 32 * (int)v, j = j0 + S.lane;
  if (j < S.ncols) {
    const T* pj = partial + j;
    T g = T(0);
    int p = 0;
    for (; p + 8 <= panels; p += 8) {
      T a[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) a[e] = __ldcs(pj + (long long)(p + e) * S.ncols);
#pragma unroll
      for (int e = 0; e < 8; ++e) g += a[e];
    }
    for (; p < panels; ++p) g += __ldcs(pj + (long long)p * S.ncols);
    op.finish(j, g, S.pre(S.slot(), j0));
  }
  S.release();
  return true;
}

// A warp's whole job sequence: prime the ring, then every job in order.
template <class T, class V, class Op>
__device__ __forceinline__ void run_warp(Ring<T, V>& S, long long v0, const T* __restrict__ gvec, const Op& op,
                                         const T* __restrict__ partial, int panels, DevState* st) {
  S.start(v0);
  for (int k = 0; k < S.depth; ++k) S.issue();
  bool ok = true;
  for (long long v = v0; ok && v < S.nvirt; v += S.GW) {
    if (v < S.ncomb) {
      ok = combine_job(S, v, partial, panels, op);
      continue;
    }
    const int u = S.u_begin + (int)(v - S.ncomb);
    const int4 info = S.H.uinfo[u];
    const long long beg = S.H.uoff[u], end = S.H.uoff[u + 1];
    if (info.y == 0)
      ok = long_unit(S, info.x, beg, end, gvec, op);
    else if (info.y == 4)
      ok = slice_unit<4>(S, info, beg, end, gvec, op);
    else if (info.y == 2)
      ok = slice_unit<2>(S, info, beg, end, gvec, op);
    else
      ok = slice_unit<1>(S, info, beg, end, gvec, op);
  }
  if (!ok) {
    if (S.lane == 0) atomicOr(&st->wait_err, 1u);
    S.drain();
  }
}

// Set-up shared by the kernels: this warp's ring in dynamic shared memory
// (warp w's slots at w * depth * slot_bytes, then every warp's mbarriers),
// its barriers initialised, and the run over jobs v = gw, gw + GW, ...
template <class T, class V, class Op>
__device__ __forceinline__ void stream_body(const Hyb& H, const V* __restrict__ vals, const T* __restrict__ gvec,
                                            const Op& op, const T* p0, const T* p1, const T* p2, const T* p3,
                                            int u_begin, int ncomb, int ncols, int panels, const T* __restrict__ partial,
                                            int depth, unsigned slot_bytes, DevState* st) {
  extern __shared__ __align__(128) unsigned char stream_smem[];
  const int nw = (int)(blockDim.x >> 5), w = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  // an earlier wait ran out (the call ends with PDHG_ERR_TIMEOUT): do nothing
  if (__shfl_sync(0xffffffffu, lane == 0 ? *(volatile unsigned*)&st->wait_err : 0u, 0)) return;
  unsigned char* ring = stream_smem + (size_t)w * depth * slot_bytes;
  const unsigned bar0 = (unsigned)__cvta_generic_to_shared(stream_smem + (size_t)nw * depth * slot_bytes) +
                        8u * (unsigned)(w * depth);
  if (lane == 0) {
    for (int s = 0; s < depth; ++s) mbar_init(bar0 + 8u * (unsigned)s);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncwarp();
  Ring<T, V> S{H, vals, {p0, p1, p2, p3}, 0, ncols, ncomb, u_begin, 0, 0, ring,
               (unsigned)__cvta_generic_to_shared(ring), bar0, depth, slot_bytes, evict_first_policy(), lane};
  S.npre = (p0 != nullptr) + (p1 != nullptr) + (p2 != nullptr) + (p3 != nullptr);
  S.nvirt = (long long)ncomb + (H.n_units - u_begin);
  S.GW = (long long)gridDim.x * nw;
  run_warp(S, (long long)blockIdx.x * nw + w, gvec, op, partial, panels, st);
}

// Halpern weight of step `it`, computed once per block (an FP64 division per
// thread would cost the FP64 pipe more than the step's multiply-adds of a row)
__device__ __forceinline__ double stream_halpern_weight(const DevState* st, int it) {
  __shared__ double w_shared;
  if (threadIdx.x == 0) w_shared = halpern_weight(st, it);
  __syncthreads();
  return w_shared;
}

// the dual half-step over the units of A: y' = y + sigma (bhat - Ahat xbar);
// y_sum += y' (accumulate) or the Halpern update (it >= 0, anchor yr)
template <class T, class V, bool HALP>
__global__ void __launch_bounds__(STREAM_TPB_MAX, 1)
    k_stream_dual(Hyb A, const V* __restrict__ vals, const T* __restrict__ xbar, const T* __restrict__ bh,
                  T* __restrict__ y, T* __restrict__ ysum_or_yr, DevState* st, int accumulate, int it,
                  const T* __restrict__ dr, T* __restrict__ yg, int depth, unsigned slot_bytes) {
  constexpr bool SC = !std::is_same<T, V>::value;
  if (HALP) {
    const T w = (T)stream_halpern_weight(st, it), rho = (T)st->rho;
    if (rho == T(1)) {  // the reflection known at compile time, as in the direct kernels
      SDualHalpernOp<T, SC, true> op{y, yg, (T)st->sigma, w, rho};
      stream_body<T, V>(A, vals, xbar, op, y, bh, ysum_or_yr, SC ? dr : nullptr, 0, 0, 0, 0, nullptr, depth,
                        slot_bytes, st);
    } else {
      SDualHalpernOp<T, SC, false> op{y, yg, (T)st->sigma, w, rho};
      stream_body<T, V>(A, vals, xbar, op, y, bh, ysum_or_yr, SC ? dr : nullptr, 0, 0, 0, 0, nullptr, depth,
                        slot_bytes, st);
    }
  } else {
    SDualOp<T, SC> op{y, ysum_or_yr, yg, (T)st->sigma, accumulate};
    stream_body<T, V>(A, vals, xbar, op, y, bh, accumulate ? ysum_or_yr : nullptr, SC ? dr : nullptr, 0, 0, 0, 0,
                nullptr, depth, slot_bytes, st);
  }
}

// the primal half-step over the units of At from u_begin on, and (ncols > 0)
// the combine of the long columns [0, ncols) from their panel partial sums:
// x' = max(0, x - tau (chat - Ahat^T y)); xbar = 2x' - x; x_sum += x'
// (accumulate), or the Halpern update (it >= 0, anchor xr)
template <class T, class V, bool HALP>
__global__ void __launch_bounds__(STREAM_TPB_MAX, 1)
    k_stream_primal(Hyb At, const V* __restrict__ vals, const T* __restrict__ y, const T* __restrict__ ch,
                    T* __restrict__ x, T* __restrict__ xbar, T* __restrict__ xsum_or_xr, DevState* st, int accumulate,
                    int it, int u_begin, int ncols, int panels, const T* __restrict__ partial,
                    const T* __restrict__ dc, const T* __restrict__ lo, int depth, unsigned slot_bytes) {
  constexpr bool SC = !std::is_same<T, V>::value;
  const int ncomb = (ncols + 31) / 32;
  const T* p3 = SC ? dc : lo;  // the fourth staged vector
  const int use_lo = !SC && lo != nullptr;
  if (HALP) {
    const T w = (T)stream_halpern_weight(st, it), rho = (T)st->rho;
    if (rho == T(1)) {
      SPrimalHalpernOp<T, SC, true> op{x, xbar, (T)st->tau, w, rho, use_lo};
      stream_body<T, V>(At, vals, y, op, x, ch, xsum_or_xr, p3, u_begin, ncomb, ncols, panels, partial, depth,
                        slot_bytes, st);
    } else {
      SPrimalHalpernOp<T, SC, false> op{x, xbar, (T)st->tau, w, rho, use_lo};
      stream_body<T, V>(At, vals, y, op, x, ch, xsum_or_xr, p3, u_begin, ncomb, ncols, panels, partial, depth,
                        slot_bytes, st);
    }
  } else {
    SPrimalOp<T, SC> op{x, xbar, xsum_or_xr, (T)st->tau, accumulate, use_lo};
    stream_body<T, V>(At, vals, y, op, x, ch, accumulate ? xsum_or_xr : nullptr, p3, u_begin, ncomb, ncols,
                      panels, partial, depth, slot_bytes, st);
  }
}

}  // namespace

// ---- launchers ------------------------------------------------------------------

size_t stream_smem(const StreamCfg& c, size_t t, size_t v) {
  return (size_t)c.warps * c.depth * (stream_slot_bytes(t, v) + 8);
}

template <class T, class V>
cudaError_t configure_stream(StreamCfg& c, int sms) {
  const size_t smem = stream_smem(c, sizeof(T), sizeof(V));
  if (smem > (size_t)STREAM_SMEM_MAX) return cudaErrorInvalidValue;
  cudaError_t e = cudaSuccess;
  auto allow = [&](const void* f) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  };
  allow((const void*)k_stream_dual<T, V, false>);
  allow((const void*)k_stream_dual<T, V, true>);
  allow((const void*)k_stream_primal<T, V, false>);
  allow((const void*)k_stream_primal<T, V, true>);
  if (e != cudaSuccess) return e;
  // resident blocks per SM: the smallest over the kernels (shared memory,
  // registers and threads)
  int per_sm = 1 << 20;
  auto occ = [&](const void* f) {
    int b = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, f, 32 * c.warps, smem);
    per_sm = std::min(per_sm, b);
  };
  occ((const void*)k_stream_dual<T, V, false>);
  occ((const void*)k_stream_dual<T, V, true>);
  occ((const void*)k_stream_primal<T, V, false>);
  occ((const void*)k_stream_primal<T, V, true>);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  c.blocks = per_sm * sms;
  c.smem = smem;
  return cudaSuccess;
}
template cudaError_t configure_stream<double, double>(StreamCfg&, int);
template cudaError_t configure_stream<float, float>(StreamCfg&, int);
template cudaError_t configure_stream<double, float>(StreamCfg&, int);

template <class T, class V>
void launch_stream_dual(const Hyb& A, const V* vals, const T* xbar, const T* bh, T* y, T* ysum_or_yr, DevState* st,
                        int accumulate, int halpern_it, const T* dr, T* yg, const StreamCfg& c, cudaStream_t s) {
  const unsigned sb = (unsigned)stream_slot_bytes(sizeof(T), sizeof(V));
  if (halpern_it >= 0)
    k_stream_dual<T, V, true><<<c.blocks, 32 * c.warps, c.smem, s>>>(A, vals, xbar, bh, y, ysum_or_yr, st, 0,
                                                                     halpern_it, dr, yg, c.depth, sb);
  else
    k_stream_dual<T, V, false><<<c.blocks, 32 * c.warps, c.smem, s>>>(A, vals, xbar, bh, y, ysum_or_yr, st,
                                                                      accumulate, 0, dr, yg, c.depth, sb);
}

template <class T, class V>
void launch_stream_primal(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, T* xsum_or_xr,
                          DevState* st, int accumulate, int halpern_it, int u_begin, int ncols, int panels,
                          const T* partial, const T* dc, const StreamCfg& c, cudaStream_t s, const T* lo) {
  const unsigned sb = (unsigned)stream_slot_bytes(sizeof(T), sizeof(V));
  if (halpern_it >= 0)
    k_stream_primal<T, V, true><<<c.blocks, 32 * c.warps, c.smem, s>>>(
        At, vals, y, ch, x, xbar, xsum_or_xr, st, 0, halpern_it, u_begin, ncols, panels, partial, dc, lo, c.depth, sb);
  else
    k_stream_primal<T, V, false><<<c.blocks, 32 * c.warps, c.smem, s>>>(
        At, vals, y, ch, x, xbar, xsum_or_xr, st, accumulate, 0, u_begin, ncols, panels, partial, dc, lo, c.depth,
        sb);
}

#define PDHG_STREAM_INST(T, V)                                                                                     \
  template void launch_stream_dual<T, V>(const Hyb&, const V*, const T*, const T*, T*, T*, DevState*, int, int,  \
                                         const T*, T*, const StreamCfg&, cudaStream_t);                           \
  template void launch_stream_primal<T, V>(const Hyb&, const V*, const T*, const T*, T*, T*, T*, DevState*, int, \
                                           int, int, int, int, const T*, const T*, const StreamCfg&, cudaStream_t, \
                                           const T*);
PDHG_STREAM_INST(double, double)
PDHG_STREAM_INST(float, float)
PDHG_STREAM_INST(double, float)
#undef PDHG_STREAM_INST

}  // namespace pdhg
