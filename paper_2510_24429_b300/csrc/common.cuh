// Internal types and device helpers of the PDHG engine (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pdhg {

// Quantities accumulated by one evaluation of a point (xhat, yhat) of the
// scaled problem Ahat = D_r A D_c, bhat = D_r b, chat = D_c c.
//   dual side (rows j of Ahat^T):  g = Ahat^T yhat, rd = max(0, g - chat)
//   primal side (rows i of Ahat):  h = Ahat xhat,   rp = bhat - h
// Unscaled residuals follow from r_P = D_r^{-1} rp and r_D = D_c^{-1} rd, and
// c^T x = chat^T xhat, b^T y = bhat^T yhat, x^T z = xhat^T zhat.
enum {
  Q_RD2S = 0,  // sum rd^2                      (scaled ||r_D||^2)
  Q_RD2U,      // sum (rd / d_c)^2              (||r_D||^2 as given)
  Q_RDINF,     // max |rd / d_c|
  Q_CX,        // sum chat * xhat               (c^T x)
  Q_XZ,        // sum xhat * max(0, chat - g)   (x^T z)
  Q_DX2,       // sum (xhat - xhat_restart)^2
  Q_RP2S,      // sum rp^2
  Q_RP2U,      // sum (rp / d_r)^2
  Q_RPINF,     // max |rp / d_r|
  Q_BY,        // sum bhat * yhat               (b^T y)
  Q_DY2,       // sum (yhat - yhat_restart)^2
  // fixed-point residual restart scheme (restart_scheme = 1): with the PDHG
  // step (x~, y~) = T(xhat, yhat)
  Q_FX2,       // sum (x~ - xhat)^2
  Q_FXR2,      // sum (x~ - xhat_restart)^2
  Q_FY2,       // sum (y~ - yhat)^2
  Q_FXY,       // sum (y~ - yhat) (Ahat (x~ - xhat))
  Q_FYR2,      // sum (y~ - yhat_restart)^2
  NQ
};

struct EvalSums {
  double q[NQ];
};

// apply modes written by the decision kernel (APPLY_RESTART_STEP: restart at
// the PDHG step T(z) of the current point, held where the average would be)
enum { APPLY_NONE = 0, APPLY_RESTART_CUR = 1, APPLY_RESTART_AVG = 2, APPLY_TAKE_AVG = 3, APPLY_RESTART_STEP = 4 };
enum { KIND_NONE = 0, KIND_CUR = 1, KIND_AVG = 2, KIND_STEP = 3 };

// Scalars of the method, resident in device memory so that kernels (and CUDA
// graphs) read the current step sizes without host round trips.
struct DevState {
  double tau, sigma, omega, eta;
  double norm_est;
  double b_norm, c_norm;  // ||b||_2, ||c||_2 of the problem as given
  // configuration
  double tol, eps_target, eps_factor;
  double beta_suff, beta_nec, beta_art, theta;
  long long snapshot_every, next_snapshot;
  int restarts_on, primal_weight_on;
  // counters
  long long k, t, restarts, evals, snapshots;
  // restart reference and previous candidate: (||rp||, ||rd||, gap) scaled
  double rs_p, rs_d, rs_g;
  double pc_p, pc_d, pc_g;
  // evaluation results
  EvalSums cur, avg;
  // decision outputs
  int candidate, kind, apply_mode, converged;
  int snapshot_flag, numeric;
  int frozen;  // batch: the instance has converged; its blocks skip all work
  // termination test: TERM_LP (rel_p, rel_d <= tol and rel_gap <= gap_tol) for
  // the LP itself; TERM_PRIMAL (rel_p <= tol) / TERM_DUAL (rel_d <= tol) in
  // the phases of feasibility polishing
  int term_mode;
  // reflected Halpern iteration: on, and the reflection rho
  int halpern, pad1;
  double rho;
  double cand_rel_kkt;
  double gap_tol;       // relative-gap tolerance; <= 0: tol
  double cand_rel_gap;  // the candidate's rel_gap (feasibility polishing trigger)
  double scratch[2];
  // the latest scheduled snapshot: its iteration and the candidate's rel_kkt
  long long snap_k;
  double snap_rel;
  // fixed-point residual restart scheme (restart_scheme = 1): the residual at
  // the last restart and at the previous evaluation, the PID gains and state
  int restart_scheme, pad2;
  double r_restart, r_prev;
  double pid_kp, pid_ki, pid_kd, pid_int, pid_prev;
  // a bounded wait of a streamed step kernel ran out (its results are then
  // incomplete; the host reports PDHG_ERR_TIMEOUT)
  unsigned wait_err;
  int pad3;
};

enum { TERM_LP = 0, TERM_PRIMAL = 1, TERM_DUAL = 2 };

struct TraceRec {
  long long iteration;
  int kind, candidate;
  double omega, rel_kkt;
};

constexpr int TRACE_CAP = 65536;

// Device layout of one copy of the scaled matrix (Ahat, or Ahat^T).
//
// Rows are stored in order of decreasing length (the engine renumbers the
// variables and constraints internally to get there) and grouped into
// "units", each processed by one warp:
//   - a long row (at least `long_row_min` entries): CSR, reduced by the whole
//     warp; it starts at an entry offset that is a multiple of 4 and is padded
//     to a multiple of 4 entries;
//   - a slice of 32*R shorter rows (R = rows per thread: 1, 2 or 4, chosen
//     from the slice's length), padded to the length Lp of its first
//     (longest) row; when Lp > 1 it is rounded up to an even number and the
//     entries are stored in pairs: entry e of the slice's row (32 q + lane)
//     sits at
//         uoff[u] + ((e / 2) * R + q) * 64 + 2 * lane + (e % 2)
//     so one thread loads its row's next two indices and values with one
//     8-byte and one 16-byte load and a warp reads contiguous 256 B / 512 B
//     lines; when Lp == 1 the entry of row (32 q + lane) sits at
//     uoff[u] + 32 q + lane.
// Padding slots hold value 0 and column 0. Only the first `valid` rows of a
// unit exist (slice row index 32 q + lane < valid); the rest are padding. In a
// batch the rows after a slice's last valid row belong to the next instance,
// so validity is never judged by row number. Empty units (valid = 0) pad each
// batch instance to whole blocks.
struct Hyb {
  int rows = 0, cols = 0;
  int n_units = 0;
  long long nnz = 0;          // stored entries (without padding)
  long long slots = 0;        // entry slots including padding
  long long* uoff = nullptr;  // [n_units + 1] entry offset of each unit
  int4* uinfo = nullptr;      // [n_units] (first row, R, valid rows, 0); R = 0 marks a long row
  int* ci = nullptr;          // [slots] column index (internal numbering)
  double* v = nullptr;        // [slots] value
  float* v32 = nullptr;       // [slots] value rounded to FP32 (FP32 / mixed precision only)
  float* u32 = nullptr;       // [slots] unscaled value, exactly (option values32 only)
  unsigned short* ci16 = nullptr;  // [slots] the column indices in 16 bits (panel layout: rows within a panel)
  unsigned* check = nullptr;  // checked build (PDHG_CHECKED): the context's error word
  int units() const { return n_units; }
};

// bits of the checked build's error word: what a kernel found out of range
// (and skipped instead of accessing)
enum { CHECK_UNIT = 1, CHECK_COLUMN = 2 };

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
// max(0, v) for FP64 by the sign bit, on the integer pipe (the FP64 pipe is
// the scarce one): -0 and negative numbers give +0, NaN passes through (NaNs
// that arithmetic makes are positive)
__device__ __forceinline__ double relu(double v) { return __double2hiint(v) < 0 ? 0.0 : v; }
__device__ __forceinline__ float relu(float v) { return v < 0.0f ? 0.0f : v; }

// slot of entry e of row (32 q + lane) in a slice of 32 R rows padded to Lp
// entries per row: pairs of entries are interleaved across the slice's
// threads, so a thread reads entries 2p and 2p+1 of its row with one load
__device__ __forceinline__ long long slice_slot(long long base, int Lp, int R, int q, int e, int lane) {
  return Lp == 1 ? base + 32 * q + lane : base + ((long long)(e >> 1) * R + q) * 64 + 2 * lane + (e & 1);
}

template <int W>
__device__ __forceinline__ double group_sum(double v) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off, W);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) { return group_sum<32>(v); }

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, off));
  return v;
}

// Block-wide reduction of NV values per thread (sum, or max where is_max[q]);
// result valid in thread 0. blockDim.x must be a multiple of 32 and <= 1024.
template <int NV>
__device__ __forceinline__ void block_reduce(double (&vals)[NV], const bool (&is_max)[NV]) {
  __shared__ double sh[32][NV];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) vals[q] = is_max[q] ? warp_max(vals[q]) : warp_sum(vals[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) sh[wid][q] = vals[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NV; ++q) {
      double v = lane < nw ? sh[lane][q] : 0.0;
      vals[q] = is_max[q] ? warp_max(v) : warp_sum(v);
    }
  }
  __syncthreads();
}

}  // namespace pdhg
