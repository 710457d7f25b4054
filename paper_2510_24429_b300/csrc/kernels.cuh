// Host-side launchers of the engine's kernels (internal).
#pragma once

#include "common.cuh"

namespace pdhg {

constexpr int TPB = 256;  // threads per block of every row kernel
constexpr int WARPS_PER_BLOCK = TPB / 32;
constexpr int STEP_TPB_MAX = 512;  // largest block of the step and evaluation kernels (option step_block)
constexpr int STEP_BLOCKS_PER_SM = 6;  // resident 256-thread step blocks per SM (the kernels' register cap)
constexpr int HOT_TPB = 1024;              // threads per block of the persistent dual step
constexpr int HOT_SMEM_MAX = 220 * 1024;   // shared memory it stages xbar[0, hot) in
constexpr int HOT_MAX = HOT_SMEM_MAX / 4;  // most xbar entries it stages (FP32; half of it in FP64)

// ---- setup (scaling, power iteration, vector helpers) ----------------------
void launch_row_absmax(const Hyb& M, double* out, int grid, cudaStream_t s);
void launch_row_abspow_sum(const Hyb& M, double alpha, double* out, int grid, cudaStream_t s);
void launch_inv_sqrt_or_one(const double* in, double* out, int len, int grid, cudaStream_t s);
// transposed == 0: M is Ahat (rows i, cols j); 1: M is Ahat^T (rows j, cols i);
// 2: M is the panel layout of Ahat^T (segment row r: column pcol[r], local
// row index c of row pbase[r] + c). Every entry becomes (r_i * a_ij) * s_j,
// the same operation order in every layout so that the copies of Ahat stay
// bit-identical.
void launch_scale(const Hyb& M, const double* r, const double* s, int transposed, int grid, cudaStream_t st,
                  const int* pcol = nullptr, const int* pbase = nullptr);
void launch_mul_inplace(double* d, const double* f, int len, int grid, cudaStream_t s);
void launch_mul(double* out, const double* a, const double* b, int len, int grid, cudaStream_t s);
void launch_div(double* out, const double* a, const double* b, int len, int grid, cudaStream_t s);
void launch_fill(double* v, double val, long long len, int grid, cudaStream_t s);
void launch_reciprocal(double* out, const double* in, int len, int grid, cudaStream_t s);
void launch_spmv(const Hyb& M, const double* x, double* y, int grid, cudaStream_t s);
// out[0] = sum v^2 (deterministic two-stage reduction through `partials`)
void launch_sumsq(const double* v, int len, double* partials, int nb, double* out, cudaStream_t s);
// v = w / sqrt(*s2) when *s2 > 0 (else v unchanged)
void launch_div_by_norm(double* v, const double* w, const double* s2, int len, int grid, cudaStream_t s);
// eta, omega0, tau, sigma from the device scalars (norm^2 estimate, ||chat||^2, ||bhat||^2, ||b||^2, ||c||^2)
void launch_finish_setup(DevState* st, const double* scal, double step_factor, int primal_weight, cudaStream_t s);

// ---- iteration --------------------------------------------------------------
// x' = max(0, x - tau (chat - Ahat^T y)); xbar = 2x' - x; x <- x'; xsum += x'
// st: the problem's state; for a batch, the instances' states and binst maps
// every block to its instance (blocks of converged instances return at once)
// (u_begin: first unit of At to process; the units before it are left to the
// panel-tiled pass)
void launch_primal_step(const Hyb& At, const double* y, const double* ch, double* x, double* xbar, double* xsum,
                        const DevState* st, int accumulate, int grid, cudaStream_t s, const int* binst = nullptr,
                        int tpb = TPB, int u_begin = 0);
// y' = y + sigma (bhat - Ahat xbar); y <- y'; ysum += y'
void launch_dual_step(const Hyb& A, const double* xbar, const double* bh, double* y, double* ysum,
                      const DevState* st, int accumulate, int grid, cudaStream_t s, const int* binst = nullptr,
                      int tpb = TPB);
// reflected Halpern form of the two half-steps (values vals of type V,
// vectors and arithmetic in precision T): it = index of the step within the
// launches since st->t was last updated; xr, yr = the anchor (the last
// restart point). V = float with T = double: the unscaled values (Hyb::u32),
// with the scaling D_c (dc) and D_r (dr); y is then D_r y as written to yg
// by the dual step, and xbar holds D_c xbar.
template <class T, class V = T>
void launch_primal_step_halpern(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, const T* xr,
                                const DevState* st, int it, int grid, cudaStream_t s, int tpb,
                                const int* binst = nullptr, int u_begin = 0, const T* dc = nullptr,
                                const T* lo = nullptr);
template <class T, class V = T>
void launch_dual_step_halpern(const Hyb& A, const V* vals, const T* xbar, const T* bh, T* y, const T* yr,
                              const DevState* st, int it, int grid, cudaStream_t s, int tpb,
                              const int* binst = nullptr, const T* dr = nullptr, T* yg = nullptr);
// the same two half-steps in FP32 (values At.v32 / A.v32, FP32 vectors and
// accumulation); tau and sigma are read from the FP64 state and rounded
void launch_primal_step32(const Hyb& At, const float* y, const float* ch, float* x, float* xbar, float* xsum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb = TPB,
                          int u_begin = 0, const float* lo = nullptr);
void launch_dual_step32(const Hyb& A, const float* xbar, const float* bh, float* y, float* ysum, const DevState* st,
                        int accumulate, int grid, cudaStream_t s, int tpb = TPB);
// the two half-steps in FP64 on the unscaled values in FP32 (At.u32 / A.u32,
// exact when every value of A is an FP32 number): the primal step gathers
// yg = D_r y and scales its sums by dc = D_c, writing D_c xbar to xbar; the
// dual step gathers that, scales its sums by dr = D_r and writes D_r y' to yg
void launch_primal_step_u(const Hyb& At, const double* yg, const double* ch, double* x, double* xbar, double* xsum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb, int u_begin,
                          const double* dc);
void launch_dual_step_u(const Hyb& A, const double* xbar, const double* bh, double* y, double* ysum,
                        const DevState* st, int accumulate, int grid, cudaStream_t s, int tpb, const double* dr,
                        double* yg);
// flag[0] = 1 if some v[i] is not exactly an FP32 number (flag is not cleared)
void launch_fp32_inexact(const double* v, long long len, int* flag, cudaStream_t s);
// precision conversions and the FP32 counterparts of make_average / apply
void launch_narrow(float* dst, const double* src, long long len, int grid, cudaStream_t s);
void launch_widen(double* dst, const float* src, long long len, int grid, cudaStream_t s);
// 16-bit copies of column indices below 65536 (the panel layout's panel-relative rows)
void launch_narrow_index(unsigned short* dst, const int* src, long long len, int grid, cudaStream_t s);
void launch_make_average32(const float* xs, const float* ys, const float* x, const float* y, double* xa, double* ya,
                           int n, int m, const DevState* st, int grid, cudaStream_t s);
void launch_apply32(const DevState* st, float* x32, float* y32, double* x, double* y, const double* xa,
                    const double* ya, double* xr, double* yr, float* xs, float* ys, int n, int m, int grid,
                    cudaStream_t s);
// option refine32: FP32 phases iterate on FP32 corrections (x32, y32) to the
// last restart point (xr, yr), held in FP64. x = xr + x32, y = yr + y32
void launch_widen_delta(double* dst, const double* ref, const float* d, long long len, int grid, cudaStream_t s);
// FP64 averages xa = xr + xs / t (t = st->t; t == 0: the current point)
void launch_make_average32_delta(const float* xs, const float* ys, const float* x, const float* y, const double* xr,
                                 const double* yr, double* xa, double* ya, int n, int m, const DevState* st, int grid,
                                 cudaStream_t s);
// the decision applied in refined FP32 phases: a restart moves the FP64
// reference (xr, yr) to the new point and clears the corrections and sums;
// taking the average sets the corrections to xa - xr
void launch_apply32_delta(const DevState* st, float* x32, float* y32, double* x, double* y, const double* xa,
                          const double* ya, double* xr, double* yr, float* xs, float* ys, int n, int m, int grid,
                          cudaStream_t s);
// re-centring after a restart (or always, with force): ch32 = chat - Ahat^T yr,
// lo32 = -xr rounded toward zero (At: Ahat^T); bh32 = bhat - Ahat xr (A: Ahat),
// computed in FP64 and rounded to FP32
void launch_recenter(const Hyb& A, const Hyb& At, const double* xr, const double* yr, const double* bh,
                     const double* ch, float* bh32, float* ch32, float* lo32, const DevState* st, int force, int grA,
                     int grT, cudaStream_t s);
// PDLP-style sums at the switch to FP64: xsum = t xr + xsum32 (t = st->t)
void launch_widen_sum_delta(double* dst, const double* ref, const float* sum32, long long len, const DevState* st,
                            int grid, cudaStream_t s);
// restart reference := st->cur, t := 0 (start of the FP64 polishing phase)
void launch_promote_state(DevState* st, cudaStream_t s);
// restart reference := st->cur, k := t := 0, snapshots off, termination test
// term_mode (start of a feasibility polishing phase)
void launch_polish_begin(DevState* st, int term_mode, cudaStream_t s);
// ---- adjoint ----------------------------------------------------------------
// one reversed iteration: adjoint primal half-step over Ahat^T then adjoint
// dual half-step over Ahat (values valsAt / valsA in precision T)
template <class T>
void launch_adj_step(const Hyb& A, const Hyb& At, const T* valsA, const T* valsAt, const T* xnext, T* gx, T* gy,
                     T* gu, T* gch, T* gbh, const DevState* st, cudaStream_t s);
template <class T>
void launch_adj_seed(T* g, const double* in, const int* perm, const double* d, int len, int grid, cudaStream_t s);
template <class T>
void launch_adj_unseed(double* out, const T* g, const int* perm, const double* d, int len, int grid, cudaStream_t s);
// ---- panel-tiled primal half-step (option primal_panels) --------------------
#ifndef PDHG_PANEL_TPB
#define PDHG_PANEL_TPB 1024
#endif
#ifndef PDHG_PANEL_MINB32
#define PDHG_PANEL_MINB32 1
#endif
constexpr int PANEL_TPB = PDHG_PANEL_TPB;     // threads per block of the panel pass
// resident FP32 panel blocks per SM the compiler plans for: one (64 registers, no spills) ran
// faster than two (32 registers, spilling) on the 1e6 x 3e6 LP
constexpr int PANEL_MINB32 = PDHG_PANEL_MINB32;
// entry pairs of a panel segment row a thread loads ahead (the slice loop's
// unroll) in the panel pass, FP32 and FP64 steps: 4 ran 3% faster than 2 in
// FP32 on the 1e6 x 3e6 Zipf LP; in FP64, 4 and 6 were 0.5% and 2% slower
constexpr int PANEL_UNROLL32 = 4, PANEL_UNROLL64 = 2;
constexpr int PANEL_SMEM_MAX = 220 * 1024;  // shared memory of one panel block
struct PanelLayout {
  int m = 0;                // rows of A (length of y)
  int ncols = 0;            // columns covered: internal columns [0, ncols), the longest rows of A^T
  int ulong = 0;            // ... which are the rows of units [0, ulong) of At; the direct primal step
                            // takes the units from ulong on
  int rows = 0;             // the tallest panel's height (entries of y in shared memory)
  int panels = 0;           // number of panels
  int* pfirst = nullptr;    // [panels + 1] first row of every panel (multiples of 16; pfirst[panels] = m)
  int* ustart = nullptr;    // [panels + 1] first unit of every panel in Pn
  int* segout = nullptr;    // [segments] position of every segment row of Pn in the dense panel-major
                            // partial sums (panel * ncols + column; slots of absent segments stay 0)
  int blocks = 0;           // blocks of the panel pass (one wave)
  int4* binfo = nullptr;    // [blocks] (panel, index among its panel's blocks, its panel's block count, 0)
};
// allow the panel kernels their shared memory (once per device, outside graph capture)
cudaError_t configure_primal_panels();
// ---- streamed step kernels (option stream_steps, stream.cu) ----------------
// Every warp owns `depth` shared-memory slots; a slot holds one bulk-copied
// piece of at most STREAM_PIECE matrix slots (indices and values) and the
// staged rows (at most STREAM_PRE_CAP per vector, alignment included) of up to
// STREAM_NPRE of the step's vectors.
constexpr int STREAM_PIECE = 512;  // a multiple of 128 (the long-row lane pattern)
constexpr int STREAM_PRE_CAP = 136;
constexpr int STREAM_NPRE = 4;
constexpr int STREAM_TPB_MAX = 512;
constexpr int STREAM_SMEM_MAX = 227 * 1024 - 256;  // dynamic shared memory of one block (static part beside it)
constexpr size_t stream_slot_bytes(size_t t, size_t v) {
  return (size_t)STREAM_PIECE * (4 + v) + (size_t)STREAM_NPRE * STREAM_PRE_CAP * t;
}
struct StreamCfg {
  int warps = 8;   // warps per block
  int depth = 3;   // slots per warp
  int blocks = 0;  // grid (resident blocks per SM x SMs), set by configure_stream
  size_t smem = 0; // dynamic shared memory per block, set by configure_stream
};
size_t stream_smem(const StreamCfg& c, size_t t, size_t v);
// allow the kernels of value type V / arithmetic T their shared memory and
// size the grid (once per context, outside graph capture)
template <class T, class V>
cudaError_t configure_stream(StreamCfg& c, int sms);
// the dual half-step over every unit of A (halpern_it >= 0: the Halpern form
// with anchor ysum_or_yr; else y_sum += y' when accumulate); V = float with
// T = double: the unscaled values with D_r (dr) and the gathered copy yg
template <class T, class V>
void launch_stream_dual(const Hyb& A, const V* vals, const T* xbar, const T* bh, T* y, T* ysum_or_yr, DevState* st,
                        int accumulate, int halpern_it, const T* dr, T* yg, const StreamCfg& c, cudaStream_t s);
// the primal half-step over the units of At from u_begin on and, when
// ncols > 0, the combine of the long columns [0, ncols) from their panel
// partial sums (panels of them, panel-major); lo: the FP32 projection bounds
// of option refine32 (nullptr: 0)
template <class T, class V>
void launch_stream_primal(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, T* xsum_or_xr,
                          DevState* st, int accumulate, int halpern_it, int u_begin, int ncols, int panels,
                          const T* partial, const T* dc, const StreamCfg& c, cudaStream_t s, const T* lo = nullptr);
// pass 1: per-(column, panel) partial sums of the long columns
template <class T, class V = T>
void launch_panel_pass(const Hyb& Pn, const V* vals, const PanelLayout& L, const T* y, T* partial, cudaStream_t s);
// pass 2 fused with the short columns' direct step (short_grid: blocks of tpb
// threads for the units of At from L.ncols on): the long columns' sums and
// update, and the direct step; halpern_it >= 0: the reflected Halpern update
// of step halpern_it with xsum as the anchor
// (V = float with T = double: the unscaled values, with dc = D_c, as above)
template <class T, class V = T>
void launch_primal_short_combine(const Hyb& At, const V* vals, const T* y, const T* ch, T* x, T* xbar, T* xsum,
                                 const DevState* st, int accumulate, int short_grid, const PanelLayout& L,
                                 const T* partial, int tpb, cudaStream_t s, int halpern_it = -1,
                                 const T* dc = nullptr, const T* lo = nullptr, int overlap = 0,
                                 int wave_blocks = 0);
// the dual step, persistent (grid = number of SMs), with xbar[0, hot) staged
// in shared memory (hot * sizeof(T) <= HOT_SMEM_MAX), values vals in
// precision T; halpern_it >= 0: the reflected Halpern form of step
// halpern_it, with ysum holding the anchor
template <class T>
void launch_dual_step_hot(const Hyb& A, const T* vals, const T* xbar, int hot, const T* bh, T* y, T* ysum,
                          const DevState* st, int accumulate, int grid, cudaStream_t s, int halpern_it = -1);
void launch_add_counters(DevState* st, long long dk, cudaStream_t s);

// ---- evaluation -------------------------------------------------------------
void launch_make_average(const double* xs, const double* ys, const double* x, const double* y, double* xa,
                         double* ya, int n, int m, const DevState* st, int grid, cudaStream_t s);
// Partial sums of one point into partials[nb][NQ]; xr/yr may be null (no
// restart distances); idr, idc = 1 / D_r, 1 / D_c. Both sides use the same nb blocks.
void launch_eval_point(const Hyb& A, const Hyb& At, const double* px, const double* py, const double* bh,
                       const double* ch, const double* idr, const double* idc, const double* xr, const double* yr,
                       double* partials, int nb, cudaStream_t s, const DevState* sts = nullptr,
                       const int* binst = nullptr, int tpb = TPB);
// The current point's evaluation with the parts of its fixed-point residual
// (restart_scheme = 1; single LPs): writes the PDHG step T(px, py) into
// (xt, yt), using ht (m entries) for Ahat xt; tau and sigma from *st
void launch_eval_point_fp(const Hyb& A, const Hyb& At, const double* px, const double* py, const double* bh,
                          const double* ch, const double* idr, const double* idc, const double* xr, const double* yr,
                          double* partials, int nb, const DevState* st, double* xt, double* ht, double* yt,
                          int spmv_grid, cudaStream_t s, int tpb);
// ---- batch (count instances; xoff/yoff: instance ranges of the column and row vectors) ----
void launch_decide_b(DevState* sts, int count, cudaStream_t s);
void launch_add_counters_b(DevState* sts, int count, long long dk, cudaStream_t s);
void launch_init_restart_ref_b(DevState* sts, int count, cudaStream_t s);
// sums of each instance's block partials into the EvalSums at out0 + i * stride bytes
void launch_eval_finalize_b(const double* partials, const int* bstart, int count, EvalSums* out0, size_t stride,
                            cudaStream_t s);
void launch_make_average_b(const double* xs, const double* ys, const double* x, const double* y, double* xa,
                           double* ya, const int* xoff, const int* yoff, const DevState* sts, int count, int gx,
                           cudaStream_t s);
void launch_apply_b(const DevState* sts, double* x, double* y, const double* xa, const double* ya, double* xr,
                    double* yr, double* xs, double* ys, const int* xoff, const int* yoff, int count, int gx,
                    cudaStream_t s);
void launch_sumsq_b(const double* v, const int* off, int count, double* out, int ostride, cudaStream_t s);
void launch_div_by_norm_b(double* v, const double* w, const double* s2, int sstride, const int* off, int count,
                          int gx, cudaStream_t s);
// ---- the whole batch in one cooperative launch (option persistent = 2) ----
enum { BATCH_ERR_NONE = 0, BATCH_ERR_TIMEOUT = 1, BATCH_ERR_NUMERIC = 2 };
// device-resident control of one launch (the host writes the first four
// fields before each launch, so a captured graph serves every call)
struct BatchCtl {
  long long k0;         // iterations of the context before this launch (the evaluation schedule)
  long long max_iters;  // iterations this launch may run
  long long budget;     // clock cycles one barrier wait may last
  long long done;       // iterations run (written at the end)
  unsigned arrive, gen; // the grid barrier's counter and generation
  int error;            // BATCH_ERR_*
  int where;            // tag (count) of the barrier at which a wait gave up
  int active;           // instances not frozen
  int pad;
};
struct BatchArgs {
  Hyb A, At;
  const int *binst, *bstart, *xoff, *yoff;  // block -> instance; instance -> blocks, columns, rows
  int nvb, count, eval_every, restarts, halpern;
  double *x, *xbar, *xsum, *xr, *xavg, *y, *ysum, *yr, *yavg;
  const double *ch, *bh, *idc, *idr;
  double *part_avg, *part_cur;  // per-block evaluation sums, nvb * NQ each
  DevState* sts;
  BatchCtl* ctl;
  // scheduled snapshots (null when none are scheduled): stacked outputs in the
  // caller's numbering, and what packing them needs
  double *snap_x, *snap_y, *snap_z;
  const int *perm_x, *perm_y;
  const double *dc, *dr;
};
// batch snapshots: for every instance whose latest evaluation scheduled one,
// its candidate (x, y, z) on its problem as given into ox, oy, oz (stacked, in
// the caller's numbering)
void launch_snap_b(const Hyb& At, const DevState* sts, const int* binst, int nblocks, const int* perm_x,
                   const int* perm_y, const double* x, const double* y, const double* xa, const double* ya,
                   const double* ch, const double* dc, const double* dr, double* ox, double* oy, double* oz,
                   const int* yoff, int count, int gx, int tpb, cudaStream_t s);
// blocks of the cooperative grid (all resident: SMs x blocks per SM at tpb threads)
cudaError_t batch_solve_grid(int tpb, int* grid);
cudaError_t launch_batch_solve(const BatchArgs& a, int grid, int tpb, cudaStream_t s);
// start vector of the power iteration (unnormalized) for every instance
// (off == nullptr: one problem of n columns, count 1)
void launch_power_start(double* v, const int* perm_x, const int* off, int count, int n, int gx, cudaStream_t s);
void launch_finish_setup_b(DevState* sts, int count, const double* scal, int sstride, double step_factor,
                           int primal_weight, cudaStream_t s);
void launch_eval_finalize(const double* partials, int nb, EvalSums* out, cudaStream_t s);
void launch_init_restart_ref(DevState* st, cudaStream_t s);
void launch_decide(DevState* st, TraceRec* trace, cudaStream_t s);
void launch_apply(const DevState* st, double* x, double* y, const double* xa, const double* ya, double* xr,
                  double* yr, double* xs, double* ys, int n, int m, int grid, cudaStream_t s);
// (x, y, z) on the problem as given, in the caller's numbering:
// x[perm_x[j]] = D_c xhat_j, y[perm_y[i]] = D_r yhat_i,
// z[perm_x[j]] = max(0, chat_j - (Ahat^T yhat)_j) / D_c_j.
void launch_pack_solution(const Hyb& At, const int* perm_x, const int* perm_y, const double* px, const double* py,
                          const double* ch, const double* dc, const double* dr, double* ox, double* oy, double* oz,
                          int grid, cudaStream_t s);

// ---- layout construction (layout.cu) ----------------------------------------
// error bits of the device-side CSR validation
enum { LAYOUT_BAD_ROW_PTR = 1, LAYOUT_BAD_COLUMN = 2, LAYOUT_UNSORTED = 4, LAYOUT_NOT_FINITE = 8 };
void launch_validate_csr(long long m, long long n, long long nnz, const long long* rp, const int* ci,
                         const double* v, int* flags, cudaStream_t s);
void launch_check_finite(const double* v, long long len, int* flags, cudaStream_t s);
// out[i] = instance of element i given the count + 1 offsets off
void launch_instance_of(const int* off, int count, long long len, int* out, cudaStream_t s);
// block-diagonal global CSR (grp [M+1], gci [Z]) and the global row of every
// entry from the instances' local arrays (instance i: rows from lrp + rpoff[i],
// entries from zoff[i], columns shifted by xoff[i]); rinst null for one LP
void launch_globalize(const long long* lrp, const int* lci, const long long* rpoff, const long long* zoff,
                      const int* xoff, const int* yoff, const int* rinst, long long M, long long Z, long long* grp,
                      int* gci, int* rowid, cudaStream_t s);
// row lengths of A (lenA), of A^T (lenT), and their maxima (maxes[0], maxes[1])
void launch_lengths(const long long* grp, long long M, const int* gci, long long Z, long long N, int* lenA,
                    int* lenT, unsigned* maxes, cudaStream_t s);
void launch_length_keys(const int* len, long long cnt, const int* inst, int maxlen, int lbits,
                        unsigned long long* keys, int* vals, cudaStream_t s, const int* sec = nullptr,
                        int sbits = 0);
// sec[c] = internal row (iy) of column c's only entry if column c has one
// entry, else 0 (the secondary key that orders one-entry columns by row)
void launch_singleton_rows(const int* gci, const int* rowid, long long Z, const int* lenT, const int* iy, int* sec,
                           long long N, cudaStream_t s);
// transpose sort keys, fed in internal row order (rpi: exclusive scan of the
// internal rows' lengths)
void launch_transpose_keys(const long long* grp, const int* py, const long long* rpi, long long M, const int* gci,
                           const int* ix, unsigned* keys, int* vals, cudaStream_t s);
// panel layout of A^T (segments = runs of one row of A^T inside one panel;
// panel p holds the internal rows [pfirst[p], pfirst[p + 1])); see
// build_panels in pdhg_api.cu. cnt[i] += the entries of the first Z sorted
// entries of A^T in internal row i (cnt zeroed by the caller)
void launch_row_counts(long long Z, const int* sval, const int* rowid, const int* iy, int* cnt, cudaStream_t s);
void launch_panel_heads(const long long* tp, long long N, const int* sval, const int* rowid, const int* iy,
                        const int* pfirst, int P, int* head, int* panel, int* col, cudaStream_t s);
void launch_panel_segments(const int* head, const int* panel, const int* col, const long long* segpos, long long Z,
                           long long S, long long* seg_start, int* seg_panel, int* seg_col, cudaStream_t s);
void launch_panel_rowinfo(const int* sp, const int* seg_col, const int* seg_panel, const int* pfirst, long long S,
                          int* pcol, int* pbase, cudaStream_t s);
void launch_panel_keys(const long long* seg_start, const int* seg_panel, long long S, int maxlen, int lbits,
                       int* seg_len, unsigned long long* keys, int* vals, int* pcount, cudaStream_t s);
void launch_panel_dense_out(const int* pcol, const int* sp, const int* seg_panel, int ncols, long long S, int* out,
                            cudaStream_t s);
void launch_max_int(const int* v, long long len, unsigned* out, cudaStream_t s);
void launch_fill_units_P(const Hyb& H, const int* slen, const int* sp, const long long* seg_start,
                         const int* seg_panel, const int* sval, const int* rowid, const int* iy, const double* v,
                         const int* pfirst, cudaStream_t s);
void launch_invert(const int* p, long long len, int* inv, cudaStream_t s);
void launch_gather_int(const int* src, const int* p, long long len, int* out, cudaStream_t s);
void launch_gather_double(const double* src, const int* p, long long len, double* out, cudaStream_t s);
// workspace lengths (long long elements) of the radix sort's histogram and of the scan
long long radix_hist_len(long long N);
long long scan_ws_len(long long len);
// Stable ascending sort of N (key, value) pairs on the low `bits` bits of the
// keys; returns 0 if the result is in (keys, vals), 1 if in (keys_alt, vals_alt).
// hist: radix_hist_len(N) elements; ws: scan_ws_len(radix_hist_len(N)).
template <class K>
int radix_sort_pairs(K* keys, int* vals, K* keys_alt, int* vals_alt, long long N, int bits, long long* hist,
                     long long* ws, cudaStream_t s);
// out[0..len] = exclusive prefix sums of in[0..len) (out[len] = total); ws: scan_ws_len(len)
void launch_scan_int(const int* in, long long len, long long* out, long long* ws, cudaStream_t s);
// write the entries of every unit of H (unit tables, ci and v allocated; ci, v zeroed)
void launch_fill_units_A(const Hyb& H, const int* slen, const long long* grp, const int* py, const int* gci,
                         const int* ix, const double* v, cudaStream_t s);
void launch_fill_units_T(const Hyb& H, const int* slen, const long long* tp, const int* sval, const int* rowid,
                         const int* iy, const double* v, cudaStream_t s);

// ---- single-block solve loop (persistent.cu) ----------------------------------
constexpr int PERSIST_TPB = 512;
// most doubles of vectors one block holds in shared memory (7 n + 6 m)
constexpr long long PERSIST_MAX_DOUBLES = 28672;
struct PersistentArgs {
  long long max_iters;
  int eval_every, evaluating, restarts, batch;
  int n, m;                         // one LP: its sizes (xoff == nullptr)
  const int *xoff, *yoff, *ustart;  // batch: column, row and unit ranges per instance
  double *x, *xbar, *xsum, *xr, *xavg, *y, *ysum, *yr, *yavg;
  const double *ch, *idc, *bh, *idr;  // idc, idr: 1 / D_c, 1 / D_r
};
size_t persistent_smem_bytes(long long n, long long m);
// one block per instance; trace may be null
cudaError_t launch_solve_block(const Hyb& A, const Hyb& At, const PersistentArgs& a, int blocks, size_t smem,
                               DevState* sts, TraceRec* trace, cudaStream_t s);

// the step kernels use no shared memory: prefer the largest L1
void prefer_l1_for_step_kernels();

}  // namespace pdhg
