// Host engine behind the C ABI of include/pdhg.h.
//
// One context = one LP (or one batch of LPs) resident on one GPU. Setup
// validates the CSR (host inputs on the host, device inputs on the device),
// copies it to the device, and does everything else there: the renumbering of
// rows and columns by decreasing length, the transpose, the packing into the
// two matrix layouts (A and its transpose as long rows plus slices; see Hyb
// and layout.cu), Ruiz and Pock-Chambolle scaling, the power iteration for
// ||Ahat||_2, the primal weight, and the evaluation of the starting point. The solve loop launches the two fused half-steps per
// iteration and, every eval_every iterations, the evaluation kernels and the
// single-thread decision kernel; the host reads back one small status struct
// per evaluation (Section 3.1: one CPU thread launches the GPU kernels and
// fetches small amounts of data from GPU memory).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <functional>
#include <future>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/pdhg.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace pdhg;

namespace {

// An NVTX range over a phase of the engine's host code (setup, an evaluation
// block, a snapshot, the reverse pass, ...), so that a profiler's timeline
// (Nsight Systems, or ncu --nvtx) shows which phase enqueued which launches.
// NVTX3 is header-only: without a tool attached a range costs a call through
// a null function pointer.
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

}  // namespace

namespace {

thread_local std::string g_create_error = "no error";
constexpr int EV_POOL = 256;
constexpr int SNAP_SLOTS = 3;  // pinned host ring of completed snapshots
// PDHG_MIXED: iterations without a 10% gain in the FP32 phase before FP64
// takes over (PDHG itself plateaus for a few thousand iterations at times).
// A refined FP32 phase (refine32) follows the FP64 iteration's trajectory, so
// its plateaus are the method's own: it gets four times the window (on the
// 1e6 x 3e6 LP the cuPDLP+ form's plateaus between 1e-6 and 1e-8 passed the
// shorter window, and the refined FP32 iteration alone reached 1e-8 in as
// many iterations as FP64)
constexpr int64_t STALL_ITERS = 16384;
constexpr int64_t STALL_ITERS_REFINED = 4 * STALL_ITERS;

}  // namespace

// failures of calls without a context (pdhg_create, pdhg_kkt_noalloc) are
// reported by pdhg_last_error(NULL)
void pdhg_set_global_error(const char* msg) { g_create_error = msg; }

// The panel-tiled primal half-step's layout of Ahat^T (option primal_panels):
// the Hyb of segments, the panel table, the partial sums (FP64, FP32), and for
// setup only the column and first row of every segment row (for its scaling)
struct PanelSet {
  Hyb Pn;
  PanelLayout pl;
  double* partial = nullptr;
  float* partial32 = nullptr;
  int *col = nullptr, *base = nullptr;
};

struct pdhg_ctx {
  int64_t m = 0, n = 0, nnz = 0;
  pdhg_options opt{};
  int device = 0, sms = 148;
  cudaStream_t stream = nullptr, side = nullptr;
  bool own_stream = false;
  Hyb A, At;
  int* perm_x = nullptr;  // internal column -> caller's column
  int* perm_y = nullptr;  // internal row -> caller's row
  double *b = nullptr, *c = nullptr, *bh = nullptr, *ch = nullptr, *dr = nullptr, *dc = nullptr;
  double *idr = nullptr, *idc = nullptr;  // 1 / D_r, 1 / D_c (the evaluation multiplies)
  double *x = nullptr, *y = nullptr, *xbar = nullptr, *xsum = nullptr, *ysum = nullptr;
  double *xavg = nullptr, *yavg = nullptr, *xr = nullptr, *yr = nullptr;
  double *tmp_n = nullptr, *tmp_m = nullptr, *tmp_n2 = nullptr;
  // FP32 iteration state (PDHG_FP32 / PDHG_MIXED); the FP64 vectors above then
  // hold the evaluation copies until the FP64 polishing phase takes over
  float *x32 = nullptr, *xbar32 = nullptr, *xsum32 = nullptr, *y32 = nullptr, *ysum32 = nullptr;
  float *ch32 = nullptr, *bh32 = nullptr;
  bool phase32 = false;
  // batch (count > 1): instance-major layouts; instance i owns columns
  // [xoff[i], xoff[i+1]) and rows [yoff[i], yoff[i+1]) of the internal
  // numbering and blocks [bstart[i], bstart[i+1]) of every unit-grid launch
  int count = 1;
  std::vector<int> xoff_h, yoff_h, bstart_h;
  int *xoff = nullptr, *yoff = nullptr, *binst = nullptr, *bstart = nullptr;
  int nblocks = 0;
  // option persistent: first unit of every instance (count + 1; batch only) and
  // the shared memory of the single-block solve loop
  int* ustart = nullptr;
  size_t persist_smem = 0;
  // warps per block of the step and evaluation kernels (option step_block)
  int wpb = WARPS_PER_BLOCK;
  // panel-tiled primal step (option primal_panels): pan[0] is the layout of
  // FP64 steps (and of FP32 steps without pan[1]); pan[1] (pan32) an FP32-tuned
  // layout - shorter columns in the panels, twice the rows per panel - for the
  // FP32 phase of PDHG_MIXED
  bool panels_on = false;
  bool check_on_device = false;  // host inputs: checked on the device after the upload (a GPU was found)
  bool pan32 = false;
  PanelSet pan[2];
  // option values32: the FP64 steps read A.u32 / At.u32 / pan[0].Pn.u32 (A's
  // unscaled values, exactly) and gather yg = D_r y (written by the dual step,
  // refreshed from y at the start of every block) and D_c xbar (in xbar)
  bool vals_u = false;
  double* yg = nullptr;
  // option refine32: FP32 phases iterate on corrections to (xr, yr); lo32 =
  // the primal corrections' lower bounds -xr (rounded toward zero)
  bool refine = false;
  float* lo32 = nullptr;
  // PDHG_LOG (environment, read at create): one JSON line per evaluation is
  // appended to that file
  FILE* log = nullptr;
  std::chrono::steady_clock::time_point t_create = std::chrono::steady_clock::now();
  // option stream_steps: the streamed step kernels' launch shapes for
  // (T, V) = (double, double), (float, float), (double, float)
  bool stream_on = false;
  StreamCfg scfg[3];
  // CUDA graphs of one evaluation block, per precision phase (FP64, FP32)
  cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
  int64_t graph_launches[2] = {0, 0};
  int64_t graph_replays = 0;  // graph launches by pdhg_iterate
  // batch with persistent = 2: the cooperative launch's control block (device
  // and pinned host copies), its second set of evaluation partial sums, its
  // grid, and the graph that replays it
  BatchCtl* bctl = nullptr;
  BatchCtl* h_bctl = nullptr;
  double* partials_avg = nullptr;
  int bgrid = 0;
  // batch snapshots (eps_cross or snapshot_every set): the latest scheduled
  // snapshot of every instance, stacked (x n, y m, z n) in the caller's numbering
  double* bsnap = nullptr;
  // checked build (PDHG_CHECKED): the error word the kernels' range checks set
  unsigned* check = nullptr;
  cudaGraphExec_t bgraph = nullptr;
  bool bgraph_failed = false;
  // recording for the adjoint: (x_k, y_k) every checkpoint_every iterations
  std::vector<void*> ck_x, ck_y;
  void *w_x = nullptr, *w_y = nullptr, *w_xbar = nullptr, *w_seg = nullptr;
  void *g_x = nullptr, *g_y = nullptr, *g_u = nullptr, *g_ch = nullptr, *g_bh = nullptr;
  double* partials = nullptr;
  int nb_eval = 1;
  double* scal = nullptr;
  DevState* st = nullptr;
  DevState* h_st = nullptr;  // pinned
  EvalSums* kkt_sums = nullptr;
  EvalSums* h_kkt = nullptr;  // pinned
  TraceRec* trace = nullptr;
  double* sol = nullptr;  // (x n, y m, z n)
  // snapshot ring
  double* snap_dev[SNAP_SLOTS] = {};
  double* snap_host[SNAP_SLOTS] = {};
  cudaEvent_t snap_packed[SNAP_SLOTS] = {}, snap_done[SNAP_SLOTS] = {};
  int64_t snap_iter[SNAP_SLOTS] = {};
  double snap_rel[SNAP_SLOTS] = {};
  int64_t snap_count = 0;  // snapshots started (by the thread that iterates)
  // hand-off to consumer threads (pdhg_snapshot_wait): a host callback on the
  // side stream marks a slot complete; consumers copy it out holding a reader
  // count, and a slot is reused only when no reader holds it
  struct SnapLanded {
    pdhg_ctx* ctx;
    int slot;
    int64_t seq;
  };
  std::mutex snap_mu;
  std::condition_variable snap_cv;
  int64_t snap_seq[SNAP_SLOTS] = {};  // 1-based index of the complete snapshot in a slot, 0 while written
  int snap_readers[SNAP_SLOTS] = {};
  SnapLanded snap_cb[SNAP_SLOTS] = {};
  // kernel timing
  cudaEvent_t ev[3 * EV_POOL] = {};
  double ms_primal = 0, ms_dual = 0;
  int64_t launches_primal = 0, launches_dual = 0;
  int64_t launches = 0;  // kernels launched by pdhg_iterate (snapshot packing included)
  // host mirrors
  int64_t k = 0;
  int64_t promoted_at = -1;  // iteration at which the FP64 polishing phase began
  double best32 = 1e300;     // best relative KKT seen in the FP32 phase, and where
  int64_t best32_k = 0;
  bool converged = false;
  // feasibility polishing: saved main state, start point, phase results and
  // saved chat / bhat (allocated on the first attempt), the iteration count
  // from which the next attempt may start, and the attempt log
  double* fp_buf = nullptr;
  int64_t fp_next = 0;
  int64_t fp_iters = 0;
  bool fp_polished = false;
  std::vector<pdhg_polish_rec> fp_log;
  std::vector<void*> allocs;
  std::string err = "no error";
};

namespace {

pdhg_status fail(pdhg_ctx* ctx, pdhg_status s, const std::string& msg) {
  if (ctx)
    ctx->err = msg;
  else
    g_create_error = msg;
  return s;
}

// largest of three ratios, NaN if any is NaN (std::max would drop a NaN
// second operand and report a finite rel_kkt for a point with a NaN term)
double max3_nan(double a, double b, double c) {
  if (std::isnan(a) || std::isnan(b) || std::isnan(c)) return NAN;
  return std::max(a, std::max(b, c));
}

pdhg_status cuda_fail(pdhg_ctx* ctx, cudaError_t e, const char* what) {
  std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(ctx, e == cudaErrorMemoryAllocation ? PDHG_ERR_OOM : PDHG_ERR_CUDA, msg);
}

#define CK(ctx, call)                                        \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
  } while (0)

// Checked build: the kernels' error word, read (and cleared) after the work
// of a call; a set bit means an index outside its array was found and skipped
pdhg_status read_check(pdhg_ctx* ctx) {
#ifdef PDHG_CHECKED
  if (!ctx->check) return PDHG_OK;
  unsigned w = 0;
  CK(ctx, cudaMemcpyAsync(&w, ctx->check, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (w) {
    CK(ctx, cudaMemsetAsync(ctx->check, 0, sizeof(unsigned), ctx->stream));
    return fail(ctx, PDHG_ERR_INVALID,
                std::string("checked build: out-of-range ") +
                    ((w & CHECK_UNIT) ? "unit extent or row " : "") + ((w & CHECK_COLUMN) ? "column index " : "") +
                    "found in the device layout and skipped");
  }
#else
  (void)ctx;
#endif
  return PDHG_OK;
}

template <class T>
cudaError_t dalloc(pdhg_ctx* ctx, T** p, size_t count) {
  void* q = nullptr;
  // 64 bytes of slack: the streamed step kernels bulk-copy vectors in whole
  // 16-byte units, up to 12 bytes past a vector's last entry
  cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T) + 64);
  if (e == cudaSuccess) ctx->allocs.push_back(q);
  *p = static_cast<T*>(q);
  return e;
}

int vec_grid(const pdhg_ctx* ctx, long long len) {
  long long g = (len + TPB - 1) / TPB;
  return (int)std::max<long long>(1, std::min<long long>(g, (long long)ctx->sms * 8));
}

// one unit (long row or 32-row slice) per warp
int unit_grid(const pdhg_ctx* ctx, const Hyb& H) {
  return std::max(1, (H.units() + ctx->wpb - 1) / ctx->wpb);
}

// grid-stride launches (setup and evaluation kernels)
int stride_grid(const pdhg_ctx* ctx, const Hyb& H) { return std::min(unit_grid(ctx, H), ctx->sms * 8); }

// grid of the direct primal step over the units of Ahat^T that the panel pass
// leaves to it (the short rows, units [pl.ncols, n_units))
int short_grid(const pdhg_ctx* ctx, const PanelSet& ps) {
  const long long units = std::max<long long>(1, ctx->At.n_units - ps.pl.ulong);
  return (int)((units + ctx->wpb - 1) / ctx->wpb);
}

pdhg_status set_device(pdhg_ctx* ctx) {
  int cur = -1;
  CK(ctx, cudaGetDevice(&cur));
  if (cur != ctx->device) CK(ctx, cudaSetDevice(ctx->device));
  return PDHG_OK;
}

// Runs fn(t) for t in [0, T) on T host threads (the calling thread included).
template <class F>
void parallel_for(int T, F fn) {
  std::vector<std::thread> th;
  th.reserve(T > 1 ? T - 1 : 0);
  for (int t = 1; t < T; ++t) {
    try {
      th.emplace_back(fn, t);
    } catch (...) {  // no thread to be had: do the share here
      fn(t);
    }
  }
  fn(0);
  for (auto& x : th) x.join();
}

// host threads for a pass over `work` elements
int host_threads(int64_t work) {
  if (work < (1 << 20)) return 1;
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  return (int)std::min<int64_t>({(int64_t)hw, 32, work >> 19});
}

bool all_finite(const double* v, int64_t len) {
  const int T = host_threads(len);
  std::vector<char> ok(T, 1);
  parallel_for(T, [&](int t) {
    const int64_t a = len * t / T, b = len * (t + 1) / T;
    for (int64_t i = a; i < b; ++i)
      if (!std::isfinite(v[i])) {
        ok[t] = 0;
        return;
      }
  });
  return std::all_of(ok.begin(), ok.end(), [](char c) { return c != 0; });
}

// Host checks of one LP, one pass over the entries in parallel over row
// ranges: every row's pointers are checked before its entries are read, so no
// read leaves [0, nnz). Precedence of the messages: a decreasing row_ptr
// anywhere, then the first bad column index (by row range), then NaN/Inf in
// the data. Touches no global state (it runs beside the context's set-up);
// *msg gets the failure's description.
pdhg_status check_lp(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                     const double* val, const double* b, const double* c, const char** msg) {
  auto fail = [msg](pdhg_status st, const char* text) {
    *msg = text;
    return st;
  };
  if (m < 1 || n < 1 || m >= (1LL << 31) - 1 || n >= (1LL << 31) - 1)
    return fail(PDHG_ERR_INVALID, "m and n must be in [1, 2^31 - 1)");
  if (nnz < 0 || nnz >= (1LL << 31) - 1) return fail(PDHG_ERR_INVALID, "nnz must be in [0, 2^31 - 1)");
  if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || !b || !c)
    return fail(PDHG_ERR_INVALID, "NULL array argument");
  if (row_ptr[0] != 0 || row_ptr[m] != nnz)
    return fail(PDHG_ERR_INVALID, "row_ptr[0] != 0 or row_ptr[m] != nnz");
  enum { OK = 0, BAD_PTR = 1, BAD_RANGE = 2, BAD_ORDER = 3 };
  const int T = host_threads(nnz + m);
  std::vector<int> bad(T, OK);
  std::vector<char> finite(T, 1);
  parallel_for(T, [&](int t) {
    const int64_t r0 = m * t / T, r1 = m * (t + 1) / T;
    const unsigned un = (unsigned)n;
    const unsigned long long EXP = 0x7ff0000000000000ull;
    unsigned long long nonfinite = 0;
    for (int64_t i = r0; i < r1; ++i) {
      const int64_t a = row_ptr[i], e = row_ptr[i + 1];
      if (e < a || a < 0 || e > nnz) {
        bad[t] = BAD_PTR;
        break;
      }
      // branch-free checks of the row (they vectorize); the rare failing row
      // is scanned again for its first bad entry
      unsigned out = 0, order = 0;
      for (int64_t k = a; k < e; ++k) {
        out |= (unsigned)col_idx[k] >= un;  // negative indices wrap to large values
        unsigned long long bits;
        memcpy(&bits, val + k, sizeof(bits));
        nonfinite |= (unsigned long long)((bits & EXP) == EXP);
      }
      for (int64_t k = a + 1; k < e; ++k) order |= col_idx[k] <= col_idx[k - 1];
      if (out | order) {
        for (int64_t k = a; k < e; ++k) {
          if ((unsigned)col_idx[k] >= un) {
            bad[t] = BAD_RANGE;
            break;
          }
          if (k > a && col_idx[k] <= col_idx[k - 1]) {
            bad[t] = BAD_ORDER;
            break;
          }
        }
        break;
      }
    }
    finite[t] = nonfinite == 0;
  });
  if (std::find(bad.begin(), bad.end(), (int)BAD_PTR) != bad.end())
    return fail(PDHG_ERR_INVALID, "row_ptr not non-decreasing");
  for (int t = 0; t < T; ++t) {
    if (bad[t] == BAD_RANGE) return fail(PDHG_ERR_INVALID, "column index out of range");
    if (bad[t] == BAD_ORDER)
      return fail(PDHG_ERR_INVALID, "column indices not strictly increasing within a row");
  }
  if (std::find(finite.begin(), finite.end(), (char)0) != finite.end() || !all_finite(b, m) || !all_finite(c, n))
    return fail(PDHG_ERR_NUMERIC, "NaN or Inf in the input data");
  return PDHG_OK;
}

pdhg_status validate_lp(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                        const double* val, const double* b, const double* c) {
  const char* msg = "";
  const pdhg_status st = check_lp(m, n, nnz, row_ptr, col_idx, val, b, c, &msg);
  return st == PDHG_OK ? st : fail(nullptr, st, msg);
}

pdhg_status read_state(pdhg_ctx* ctx) {
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

// Evaluate a point into *dst (EvalSums in device memory).
void eval_point(pdhg_ctx* ctx, const double* px, const double* py, const double* xr, const double* yr,
                EvalSums* dst) {
  launch_eval_point(ctx->A, ctx->At, px, py, ctx->bh, ctx->ch, ctx->idr, ctx->idc, xr, yr, ctx->partials,
                    ctx->nb_eval, ctx->stream, nullptr, nullptr, 32 * ctx->wpb);
  launch_eval_finalize(ctx->partials, ctx->nb_eval, dst, ctx->stream);
}

// The current point's evaluation with its fixed-point residual (option
// restart_scheme = 1): the PDHG step T(x, y) goes to (xavg, yavg), which this
// form (reflected Halpern, no averages) does not otherwise use.
void eval_point_fp(pdhg_ctx* ctx, EvalSums* dst) {
  launch_eval_point_fp(ctx->A, ctx->At, ctx->x, ctx->y, ctx->bh, ctx->ch, ctx->idr, ctx->idc, ctx->xr, ctx->yr,
                       ctx->partials, ctx->nb_eval, ctx->st, ctx->xavg, ctx->tmp_m, ctx->yavg,
                       stride_grid(ctx, ctx->A), ctx->stream, 32 * ctx->wpb);
  launch_eval_finalize(ctx->partials, ctx->nb_eval, dst, ctx->stream);
}

// During the FP32 phase: refresh the FP64 copies of the current iterate.
// (option refine32: the FP64 restart point plus the FP32 corrections)
void widen_current(pdhg_ctx* ctx) {
  if (ctx->refine) {
    launch_widen_delta(ctx->x, ctx->xr, ctx->x32, ctx->n, vec_grid(ctx, ctx->n), ctx->stream);
    launch_widen_delta(ctx->y, ctx->yr, ctx->y32, ctx->m, vec_grid(ctx, ctx->m), ctx->stream);
    return;
  }
  launch_widen(ctx->x, ctx->x32, ctx->n, vec_grid(ctx, ctx->n), ctx->stream);
  launch_widen(ctx->y, ctx->y32, ctx->m, vec_grid(ctx, ctx->m), ctx->stream);
}

// During the FP32 phase: the FP64 average of the current restart epoch.
void average32(pdhg_ctx* ctx) {
  const int n = (int)ctx->n, m = (int)ctx->m, gv = vec_grid(ctx, std::max(ctx->n, ctx->m));
  if (ctx->refine)
    launch_make_average32_delta(ctx->xsum32, ctx->ysum32, ctx->x32, ctx->y32, ctx->xr, ctx->yr, ctx->xavg,
                                ctx->yavg, n, m, ctx->st, gv, ctx->stream);
  else
    launch_make_average32(ctx->xsum32, ctx->ysum32, ctx->x32, ctx->y32, ctx->xavg, ctx->yavg, n, m, ctx->st, gv,
                          ctx->stream);
}

void point_of(pdhg_ctx* ctx, int which, const double** px, const double** py) {
  if (ctx->phase32) widen_current(ctx);
  if (which == PDHG_AVERAGE) {
    if (ctx->phase32)
      average32(ctx);
    else
      launch_make_average(ctx->xsum, ctx->ysum, ctx->x, ctx->y, ctx->xavg, ctx->yavg, (int)ctx->n, (int)ctx->m,
                          ctx->st, vec_grid(ctx, std::max(ctx->n, ctx->m)), ctx->stream);
    *px = ctx->xavg;
    *py = ctx->yavg;
  } else if (which == PDHG_LAST_RESTART) {
    *px = ctx->xr;
    *py = ctx->yr;
  } else {
    *px = ctx->x;
    *py = ctx->y;
  }
}

// Save (x_k, y_k) when k is a multiple of checkpoint_every and not saved yet.
pdhg_status record_checkpoint(pdhg_ctx* ctx, int64_t k) {
  const int64_t C = ctx->opt.checkpoint_every;
  if (k % C != 0 || (int64_t)ctx->ck_x.size() != k / C) return PDHG_OK;
  const size_t es = ctx->phase32 ? sizeof(float) : sizeof(double);
  char *cx = nullptr, *cy = nullptr;
  CK(ctx, dalloc(ctx, &cx, es * ctx->n));
  CK(ctx, dalloc(ctx, &cy, es * ctx->m));
  CK(ctx, cudaMemcpyAsync(cx, ctx->phase32 ? (void*)ctx->x32 : (void*)ctx->x, es * ctx->n, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  CK(ctx, cudaMemcpyAsync(cy, ctx->phase32 ? (void*)ctx->y32 : (void*)ctx->y, es * ctx->m, cudaMemcpyDeviceToDevice,
                          ctx->stream));
  ctx->ck_x.push_back(cx);
  ctx->ck_y.push_back(cy);
  return PDHG_OK;
}

// Reverse pass over every iteration run so far, in precision T.
pdhg_status primal_step(pdhg_ctx* ctx, bool f32, const void* y, void* x, void* xbar, void* xsum, int accumulate,
                        int grT, int tpb);

template <class T>
pdhg_status backward_impl(pdhg_ctx* ctx, const double* dx, const double* dy, double* dc, double* db) {
  Range nvtx_range("pdhg/backward");
  const int64_t K = ctx->k, C = ctx->opt.checkpoint_every, n = ctx->n, m = ctx->m;
  const bool f32 = std::is_same<T, float>::value;
  cudaStream_t s = ctx->stream;
  if (!ctx->g_x) {
    CK(ctx, dalloc(ctx, (T**)&ctx->w_x, n));
    CK(ctx, dalloc(ctx, (T**)&ctx->w_y, m));
    CK(ctx, dalloc(ctx, (T**)&ctx->w_xbar, n));
    CK(ctx, dalloc(ctx, (T**)&ctx->w_seg, (size_t)C * n));
    CK(ctx, dalloc(ctx, (T**)&ctx->g_x, n));
    CK(ctx, dalloc(ctx, (T**)&ctx->g_y, m));
    CK(ctx, dalloc(ctx, (T**)&ctx->g_u, n));
    CK(ctx, dalloc(ctx, (T**)&ctx->g_ch, n));
    CK(ctx, dalloc(ctx, (T**)&ctx->g_bh, m));
  }
  T *wx = (T*)ctx->w_x, *wy = (T*)ctx->w_y, *wxbar = (T*)ctx->w_xbar, *seg = (T*)ctx->w_seg;
  T *gx = (T*)ctx->g_x, *gy = (T*)ctx->g_y, *gu = (T*)ctx->g_u, *gch = (T*)ctx->g_ch, *gbh = (T*)ctx->g_bh;
  const int gn = vec_grid(ctx, n), gm = vec_grid(ctx, m);
  const int grT = unit_grid(ctx, ctx->At), grA = unit_grid(ctx, ctx->A), tpb = 32 * ctx->wpb;
  launch_adj_seed<T>(gx, dx, ctx->perm_x, ctx->dc, (int)n, gn, s);
  launch_adj_seed<T>(gy, dy, ctx->perm_y, ctx->dr, (int)m, gm, s);
  CK(ctx, cudaMemsetAsync(gch, 0, sizeof(T) * n, s));
  CK(ctx, cudaMemsetAsync(gbh, 0, sizeof(T) * m, s));
  for (int64_t sg = (K - 1) / C; sg >= 0 && K > 0; --sg) {
    const int64_t start = sg * C, end = std::min(start + C, K);
    // recompute the segment's forward pass from its checkpoint
    CK(ctx, cudaMemcpyAsync(wx, ctx->ck_x[sg], sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    CK(ctx, cudaMemcpyAsync(wy, ctx->ck_y[sg], sizeof(T) * m, cudaMemcpyDeviceToDevice, s));
    for (int64_t k = start; k < end; ++k) {
      pdhg_status rs = primal_step(ctx, f32, wy, wx, wxbar, nullptr, 0, grT, tpb);
      if (rs != PDHG_OK) return rs;
      if (f32)
        launch_dual_step32(ctx->A, (const float*)wxbar, ctx->bh32, (float*)wy, nullptr, ctx->st, 0, grA, s, tpb);
      else
        launch_dual_step(ctx->A, (const double*)wxbar, ctx->bh, (double*)wy, nullptr, ctx->st, 0, grA, s, nullptr,
                         tpb);
      CK(ctx, cudaMemcpyAsync(seg + (k - start) * n, wx, sizeof(T) * n, cudaMemcpyDeviceToDevice, s));
    }
    // reverse it
    const T* valsA = f32 ? (const T*)ctx->A.v32 : (const T*)ctx->A.v;
    const T* valsAt = f32 ? (const T*)ctx->At.v32 : (const T*)ctx->At.v;
    for (int64_t k = end - 1; k >= start; --k)
      launch_adj_step<T>(ctx->A, ctx->At, valsA, valsAt, seg + (k - start) * n, gx, gy, gu, gch, gbh, ctx->st, s);
    CK(ctx, cudaGetLastError());
  }
  launch_adj_unseed<T>(dc, gch, ctx->perm_x, ctx->dc, (int)n, gn, s);
  launch_adj_unseed<T>(db, gbh, ctx->perm_y, ctx->dr, (int)m, gm, s);
  CK(ctx, cudaGetLastError());
  return PDHG_OK;
}

// host callback after a snapshot's copy to pinned memory (runs on a CUDA
// thread: no CUDA calls here)
void CUDART_CB snapshot_landed(void* p) {
  auto* d = static_cast<pdhg_ctx::SnapLanded*>(p);
  pdhg_ctx* ctx = d->ctx;
  {
    std::lock_guard<std::mutex> lk(ctx->snap_mu);
    ctx->snap_seq[d->slot] = d->seq;
  }
  ctx->snap_cv.notify_all();
}

pdhg_status take_snapshot(pdhg_ctx* ctx) {
  Range nvtx_range("pdhg/snapshot");
  const int slot = (int)(ctx->snap_count % SNAP_SLOTS);
  if (!ctx->snap_host[slot]) {
    // ring slots are allocated on first use (pinned memory is slow to allocate)
    const int64_t len = 2 * ctx->n + ctx->m;
    CK(ctx, dalloc(ctx, &ctx->snap_dev[slot], len));
    CK(ctx, cudaMallocHost(&ctx->snap_host[slot], sizeof(double) * len));
    CK(ctx, cudaEventCreateWithFlags(&ctx->snap_packed[slot], cudaEventDisableTiming));
    CK(ctx, cudaEventCreateWithFlags(&ctx->snap_done[slot], cudaEventDisableTiming));
  }
  // the slot's previous copy and its callback are done
  if (ctx->snap_count >= SNAP_SLOTS) CK(ctx, cudaEventSynchronize(ctx->snap_done[slot]));
  {
    std::unique_lock<std::mutex> lk(ctx->snap_mu);
    // a consumer thread still copying this slot out: wait for it (bounded)
    if (!ctx->snap_cv.wait_for(lk, std::chrono::seconds(60), [&] { return ctx->snap_readers[slot] == 0; }))
      return fail(ctx, PDHG_ERR_TIMEOUT, "a snapshot consumer held a ring slot for more than 60 s");
    ctx->snap_seq[slot] = 0;
    ctx->snap_iter[slot] = ctx->h_st->k;
    ctx->snap_rel[slot] = ctx->h_st->cand_rel_kkt;
  }
  const bool avg = ctx->h_st->candidate == KIND_AVG;
  const double* px = avg ? ctx->xavg : ctx->x;
  const double* py = avg ? ctx->yavg : ctx->y;
  double* base = ctx->snap_dev[slot];
  launch_pack_solution(ctx->At, ctx->perm_x, ctx->perm_y, px, py, ctx->ch, ctx->dc, ctx->dr, base, base + ctx->n,
                       base + ctx->n + ctx->m, stride_grid(ctx, ctx->At), ctx->stream);
  CK(ctx, cudaGetLastError());
  CK(ctx, cudaEventRecord(ctx->snap_packed[slot], ctx->stream));
  CK(ctx, cudaStreamWaitEvent(ctx->side, ctx->snap_packed[slot], 0));
  CK(ctx, cudaMemcpyAsync(ctx->snap_host[slot], base, sizeof(double) * (2 * ctx->n + ctx->m), cudaMemcpyDeviceToHost,
                          ctx->side));
  ctx->snap_cb[slot] = {ctx, slot, ctx->snap_count + 1};
  CK(ctx, cudaLaunchHostFunc(ctx->side, snapshot_landed, &ctx->snap_cb[slot]));
  // recorded after the callback, so that waiting on it also waits for the callback
  CK(ctx, cudaEventRecord(ctx->snap_done[slot], ctx->side));
  ctx->snap_count += 1;
  return PDHG_OK;
}

// ---- layout construction ---------------------------------------------------

// Device memory owned by one setup call, released (after the stream is idle)
// when the call returns.
struct Scratch {
  cudaStream_t s = nullptr;
  std::vector<void*> ptrs;
  explicit Scratch(cudaStream_t st) : s(st) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    if (s) cudaStreamSynchronize(s);
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t take(T** p, size_t count) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(1, count) * sizeof(T));
    if (e == cudaSuccess) {
      ptrs.push_back(q);
      *p = static_cast<T*>(q);
    }
    return e;
  }
};

// Unit table of one layout (see Hyb), built on the host from the sorted row
// lengths; the entries are packed on the device.
struct HostUnits {
  int64_t nnz = 0;
  std::vector<long long> uoff{0};  // unit offsets (n_units + 1)
  std::vector<int> uinfo;          // (first row, R, valid rows, 0) per unit; R = 0: long row
  int n_units() const { return (int)uinfo.size() / 4; }
  void add(int row0, int R, int valid, long long slots) {
    uinfo.insert(uinfo.end(), {row0, R, valid, 0});
    uoff.push_back(uoff.back() + slots);
  }
};

// Units of `nrows` rows numbered from row_base whose lengths slen are sorted
// in decreasing order. Rows with >= long_min entries become 4-aligned,
// 4-padded warp units; the rest slices of 32*R rows, R = 4 for rows of length
// <= 1, 2 for length <= 8, else 1 (capped by max_rpt), padded to the slice's
// first (longest) row, rounded up to even when above 1 (entries in pairs).
void append_unit_table(HostUnits& H, int row_base, int nrows, const int* slen, int long_min, int max_rpt) {
  for (int r = 0; r < nrows; ++r) H.nnz += slen[r];
  int r = 0;
  for (; r < nrows && slen[r] >= long_min; ++r) H.add(row_base + r, 0, 1, ((slen[r] + 3LL) / 4) * 4);
  while (r < nrows) {
    const int L = slen[r];
    int R = L <= 1 ? 4 : (L <= 8 ? 2 : 1);
    R = std::max(1, std::min(R, max_rpt));
    const int Lp = L <= 1 ? L : (L + 1) / 2 * 2;
    H.add(row_base + r, R, std::min(32 * R, nrows - r), 32LL * R * Lp);
    r += 32 * R;
  }
}

// Append empty units (no entries; rows numbered from `empty_row`, which is
// past the last row) until the table has `target` units, so that a batch
// instance fills whole blocks.
void pad_units_to(HostUnits& H, int target, int empty_row) {
  while (H.n_units() < target) H.add(empty_row, 1, 0, 0);
}

pdhg_status upload_units(pdhg_ctx* ctx, const HostUnits& h, int rows, int cols, Hyb& d) {
#ifdef PDHG_CHECKED
  if (!ctx->check) {
    CK(ctx, dalloc(ctx, &ctx->check, 1));
    CK(ctx, cudaMemsetAsync(ctx->check, 0, sizeof(unsigned), ctx->stream));
  }
  d.check = ctx->check;
#endif
  d.rows = rows;
  d.cols = cols;
  d.n_units = h.n_units();
  d.nnz = h.nnz;
  d.slots = h.uoff.back();
  CK(ctx, dalloc(ctx, &d.uoff, h.uoff.size()));
  CK(ctx, dalloc(ctx, &d.uinfo, std::max<size_t>(1, h.uinfo.size() / 4)));
  CK(ctx, dalloc(ctx, &d.ci, std::max<long long>(1, d.slots)));
  CK(ctx, dalloc(ctx, &d.v, std::max<long long>(1, d.slots)));
  cudaStream_t s = ctx->stream;
  CK(ctx, cudaMemcpyAsync(d.uoff, h.uoff.data(), sizeof(long long) * h.uoff.size(), cudaMemcpyHostToDevice, s));
  if (!h.uinfo.empty())
    CK(ctx, cudaMemcpyAsync(d.uinfo, h.uinfo.data(), sizeof(int) * h.uinfo.size(), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemsetAsync(d.ci, 0, sizeof(int) * std::max<long long>(1, d.slots), s));
  CK(ctx, cudaMemsetAsync(d.v, 0, sizeof(double) * std::max<long long>(1, d.slots), s));
  return PDHG_OK;
}

// bits needed to hold the values 0..v
int bit_length(unsigned long long v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

// Panel heights for the panel-tiled primal step. Equal heights (option
// panel_balance = 0): every panel ps.pl.rows rows. Balanced (the default
// without panel_rows): the heights follow the entries of the long columns:
// every panel gets a whole number k of the panel pass's blocks and about k * T
// entries (T = the entries per block of one wave), at most hmax rows (what
// fits in shared memory, or panel_rows rounded down to 16); a panel whose
// first T entries need more rows gets hmax rows and one block. T is the smallest (by bisection) that
// fits in one wave. Rows are sorted by decreasing length, so the first panels
// are short and the last ones tall. With equal heights the blocks' shares
// differ by the rounding of each panel's entries to whole blocks (one block
// carried 1.22 times the mean on the 1e6 x 3e6 Zipf LP). Panel starts are
// multiples of 16 rows (16-byte aligned copies of y into shared memory).
pdhg_status plan_panels(pdhg_ctx* ctx, PanelSet& ps, Scratch& sc, const long long* tp, const int* sval,
                        const int* rowid, const int* iy, long long nlong, long long hmax) {
  const long long m = ctx->m;
  cudaStream_t s = ctx->stream;
  const int total = PANEL_MINB32 * ctx->sms;
  std::vector<int> pf;
  auto uniform = [&](long long H) {
    pf.clear();
    for (long long i = 0; i < m; i += H) pf.push_back((int)i);
    pf.push_back((int)m);
  };
  uniform(ps.pl.rows);
  const pdhg_options& o = ctx->opt;
  const bool balance = o.panel_balance == 1 || (o.panel_balance == -1 && o.panel_rows == 0);
  if (o.panel_rows > 0) hmax = std::min(hmax, (long long)o.panel_rows / 16 * 16);
  if (balance && hmax >= 16 && (long long)pf.size() - 1 <= total) {
    long long Z = 0;
    CK(ctx, cudaMemcpyAsync(&Z, tp + nlong, sizeof(long long), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    int* cnt = nullptr;
    CK(ctx, sc.take(&cnt, m));
    CK(ctx, cudaMemsetAsync(cnt, 0, sizeof(int) * m, s));
    launch_row_counts(Z, sval, rowid, iy, cnt, s);
    std::vector<int> hc(m);
    CK(ctx, cudaMemcpyAsync(hc.data(), cnt, sizeof(int) * m, cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    std::vector<long long> cum(m + 1, 0);
    for (long long i = 0; i < m; ++i) cum[i + 1] = cum[i] + hc[i];
    // the first row e (a multiple of 16, or m) with cum[e] >= target
    auto row_for = [&](double target) -> long long {
      const long long e = std::lower_bound(cum.begin(), cum.end(), (long long)std::ceil(target)) - cum.begin();
      return std::min(m, (e + 15) / 16 * 16);
    };
    // panel starts for entries per block T; returns the blocks they take
    auto greedy = [&](double T, std::vector<int>* out) -> long long {
      long long st = 0, blocks = 0;
      if (out) out->assign(1, 0);
      while (st < m) {
        long long k = 0, e = st;
        for (;;) {
          const long long ek = row_for((double)cum[st] + (double)(k + 1) * T);
          if (ek - st > hmax) break;
          ++k;
          e = ek;
          if (ek >= m) break;
        }
        if (k == 0) {
          k = 1;
          e = std::min(m, st + hmax);
        }
        blocks += k;
        st = e;
        if (out) out->push_back((int)st);
      }
      return blocks;
    };
    double lo = (double)cum[m] / total, hi = lo;
    while (greedy(hi, nullptr) > total && hi < 1e18) hi *= 2;
    if (greedy(hi, nullptr) <= total) {
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (greedy(mid, nullptr) <= total)
          hi = mid;
        else
          lo = mid;
      }
      greedy(hi, &pf);
    }
  }
  int H = 0;
  for (size_t p = 0; p + 1 < pf.size(); ++p) H = std::max(H, pf[p + 1] - pf[p]);
  ps.pl.rows = H;
  ps.pl.panels = (int)pf.size() - 1;
  CK(ctx, dalloc(ctx, &ps.pl.pfirst, pf.size()));
  CK(ctx, cudaMemcpyAsync(ps.pl.pfirst, pf.data(), sizeof(int) * pf.size(), cudaMemcpyHostToDevice, s));
  return PDHG_OK;
}

// Panel layout of Ahat^T for the panel-tiled primal step (one LP): the entries
// of every long row j < nlong of A^T (the rows with at least long_row_min
// entries, which come first in the internal numbering; sorted by internal row
// i) are cut into segments, one per panel (consecutive rows i, see plan_panels);
// short rows stay with the direct step (a one-entry segment would cost a
// partial sum's write and read to save one gather). The segments of each panel,
// sorted by decreasing length, become the rows of the Hyb ps.Pn with row
// indices relative to the panel. Segments are numbered column by column
// (their partial sums' positions, segout), so that column j's partial sums
// are positions [cptr[j], cptr[j+1]) in panel order.
pdhg_status build_panels(pdhg_ctx* ctx, PanelSet& ps, Scratch& sc, const long long* tp, const int* sval,
                         const int* rowid, const int* iy, const double* val, unsigned max_col_len, long long nlong,
                         long long* hist, long long* ws) {
  const pdhg_options& o = ctx->opt;
  const long long N = nlong;
  const int H = ps.pl.rows, P = ps.pl.panels;
  const int* pfirst = ps.pl.pfirst;
  cudaStream_t s = ctx->stream;
  long long Z = 0;  // entries of the long rows: tp[nlong]
  CK(ctx, cudaMemcpyAsync(&Z, tp + N, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  ps.pl.ncols = (int)N;
  int *head = nullptr, *panel = nullptr, *col = nullptr;
  long long* segpos = nullptr;
  CK(ctx, sc.take(&head, Z));
  CK(ctx, sc.take(&panel, Z));
  CK(ctx, sc.take(&col, Z));
  CK(ctx, sc.take(&segpos, Z + 1));
  launch_panel_heads(tp, N, sval, rowid, iy, pfirst, P, head, panel, col, s);
  launch_scan_int(head, Z, segpos, ws, s);
  long long S = 0;
  CK(ctx, cudaMemcpyAsync(&S, segpos + Z, sizeof(long long), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  long long* seg_start = nullptr;
  int *seg_panel = nullptr, *seg_col = nullptr, *seg_len = nullptr, *va = nullptr, *vb = nullptr, *pcount = nullptr;
  int* slen = nullptr;
  unsigned long long *ka = nullptr, *kb = nullptr;
  CK(ctx, sc.take(&seg_start, S + 1));
  CK(ctx, sc.take(&seg_panel, S));
  CK(ctx, sc.take(&seg_col, S));
  CK(ctx, sc.take(&seg_len, S));
  CK(ctx, sc.take(&ka, S));
  CK(ctx, sc.take(&kb, S));
  CK(ctx, sc.take(&va, S));
  CK(ctx, sc.take(&vb, S));
  CK(ctx, sc.take(&pcount, P));
  CK(ctx, sc.take(&slen, S));
  CK(ctx, sc.take(&ps.col, S));
  CK(ctx, sc.take(&ps.base, S));
  launch_panel_segments(head, panel, col, segpos, Z, S, seg_start, seg_panel, seg_col, s);
  CK(ctx, cudaMemsetAsync(pcount, 0, sizeof(int) * P, s));
  const int lbits = bit_length(max_col_len);
  launch_panel_keys(seg_start, seg_panel, S, (int)max_col_len, lbits, seg_len, ka, va, pcount, s);
  const int alt = radix_sort_pairs<unsigned long long>(ka, va, kb, vb, S,
                                                        lbits + bit_length((unsigned long long)(P - 1)), hist, ws, s);
  const int* sp = alt ? vb : va;
  launch_gather_int(seg_len, sp, S, slen, s);
  launch_panel_rowinfo(sp, seg_col, seg_panel, pfirst, S, ps.col, ps.base, s);
  CK(ctx, dalloc(ctx, &ps.pl.segout, S));
  launch_panel_dense_out(ps.col, sp, seg_panel, (int)N, S, ps.pl.segout, s);
  std::vector<int> hs(S), hc(P);
  CK(ctx, cudaMemcpyAsync(hs.data(), slen, sizeof(int) * S, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(hc.data(), pcount, sizeof(int) * P, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  HostUnits uP;
  std::vector<int> ust(P + 1, 0);
  long long base = 0;
  for (int p = 0; p < P; ++p) {
    ust[p] = uP.n_units();
    append_unit_table(uP, (int)base, hc[p], hs.data() + base, o.long_row_min, o.rows_per_thread);
    base += hc[p];
  }
  ust[P] = uP.n_units();
  // one wave of blocks (PANEL_MINB32 per SM), shared among the panels in
  // proportion to their stored entries, at least one each
  std::vector<int> nb(P, 1);
  {
    const int total = std::max(PANEL_MINB32 * ctx->sms, P);
    const double slots = (double)std::max(1LL, uP.uoff.back());
    auto work = [&](int p) { return (double)(uP.uoff[ust[p + 1]] - uP.uoff[ust[p]]); };
    int used = 0;
    for (int p = 0; p < P; ++p) {
      nb[p] = std::max(1, (int)std::floor(work(p) / slots * total));
      used += nb[p];
    }
    // what rounding left goes to the panels with the most entries per block
    while (used < total) {
      int best = 0;
      for (int p = 1; p < P; ++p)
        if (work(p) / nb[p] > work(best) / nb[best]) best = p;
      nb[best] += 1;
      ++used;
    }
  }
  std::vector<int> binfo;
  for (int p = 0; p < P; ++p)
    for (int b = 0; b < nb[p]; ++b) binfo.insert(binfo.end(), {p, b, nb[p], 0});
  ps.pl.blocks = (int)(binfo.size() / 4);
  CK(ctx, dalloc(ctx, &ps.pl.binfo, ps.pl.blocks));
  CK(ctx, cudaMemcpyAsync(ps.pl.binfo, binfo.data(), sizeof(int) * binfo.size(), cudaMemcpyHostToDevice, s));
  pdhg_status rs = upload_units(ctx, uP, (int)S, H, ps.Pn);
  if (rs != PDHG_OK) return rs;
  CK(ctx, dalloc(ctx, &ps.pl.ustart, P + 1));
  CK(ctx, cudaMemcpyAsync(ps.pl.ustart, ust.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice, s));
  launch_fill_units_P(ps.Pn, slen, sp, seg_start, seg_panel, sval, rowid, iy, val, pfirst, s);
  // the panel pass reads the panel-relative row indices (< H <= 56320) in 16
  // bits: 2 bytes less per entry of the long columns
  if (H <= 65536 && ps.Pn.slots > 0) {
    CK(ctx, dalloc(ctx, &ps.Pn.ci16, ps.Pn.slots));
    launch_narrow_index(ps.Pn.ci16, ps.Pn.ci, ps.Pn.slots, vec_grid(ctx, ps.Pn.slots), s);
  }
  // dense panel-major partial sums; the slots of absent segments stay 0
  const long long slots = std::max<long long>(1, (long long)P * N);
  CK(ctx, dalloc(ctx, &ps.partial, slots));
  CK(ctx, cudaMemsetAsync(ps.partial, 0, sizeof(double) * slots, s));
  CK(ctx, cudaGetLastError());
  CK(ctx, cudaStreamSynchronize(s));  // the host tables are released on return
  return PDHG_OK;
}

// Builds ctx->A, ctx->At, ctx->perm_x, ctx->perm_y (and for a batch ctx->binst,
// ctx->bstart, ctx->nblocks) on the device from the instances' CSRs in device
// memory: instance i's m_i + 1 row pointers start at lrp + rpoff_h[i], its
// column indices and values at lci + zoff_h[i], val + zoff_h[i]; its rows and
// columns are ctx->yoff_h[i].. and ctx->xoff_h[i].. of the stacked problem.
// Internal numbering: every instance's rows (and columns) by decreasing
// length, stable, each instance keeping its own range.
pdhg_status build_layouts(pdhg_ctx* ctx, Scratch& sc, const long long* lrp, const int* lci, const double* val,
                          const std::vector<long long>& rpoff_h, const std::vector<long long>& zoff_h) {
  Range nvtx_range("pdhg/layout");
  const pdhg_options& o = ctx->opt;
  const int count = ctx->count;
  const bool batch = count > 1;
  const long long M = ctx->m, N = ctx->n, Z = ctx->nnz;
  cudaStream_t s = ctx->stream;

  long long *d_rpoff = nullptr, *d_zoff = nullptr;
  int *d_xoff = nullptr, *d_yoff = nullptr;
  CK(ctx, sc.take(&d_rpoff, count));
  CK(ctx, sc.take(&d_zoff, count + 1));
  CK(ctx, sc.take(&d_xoff, count + 1));
  CK(ctx, sc.take(&d_yoff, count + 1));
  CK(ctx, cudaMemcpyAsync(d_rpoff, rpoff_h.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_zoff, zoff_h.data(), sizeof(long long) * (count + 1), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_xoff, ctx->xoff_h.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(d_yoff, ctx->yoff_h.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
  int *rinst = nullptr, *cinst = nullptr;
  if (batch) {
    CK(ctx, sc.take(&rinst, M));
    CK(ctx, sc.take(&cinst, N));
    launch_instance_of(d_yoff, count, M, rinst, s);
    launch_instance_of(d_xoff, count, N, cinst, s);
  }

  // stacked CSR, row lengths of A and A^T
  long long* grp = nullptr;
  int *gci = nullptr, *rowid = nullptr, *lenA = nullptr, *lenT = nullptr;
  unsigned* maxes = nullptr;
  CK(ctx, sc.take(&grp, M + 1));
  CK(ctx, sc.take(&gci, Z));
  CK(ctx, sc.take(&rowid, Z));
  CK(ctx, sc.take(&lenA, M));
  CK(ctx, sc.take(&lenT, N));
  CK(ctx, sc.take(&maxes, 2));
  launch_globalize(lrp, lci, d_rpoff, d_zoff, d_xoff, d_yoff, rinst, M, Z, grp, gci, rowid, s);
  launch_lengths(grp, M, gci, Z, N, lenA, lenT, maxes, s);
  unsigned h_max[2] = {0, 0};
  CK(ctx, cudaMemcpyAsync(h_max, maxes, sizeof(h_max), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));

  // renumbering: stable sort by (instance, decreasing length)
  const long long MN = std::max(M, N);
  const long long hist_len = radix_hist_len(std::max(MN, Z));
  unsigned long long *k64a = nullptr, *k64b = nullptr;
  int *va = nullptr, *vb = nullptr;
  long long *hist = nullptr, *ws = nullptr;
  CK(ctx, sc.take(&k64a, MN));
  CK(ctx, sc.take(&k64b, MN));
  CK(ctx, sc.take(&va, MN));
  CK(ctx, sc.take(&vb, MN));
  CK(ctx, sc.take(&hist, hist_len));
  CK(ctx, sc.take(&ws, scan_ws_len(std::max({hist_len, M, N, Z}))));
  CK(ctx, dalloc(ctx, &ctx->perm_y, M));
  CK(ctx, dalloc(ctx, &ctx->perm_x, N));
  const int ibits = batch ? bit_length((unsigned long long)(count - 1)) : 0;
  const int* lens[2] = {lenA, lenT};
  const int* insts[2] = {rinst, cinst};
  const long long cnts[2] = {M, N};
  int* perms[2] = {ctx->perm_y, ctx->perm_x};
  int *iy = nullptr, *ix = nullptr, *slA = nullptr, *slT = nullptr, *sec = nullptr;
  CK(ctx, sc.take(&iy, M));
  CK(ctx, sc.take(&ix, N));
  CK(ctx, sc.take(&slA, M));
  CK(ctx, sc.take(&slT, N));
  // option singleton_order (single LPs): columns with one entry ordered by
  // the internal row of that entry, so that consecutive such columns gather
  // neighbouring entries of y (primal step) and a row's one-entry columns sit
  // side by side in xbar (dual step)
  const int rbits = bit_length((unsigned long long)std::max<long long>(M - 1, 1));
  const bool singles = o.singleton_order && !batch && bit_length(h_max[1]) + rbits <= 62;
  if (singles) CK(ctx, sc.take(&sec, N));
  for (int side = 0; side < 2; ++side) {
    const int lbits = bit_length(h_max[side]);
    const int sbits = side == 1 && singles ? rbits : 0;
    if (sbits) launch_singleton_rows(gci, rowid, Z, lenT, iy, sec, N, s);
    launch_length_keys(lens[side], cnts[side], insts[side], (int)h_max[side], lbits, k64a, va, s,
                       sbits ? sec : nullptr, sbits);
    const int alt = radix_sort_pairs<unsigned long long>(k64a, va, k64b, vb, cnts[side], lbits + ibits + sbits, hist,
                                                         ws, s);
    CK(ctx, cudaMemcpyAsync(perms[side], alt ? vb : va, sizeof(int) * cnts[side], cudaMemcpyDeviceToDevice, s));
    if (side == 0) launch_invert(ctx->perm_y, M, iy, s);  // the rows' numbering, which side 1 may sort by
  }
  launch_invert(ctx->perm_x, N, ix, s);
  launch_gather_int(lenA, ctx->perm_y, M, slA, s);
  launch_gather_int(lenT, ctx->perm_x, N, slT, s);

  // transpose: entries by internal column, by increasing internal row within one
  unsigned *k32a = nullptr, *k32b = nullptr;
  int *za = nullptr, *zb = nullptr;
  long long *tp = nullptr, *rpi = nullptr;
  CK(ctx, sc.take(&k32a, Z));
  CK(ctx, sc.take(&k32b, Z));
  CK(ctx, sc.take(&za, Z));
  CK(ctx, sc.take(&zb, Z));
  CK(ctx, sc.take(&tp, N + 1));
  CK(ctx, sc.take(&rpi, M + 1));
  launch_scan_int(slA, M, rpi, ws, s);
  launch_transpose_keys(grp, ctx->perm_y, rpi, M, gci, ix, k32a, za, s);
  const int alt = radix_sort_pairs<unsigned>(k32a, za, k32b, zb, Z, bit_length((unsigned long long)(N - 1)), hist,
                                             ws, s);
  const int* sval = alt ? zb : za;
  launch_scan_int(slT, N, tp, ws, s);

  // unit tables from the sorted lengths
  std::vector<int> hA(M), hT(N);
  CK(ctx, cudaMemcpyAsync(hA.data(), slA, sizeof(int) * M, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(hT.data(), slT, sizeof(int) * N, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  HostUnits uA, uT;
  std::vector<int> binst;
  ctx->bstart_h.assign(count + 1, 0);
  for (int inst = 0; inst < count; ++inst) {
    const int y0 = ctx->yoff_h[inst], x0 = ctx->xoff_h[inst];
    const int before = uA.n_units();
    append_unit_table(uA, y0, ctx->yoff_h[inst + 1] - y0, hA.data() + y0, o.long_row_min, o.rows_per_thread);
    append_unit_table(uT, x0, ctx->xoff_h[inst + 1] - x0, hT.data() + x0, o.long_row_min, o.rows_per_thread);
    if (batch) {
      // both layouts get the same whole number of blocks for this instance
      const int units = std::max(uA.n_units(), uT.n_units()) - before;
      const int blocks = (units + ctx->wpb - 1) / ctx->wpb;
      pad_units_to(uA, before + blocks * ctx->wpb, (int)M);
      pad_units_to(uT, before + blocks * ctx->wpb, (int)N);
      ctx->bstart_h[inst + 1] = ctx->bstart_h[inst] + blocks;
      for (int b = 0; b < blocks; ++b) binst.push_back(inst);
    }
  }
  pdhg_status rs = upload_units(ctx, uA, (int)M, (int)N, ctx->A);
  if (rs != PDHG_OK) return rs;
  rs = upload_units(ctx, uT, (int)N, (int)M, ctx->At);
  if (rs != PDHG_OK) return rs;
  launch_fill_units_A(ctx->A, slA, grp, ctx->perm_y, gci, ix, val, s);
  launch_fill_units_T(ctx->At, slT, tp, sval, rowid, iy, val, s);
  CK(ctx, cudaGetLastError());
  if (ctx->panels_on) {
    // the longest rows of A^T (a prefix of the internal columns, whole units
    // of the A^T layout: every unit whose shortest row has at least pmin
    // entries) go to the panels; the direct step takes the units after them.
    // pmin: panel_min_len if set; else 32 for a layout of FP32 steps (its
    // partial sums cost half as much) and long_row_min for FP64 steps.
    auto prefix = [&](int pmin, int* ulong_out) -> long long {
      int ulong = 0;
      while (ulong < uT.n_units()) {
        const int* ui = &uT.uinfo[4 * (size_t)ulong];
        const int last = ui[1] == 0 ? ui[0] : ui[0] + ui[2] - 1;  // the unit's shortest valid row
        if ((ui[2] == 0 && ui[1] != 0) || hT[last] < pmin) break;
        ++ulong;
      }
      *ulong_out = ulong;
      return ulong < uT.n_units() ? uT.uinfo[4 * (size_t)ulong] : N;
    };
    const int nsets = ctx->pan32 ? 2 : 1;
    for (int k = 0; k < nsets && ctx->panels_on; ++k) {
      PanelSet& ps = ctx->pan[k];
      const bool fp32_steps = k == 1 || o.precision == PDHG_FP32;
      const int pmin = o.panel_min_len > 0 ? o.panel_min_len : (fp32_steps ? 32 : o.long_row_min);
      const long long nlong = prefix(pmin, &ps.pl.ulong);
      if (nlong > 0) {
        rs = plan_panels(ctx, ps, sc, tp, sval, rowid, iy, nlong, PANEL_SMEM_MAX / (fp32_steps ? 4LL : 8LL));
        if (rs != PDHG_OK) return rs;
      }
      const long long dense = (long long)ps.pl.panels * nlong;  // slots of the panel-major partial sums
      if (nlong == 0 || dense > 64LL * Z + (1LL << 20) || dense >= (1LL << 31) - 1) {
        // nothing to tile, or partial sums far larger than the matrix: the
        // direct step takes every column
        if (k == 0) ctx->panels_on = false;
        ctx->pan32 = false;
      } else {
        rs = build_panels(ctx, ps, sc, tp, sval, rowid, iy, val, h_max[1], nlong, hist, ws);
        if (rs != PDHG_OK) return rs;
      }
    }
  }
  if (batch) {
    ctx->nblocks = ctx->bstart_h[count];
    CK(ctx, dalloc(ctx, &ctx->binst, ctx->nblocks));
    CK(ctx, cudaMemcpyAsync(ctx->binst, binst.data(), sizeof(int) * ctx->nblocks, cudaMemcpyHostToDevice, s));
  }
  // the host tables are released on return: wait for their copies
  CK(ctx, cudaStreamSynchronize(s));
  return PDHG_OK;
}

// host_checks: waits for the host threads' checks of host inputs (see
// pdhg_create) and returns their status; called once the upload is queued,
// before anything reads the uploaded data. With ctx->check_on_device the
// uploaded copies are checked on the device instead.
pdhg_status setup(pdhg_ctx* ctx, const int64_t* row_ptr, const int32_t* col_idx, const double* val, const double* b,
                  const double* c, const double* x0, const double* y0, const std::function<pdhg_status()>& host_checks) {
  Range nvtx_range("pdhg/setup");
  const int64_t m = ctx->m, n = ctx->n, nnz = ctx->nnz;
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  Scratch sc(s);
  ctx->count = 1;
  ctx->xoff_h = {0, (int)n};
  ctx->yoff_h = {0, (int)m};
  // the caller's arrays on the device
  const long long* d_rp = nullptr;
  const int* d_ci = nullptr;
  const double *d_v = nullptr, *d_b = nullptr, *d_c = nullptr, *d_x0 = nullptr, *d_y0 = nullptr;
  if (o.inputs_on_device) {
    d_rp = reinterpret_cast<const long long*>(row_ptr);
    d_ci = col_idx;
    d_v = val;
    d_b = b;
    d_c = c;
    d_x0 = x0;
    d_y0 = y0;
  } else {
    long long* rp_ = nullptr;
    int* ci_ = nullptr;
    double *v_ = nullptr, *b_ = nullptr, *c_ = nullptr;
    CK(ctx, sc.take(&rp_, m + 1));
    CK(ctx, sc.take(&ci_, nnz));
    CK(ctx, sc.take(&v_, nnz));
    CK(ctx, sc.take(&b_, m));
    CK(ctx, sc.take(&c_, n));
    CK(ctx, cudaMemcpyAsync(rp_, row_ptr, sizeof(long long) * (m + 1), cudaMemcpyHostToDevice, s));
    if (nnz) {
      CK(ctx, cudaMemcpyAsync(ci_, col_idx, sizeof(int) * nnz, cudaMemcpyHostToDevice, s));
      CK(ctx, cudaMemcpyAsync(v_, val, sizeof(double) * nnz, cudaMemcpyHostToDevice, s));
    }
    CK(ctx, cudaMemcpyAsync(b_, b, sizeof(double) * m, cudaMemcpyHostToDevice, s));
    CK(ctx, cudaMemcpyAsync(c_, c, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    if (x0) {
      double* x0_ = nullptr;
      CK(ctx, sc.take(&x0_, n));
      CK(ctx, cudaMemcpyAsync(x0_, x0, sizeof(double) * n, cudaMemcpyHostToDevice, s));
      d_x0 = x0_;
    }
    if (y0) {
      double* y0_ = nullptr;
      CK(ctx, sc.take(&y0_, m));
      CK(ctx, cudaMemcpyAsync(y0_, y0, sizeof(double) * m, cudaMemcpyHostToDevice, s));
      d_y0 = y0_;
    }
    d_rp = rp_;
    d_ci = ci_;
    d_v = v_;
    d_b = b_;
    d_c = c_;
    if (!ctx->check_on_device) {
      const pdhg_status checked = host_checks();
      if (checked != PDHG_OK) return checked;  // the caller reports the checks' message
    }
  }
  if (o.inputs_on_device || ctx->check_on_device) {
    // the checks pdhg_create makes on host inputs without a GPU, on the
    // device: the CSR structure and finite data, before anything reads them
    int* flags = nullptr;
    CK(ctx, sc.take(&flags, 1));
    CK(ctx, cudaMemsetAsync(flags, 0, sizeof(int), s));
    launch_validate_csr(m, n, nnz, d_rp, d_ci, d_v, flags, s);
    launch_check_finite(d_b, m, flags, s);
    launch_check_finite(d_c, n, flags, s);
    if (d_x0) launch_check_finite(d_x0, n, flags, s);
    if (d_y0) launch_check_finite(d_y0, m, flags, s);
    int hf = 0;
    CK(ctx, cudaGetLastError());
    CK(ctx, cudaMemcpyAsync(&hf, flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    if (hf & LAYOUT_BAD_ROW_PTR)
      return fail(ctx, PDHG_ERR_INVALID, "row_ptr[0] != 0, row_ptr[m] != nnz or row_ptr not non-decreasing");
    if (hf & LAYOUT_BAD_COLUMN) return fail(ctx, PDHG_ERR_INVALID, "column index out of range");
    if (hf & LAYOUT_UNSORTED)
      return fail(ctx, PDHG_ERR_INVALID, "column indices not strictly increasing within a row");
    if (hf & LAYOUT_NOT_FINITE) return fail(ctx, PDHG_ERR_NUMERIC, "NaN or Inf in the input data");
  }
  pdhg_status rs = build_layouts(ctx, sc, d_rp, d_ci, d_v, {0}, {0, (long long)nnz});
  if (rs != PDHG_OK) return rs;
  ctx->persist_smem = persistent_smem_bytes(n, m);
  if (ctx->panels_on) CK(ctx, configure_primal_panels());
  Hyb& A = ctx->A;
  Hyb& At = ctx->At;
  double** vecs_n[] = {&ctx->c, &ctx->ch, &ctx->dc, &ctx->idc, &ctx->x, &ctx->xbar, &ctx->xsum, &ctx->xavg,
                       &ctx->xr, &ctx->tmp_n, &ctx->tmp_n2};
  double** vecs_m[] = {&ctx->b, &ctx->bh, &ctx->dr, &ctx->idr, &ctx->y, &ctx->ysum, &ctx->yavg, &ctx->yr,
                       &ctx->tmp_m};
  for (double** p : vecs_n) CK(ctx, dalloc(ctx, p, n));
  for (double** p : vecs_m) CK(ctx, dalloc(ctx, p, m));
  ctx->nb_eval = std::max(1, std::min(ctx->sms * 16, std::max(unit_grid(ctx, A), unit_grid(ctx, At))));
  prefer_l1_for_step_kernels();
  CK(ctx, dalloc(ctx, &ctx->partials, (size_t)std::max(ctx->nb_eval, ctx->sms * 8) * NQ));
  CK(ctx, dalloc(ctx, &ctx->scal, 16));
  CK(ctx, dalloc(ctx, &ctx->st, 1));
  CK(ctx, dalloc(ctx, &ctx->kkt_sums, 1));
  CK(ctx, dalloc(ctx, &ctx->trace, TRACE_CAP));
  CK(ctx, dalloc(ctx, &ctx->sol, 2 * n + m));
  CK(ctx, cudaMallocHost(&ctx->h_st, sizeof(DevState)));
  CK(ctx, cudaMallocHost(&ctx->h_kkt, sizeof(EvalSums)));
  for (int i = 0; i < 3 * EV_POOL; ++i) CK(ctx, cudaEventCreate(&ctx->ev[i]));

  launch_gather_double(d_b, ctx->perm_y, m, ctx->b, s);
  launch_gather_double(d_c, ctx->perm_x, n, ctx->c, s);

  // ---- device: FP32 copies of the unscaled values (option values32) ----
  if (o.values32 != 0 && o.precision != PDHG_FP32 && !o.persistent && !o.record_for_backward &&
      (o.values32 == 1 || o.precision == PDHG_MIXED)) {
    int* flag = nullptr;
    CK(ctx, sc.take(&flag, 1));
    CK(ctx, cudaMemsetAsync(flag, 0, sizeof(int), s));
    launch_fp32_inexact(A.v, A.slots, flag, s);
    int inexact = 0;
    CK(ctx, cudaMemcpyAsync(&inexact, flag, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    if (inexact && o.values32 == 1)
      return fail(ctx, PDHG_ERR_INVALID, "values32 = 1: a value of A is not an FP32 number");
    ctx->vals_u = !inexact;
  }
  if (ctx->vals_u) {
    Hyb* hs[] = {&A, &At, ctx->panels_on ? &ctx->pan[0].Pn : nullptr};
    for (Hyb* h : hs) {
      if (!h) continue;
      CK(ctx, dalloc(ctx, &h->u32, h->slots));
      launch_narrow(h->u32, h->v, h->slots, vec_grid(ctx, h->slots), s);
    }
    CK(ctx, dalloc(ctx, &ctx->yg, m));
  }
#ifndef PDHG_CHECKED
  // ---- option stream_steps: launch shapes of the streamed step kernels ----
  if (o.stream_steps) {
    // (T, V) per configuration, and whether this context runs it
    const size_t tv[3][2] = {{8, 8}, {4, 4}, {8, 4}};
    const bool used[3] = {o.precision != PDHG_FP32 && !ctx->vals_u, o.precision != PDHG_FP64, ctx->vals_u};
    for (int i = 0; i < 3; ++i) {
      if (!used[i]) continue;
      StreamCfg& c = ctx->scfg[i];
      c.depth = o.stream_depth;
      const size_t per_warp = (size_t)c.depth * (stream_slot_bytes(tv[i][0], tv[i][1]) + 8);
      c.warps = o.stream_warps ? o.stream_warps : (int)std::min<size_t>(16, (size_t)STREAM_SMEM_MAX / per_warp);
      if (c.warps < 1 || stream_smem(c, tv[i][0], tv[i][1]) > (size_t)STREAM_SMEM_MAX)
        return fail(ctx, PDHG_ERR_INVALID, "stream_steps: stream_warps x stream_depth slots exceed 227 KB of "
                                           "shared memory");
      cudaError_t e = cudaSuccess;
      if (i == 0)
        e = configure_stream<double, double>(c, ctx->sms);
      else if (i == 1)
        e = configure_stream<float, float>(c, ctx->sms);
      else
        e = configure_stream<double, float>(c, ctx->sms);
      CK(ctx, e);
    }
    ctx->stream_on = true;
  }
#endif

  // ---- device: scaling ----
  const int gn = vec_grid(ctx, n), gm = vec_grid(ctx, m);
  const int grA = stride_grid(ctx, A), grT = stride_grid(ctx, At);
  launch_fill(ctx->dr, 1.0, m, gm, s);
  launch_fill(ctx->dc, 1.0, n, gn, s);
  double* r = ctx->tmp_m;   // row factors
  double* sf = ctx->tmp_n;  // column factors
  for (int it = 0; it < o.ruiz_iters; ++it) {
    launch_row_absmax(A, r, grA, s);
    launch_row_absmax(At, sf, grT, s);
    launch_inv_sqrt_or_one(r, r, (int)m, gm, s);
    launch_inv_sqrt_or_one(sf, sf, (int)n, gn, s);
    launch_scale(A, r, sf, 0, grA, s);
    launch_scale(At, r, sf, 1, grT, s);
    for (int k = 0; ctx->panels_on && k < (ctx->pan32 ? 2 : 1); ++k)
      launch_scale(ctx->pan[k].Pn, r, sf, 2, stride_grid(ctx, ctx->pan[k].Pn), s, ctx->pan[k].col, ctx->pan[k].base);
    launch_mul_inplace(ctx->dr, r, (int)m, gm, s);
    launch_mul_inplace(ctx->dc, sf, (int)n, gn, s);
  }
  if (o.pock_chambolle) {
    launch_row_abspow_sum(A, o.pc_alpha, r, grA, s);
    launch_row_abspow_sum(At, 2.0 - o.pc_alpha, sf, grT, s);
    launch_inv_sqrt_or_one(r, r, (int)m, gm, s);
    launch_inv_sqrt_or_one(sf, sf, (int)n, gn, s);
    launch_scale(A, r, sf, 0, grA, s);
    launch_scale(At, r, sf, 1, grT, s);
    for (int k = 0; ctx->panels_on && k < (ctx->pan32 ? 2 : 1); ++k)
      launch_scale(ctx->pan[k].Pn, r, sf, 2, stride_grid(ctx, ctx->pan[k].Pn), s, ctx->pan[k].col, ctx->pan[k].base);
    launch_mul_inplace(ctx->dr, r, (int)m, gm, s);
    launch_mul_inplace(ctx->dc, sf, (int)n, gn, s);
  }
  launch_mul(ctx->bh, ctx->dr, ctx->b, (int)m, gm, s);
  launch_mul(ctx->ch, ctx->dc, ctx->c, (int)n, gn, s);
  launch_reciprocal(ctx->idr, ctx->dr, (int)m, gm, s);
  launch_reciprocal(ctx->idc, ctx->dc, (int)n, gn, s);
  CK(ctx, cudaGetLastError());

  // ---- device: power iteration for ||Ahat||_2 from a fixed pseudo-random vector ----
  double* v = ctx->tmp_n;
  double* w = ctx->tmp_n2;
  double* u = ctx->tmp_m;
  const int nbs = std::min(ctx->sms * 4, std::max(gn, gm));
  launch_fill(ctx->scal, 0.0, 16, 1, s);
  launch_power_start(w, ctx->perm_x, nullptr, 1, (int)n, gn, s);
  launch_sumsq(w, (int)n, ctx->partials, nbs, ctx->scal + 6, s);
  launch_div_by_norm(v, w, ctx->scal + 6, (int)n, gn, s);
  // the estimate is ||Ahat v|| of the last iteration (a zero ||w|| leaves v,
  // so the later iterations repeat it), so only that one's norm is taken
  for (int it = 0; it < o.power_iters; ++it) {
    launch_spmv(A, v, u, grA, s);
    if (it == o.power_iters - 1) launch_sumsq(u, (int)m, ctx->partials, nbs, ctx->scal + 0, s);
    launch_spmv(At, u, w, grT, s);
    launch_sumsq(w, (int)n, ctx->partials, nbs, ctx->scal + 5, s);
    launch_div_by_norm(v, w, ctx->scal + 5, (int)n, gn, s);
  }
  launch_sumsq(ctx->ch, (int)n, ctx->partials, nbs, ctx->scal + 1, s);
  launch_sumsq(ctx->bh, (int)m, ctx->partials, nbs, ctx->scal + 2, s);
  launch_sumsq(ctx->b, (int)m, ctx->partials, nbs, ctx->scal + 3, s);
  launch_sumsq(ctx->c, (int)n, ctx->partials, nbs, ctx->scal + 4, s);
  CK(ctx, cudaGetLastError());

  // ---- device state ----
  DevState h{};
  h.tol = 0.0;
  h.eps_target = o.eps_cross;
  h.eps_factor = o.eps_factor;
  h.beta_suff = o.beta_suff;
  h.beta_nec = o.beta_nec;
  h.beta_art = o.beta_art;
  h.theta = o.theta;
  h.snapshot_every = o.snapshot_every;
  h.next_snapshot = o.snapshot_every;
  h.restarts_on = o.restarts;
  h.primal_weight_on = o.primal_weight;
  h.halpern = o.halpern;
  h.rho = o.halpern_reflect;
  h.gap_tol = o.gap_tol;
  h.restart_scheme = o.restart_scheme;
  h.pid_kp = o.pid_kp;
  h.pid_ki = o.pid_ki;
  h.pid_kd = o.pid_kd;
  *ctx->h_st = h;
  CK(ctx, cudaMemcpyAsync(ctx->st, ctx->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  launch_finish_setup(ctx->st, ctx->scal, o.step_factor, o.primal_weight, s);

  // ---- starting point (scaled: xhat = x0 / D_c, yhat = y0 / D_r) ----
  launch_fill(ctx->x, 0.0, n, gn, s);
  launch_fill(ctx->y, 0.0, m, gm, s);
  if (d_x0) {
    launch_gather_double(d_x0, ctx->perm_x, n, ctx->tmp_n, s);
    launch_div(ctx->x, ctx->tmp_n, ctx->dc, (int)n, gn, s);
  }
  if (d_y0) {
    launch_gather_double(d_y0, ctx->perm_y, m, ctx->tmp_m, s);
    launch_div(ctx->y, ctx->tmp_m, ctx->dr, (int)m, gm, s);
  }
  launch_fill(ctx->xsum, 0.0, n, gn, s);
  launch_fill(ctx->ysum, 0.0, m, gm, s);
  CK(ctx, cudaMemcpyAsync(ctx->xr, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->yr, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->xavg, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->yavg, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  // FP32 iteration state: rounded copies of the scaled matrix and vectors
  if (o.precision != PDHG_FP64) {
    CK(ctx, dalloc(ctx, &A.v32, A.slots));
    CK(ctx, dalloc(ctx, &At.v32, At.slots));
    float** f_n[] = {&ctx->x32, &ctx->xbar32, &ctx->xsum32, &ctx->ch32};
    float** f_m[] = {&ctx->y32, &ctx->ysum32, &ctx->bh32};
    for (float** p : f_n) CK(ctx, dalloc(ctx, p, n));
    for (float** p : f_m) CK(ctx, dalloc(ctx, p, m));
    launch_narrow(A.v32, A.v, A.slots, vec_grid(ctx, A.slots), s);
    launch_narrow(At.v32, At.v, At.slots, vec_grid(ctx, At.slots), s);
    if (ctx->panels_on) {
      // the FP32 steps' panel layout: pan[1] when it exists, else pan[0]
      PanelSet& ps = ctx->pan[ctx->pan32 ? 1 : 0];
      CK(ctx, dalloc(ctx, &ps.Pn.v32, ps.Pn.slots));
      const long long slots = std::max<long long>(1, (long long)ps.pl.panels * ps.pl.ncols);
      CK(ctx, dalloc(ctx, &ps.partial32, slots));
      CK(ctx, cudaMemsetAsync(ps.partial32, 0, sizeof(float) * slots, s));
      launch_narrow(ps.Pn.v32, ps.Pn.v, ps.Pn.slots, vec_grid(ctx, ps.Pn.slots), s);
    }
    if (o.refine32 == 1 || (o.refine32 == -1 && o.precision == PDHG_MIXED && !o.record_for_backward &&
                            !o.persistent)) {
      // option refine32: the FP32 iteration runs on corrections to the FP64
      // restart point (xr, yr) = the starting point, copied above: the
      // corrections and sums start at zero, and the FP32 costs are the
      // residuals chat - Ahat^T yr and bhat - Ahat xr at the reference
      ctx->refine = true;
      CK(ctx, dalloc(ctx, &ctx->lo32, n));
      CK(ctx, cudaMemsetAsync(ctx->x32, 0, sizeof(float) * n, s));
      CK(ctx, cudaMemsetAsync(ctx->y32, 0, sizeof(float) * m, s));
      CK(ctx, cudaMemsetAsync(ctx->xsum32, 0, sizeof(float) * n, s));
      CK(ctx, cudaMemsetAsync(ctx->ysum32, 0, sizeof(float) * m, s));
      launch_recenter(A, At, ctx->xr, ctx->yr, ctx->bh, ctx->ch, ctx->bh32, ctx->ch32, ctx->lo32, ctx->st, 1, grA, grT,
                      s);
      ctx->phase32 = true;
    }
  }
  if (o.precision != PDHG_FP64 && !ctx->refine) {
    launch_narrow(ctx->ch32, ctx->ch, n, gn, s);
    launch_narrow(ctx->bh32, ctx->bh, m, gm, s);
    launch_narrow(ctx->x32, ctx->x, n, gn, s);
    launch_narrow(ctx->y32, ctx->y, m, gm, s);
    if (o.halpern) {  // the FP32 sums hold the Halpern anchor: the starting point
      CK(ctx, cudaMemcpyAsync(ctx->xsum32, ctx->x32, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
      CK(ctx, cudaMemcpyAsync(ctx->ysum32, ctx->y32, sizeof(float) * m, cudaMemcpyDeviceToDevice, s));
    } else {
      CK(ctx, cudaMemsetAsync(ctx->xsum32, 0, sizeof(float) * n, s));
      CK(ctx, cudaMemsetAsync(ctx->ysum32, 0, sizeof(float) * m, s));
    }
    // the FP64 evaluation point is the FP32 iterate, exactly
    launch_widen(ctx->x, ctx->x32, n, gn, s);
    launch_widen(ctx->y, ctx->y32, m, gm, s);
    CK(ctx, cudaMemcpyAsync(ctx->xr, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    CK(ctx, cudaMemcpyAsync(ctx->yr, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
    ctx->phase32 = true;
  }
  // restart reference = the starting point (with its fixed-point residual
  // under restart_scheme = 1)
  if (o.restart_scheme == 1)
    eval_point_fp(ctx, &ctx->st->cur);
  else
    eval_point(ctx, ctx->x, ctx->y, nullptr, nullptr, &ctx->st->cur);
  launch_init_restart_ref(ctx->st, s);
  CK(ctx, cudaGetLastError());
  rs = read_state(ctx);
  if (rs != PDHG_OK) return rs;
  for (PanelSet& ps : ctx->pan) ps.col = ps.base = nullptr;  // setup scratch, released on return
  if (!std::isfinite(ctx->h_st->norm_est) || !std::isfinite(ctx->h_st->omega))
    return fail(ctx, PDHG_ERR_NUMERIC, "non-finite norm estimate or primal weight after scaling");
  return PDHG_OK;
}

// ---- one evaluation block -------------------------------------------------------

// The panel-tiled primal half-step of precision T: the panel pass over the
// long columns, then one launch that adds their partial sums and applies the
// update (plain, or the reflected Halpern one of step halpern_it with xsum as
// the anchor) beside the direct step over the short columns.
// With V = float and T = double: the unscaled values, y = D_r y and dc = D_c
// (option values32).
template <class T, class V = T>
pdhg_status panel_half_step(pdhg_ctx* ctx, const PanelSet& ps, const V* vals, const V* valsT, const T* y, const T* ch,
                            T* x, T* xbar, T* xsum, T* partial, int accumulate, int tpb, int halpern_it,
                            const T* dc = nullptr, const T* lo = nullptr) {
  cudaStream_t s = ctx->stream;
  launch_panel_pass<T, V>(ps.Pn, vals, ps.pl, y, partial, s);
  launch_primal_short_combine<T, V>(ctx->At, valsT, y, ch, x, xbar, xsum, ctx->st, accumulate, short_grid(ctx, ps),
                                    ps.pl, partial, tpb, s, halpern_it, dc, lo,
                                    ctx->opt.panel_overlap >= 0 ? ctx->opt.panel_overlap : (sizeof(T) == 4 ? 1 : 0),
                                    ctx->sms * STEP_BLOCKS_PER_SM * TPB / tpb);
  CK(ctx, cudaGetLastError());
  ctx->launches += 1;  // two launches; the caller counts one primal step
  return PDHG_OK;
}

// The primal half-step on (y, x, xbar, xsum) in FP32 or FP64: when the panel
// layout exists, the panel pass over the long columns and the combine fused
// with the direct step over the short ones (two kernels); else the direct
// step over every column.
pdhg_status primal_step(pdhg_ctx* ctx, bool f32, const void* y, void* x, void* xbar, void* xsum, int accumulate,
                        int grT, int tpb) {
  cudaStream_t s = ctx->stream;
  if (!f32 && ctx->vals_u) {  // FP64 on the unscaled FP32 values: y is D_r y here
    if (ctx->panels_on)
      return panel_half_step<double, float>(ctx, ctx->pan[0], ctx->pan[0].Pn.u32, ctx->At.u32, (const double*)y,
                                            ctx->ch, (double*)x, (double*)xbar, (double*)xsum, ctx->pan[0].partial,
                                            accumulate, tpb, -1, ctx->dc);
    launch_primal_step_u(ctx->At, (const double*)y, ctx->ch, (double*)x, (double*)xbar, (double*)xsum, ctx->st,
                         accumulate, grT, s, tpb, 0, ctx->dc);
    return PDHG_OK;
  }
  if (ctx->panels_on) {
    if (f32) {
      const PanelSet& ps = ctx->pan[ctx->pan32 ? 1 : 0];
      return panel_half_step<float>(ctx, ps, ps.Pn.v32, ctx->At.v32, (const float*)y, ctx->ch32, (float*)x,
                                    (float*)xbar, (float*)xsum, ps.partial32, accumulate, tpb, -1, nullptr,
                                    ctx->lo32);
    }
    return panel_half_step<double>(ctx, ctx->pan[0], ctx->pan[0].Pn.v, ctx->At.v, (const double*)y, ctx->ch,
                                   (double*)x, (double*)xbar, (double*)xsum, ctx->pan[0].partial, accumulate, tpb, -1);
  } else if (f32) {
    launch_primal_step32(ctx->At, (const float*)y, ctx->ch32, (float*)x, (float*)xbar, (float*)xsum, ctx->st,
                         accumulate, grT, s, tpb, 0, ctx->lo32);
  } else {
    launch_primal_step(ctx->At, (const double*)y, ctx->ch, (double*)x, (double*)xbar, (double*)xsum, ctx->st,
                       accumulate, grT, s, nullptr, tpb);
  }
  return PDHG_OK;
}

// The primal half-step of iteration `it` of the block as streamed kernels
// (option stream_steps), in the phase's precision and form: with the panel
// layout, the panel pass over the long columns, then one streamed launch that
// combines their partial sums and steps the short columns; else one streamed
// launch over every column.
void stream_primal(pdhg_ctx* ctx, int it, const double* yg64) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int hit = o.halpern ? it : -1, acc = o.halpern ? 0 : o.restarts;
  if (ctx->phase32) {
    const PanelSet* ps = ctx->panels_on ? &ctx->pan[ctx->pan32 ? 1 : 0] : nullptr;
    if (ps) launch_panel_pass<float, float>(ps->Pn, ps->Pn.v32, ps->pl, ctx->y32, ps->partial32, s);
    launch_stream_primal<float, float>(ctx->At, ctx->At.v32, ctx->y32, ctx->ch32, ctx->x32, ctx->xbar32,
                                       ctx->xsum32, ctx->st, acc, hit, ps ? ps->pl.ulong : 0, ps ? ps->pl.ncols : 0,
                                       ps ? ps->pl.panels : 0, ps ? ps->partial32 : nullptr, nullptr, ctx->scfg[1], s,
                                       ctx->lo32);
  } else {
    const bool vu = ctx->vals_u;
    const PanelSet* ps = ctx->panels_on ? &ctx->pan[0] : nullptr;
    double* sum = o.halpern ? ctx->xr : ctx->xsum;
    if (vu) {
      if (ps) launch_panel_pass<double, float>(ps->Pn, ps->Pn.u32, ps->pl, yg64, ps->partial, s);
      launch_stream_primal<double, float>(ctx->At, ctx->At.u32, yg64, ctx->ch, ctx->x, ctx->xbar, sum, ctx->st, acc,
                                          hit, ps ? ps->pl.ulong : 0, ps ? ps->pl.ncols : 0, ps ? ps->pl.panels : 0,
                                          ps ? ps->partial : nullptr, ctx->dc, ctx->scfg[2], s);
    } else {
      if (ps) launch_panel_pass<double, double>(ps->Pn, ps->Pn.v, ps->pl, ctx->y, ps->partial, s);
      launch_stream_primal<double, double>(ctx->At, ctx->At.v, ctx->y, ctx->ch, ctx->x, ctx->xbar, sum, ctx->st,
                                           acc, hit, ps ? ps->pl.ulong : 0, ps ? ps->pl.ncols : 0,
                                           ps ? ps->pl.panels : 0, ps ? ps->partial : nullptr, nullptr, ctx->scfg[0],
                                           s);
    }
  }
  if (ctx->panels_on) ctx->launches += 1;  // two launches; the caller counts one
}

// The dual half-step of iteration `it` of the block as one streamed launch.
void stream_dual(pdhg_ctx* ctx, int it) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int hit = o.halpern ? it : -1, acc = o.halpern ? 0 : o.restarts;
  if (ctx->phase32)
    launch_stream_dual<float, float>(ctx->A, ctx->A.v32, ctx->xbar32, ctx->bh32, ctx->y32, ctx->ysum32, ctx->st, acc,
                                     hit, nullptr, nullptr, ctx->scfg[1], s);
  else if (ctx->vals_u)
    launch_stream_dual<double, float>(ctx->A, ctx->A.u32, ctx->xbar, ctx->bh, ctx->y, o.halpern ? ctx->yr : ctx->ysum,
                                      ctx->st, acc, hit, ctx->dr, ctx->yg, ctx->scfg[2], s);
  else
    launch_stream_dual<double, double>(ctx->A, ctx->A.v, ctx->xbar, ctx->bh, ctx->y,
                                       o.halpern ? ctx->yr : ctx->ysum, ctx->st, acc, hit, nullptr, nullptr,
                                       ctx->scfg[0], s);
}

// The step launches of nb iterations (plus adjoint checkpoints and kernel
// timing events when asked) and the counter update.
pdhg_status enqueue_steps(pdhg_ctx* ctx, int64_t nb, bool timing) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int grT = unit_grid(ctx, ctx->At), grA = unit_grid(ctx, ctx->A), tpb = 32 * ctx->wpb;
  // entries of xbar the dual step stages in shared memory, per precision (none
  // in FP64 phases on the unscaled values)
  const bool vu = ctx->vals_u && !ctx->phase32;
  const int hot = vu ? 0
                     : (int)std::min<int64_t>({(int64_t)o.dual_hot_cols, ctx->n,
                                               (int64_t)(HOT_SMEM_MAX / (ctx->phase32 ? 4 : 8))});
  // the primal step's gather vector D_r y from y (which evaluations, restarts
  // and phase changes set between blocks)
  if (vu) {
    launch_mul(ctx->yg, ctx->dr, ctx->y, (int)ctx->m, vec_grid(ctx, ctx->m), s);
    ctx->launches += 1;
  }
  double* const yg64 = vu ? ctx->yg : ctx->y;  // what the FP64 primal steps gather
  for (int64_t it = 0; it < nb; ++it) {
    if (o.record_for_backward) {
      pdhg_status rs = record_checkpoint(ctx, ctx->k + it);
      if (rs != PDHG_OK) return rs;
    }
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it], s));
    if (ctx->stream_on) {
      stream_primal(ctx, (int)it, yg64);
      if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 1], s));
      stream_dual(ctx, (int)it);
      if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 2], s));
      continue;
    }
    if (o.halpern && vu) {
      if (ctx->panels_on) {
        pdhg_status rs = panel_half_step<double, float>(ctx, ctx->pan[0], ctx->pan[0].Pn.u32, ctx->At.u32, yg64,
                                                        ctx->ch, ctx->x, ctx->xbar, ctx->xr, ctx->pan[0].partial, 0,
                                                        tpb, (int)it, ctx->dc);
        if (rs != PDHG_OK) return rs;
      } else {
        launch_primal_step_halpern<double, float>(ctx->At, ctx->At.u32, yg64, ctx->ch, ctx->x, ctx->xbar, ctx->xr,
                                                  ctx->st, (int)it, grT, s, tpb, nullptr, 0, ctx->dc);
      }
    } else if (o.halpern && !ctx->phase32) {
      if (ctx->panels_on) {  // the anchor (last restart point) in place of the sums
        pdhg_status rs = panel_half_step<double>(ctx, ctx->pan[0], ctx->pan[0].Pn.v, ctx->At.v, ctx->y, ctx->ch,
                                                 ctx->x, ctx->xbar, ctx->xr, ctx->pan[0].partial, 0, tpb, (int)it);
        if (rs != PDHG_OK) return rs;
      } else {
        launch_primal_step_halpern<double>(ctx->At, ctx->At.v, ctx->y, ctx->ch, ctx->x, ctx->xbar, ctx->xr, ctx->st,
                                           (int)it, grT, s, tpb);
      }
    } else if (o.halpern) {
      // FP32 Halpern: the FP32 sums hold the FP32 anchor (no averages in this form)
      if (ctx->panels_on) {
        const PanelSet& ps = ctx->pan[ctx->pan32 ? 1 : 0];
        pdhg_status rs = panel_half_step<float>(ctx, ps, ps.Pn.v32, ctx->At.v32, ctx->y32, ctx->ch32, ctx->x32,
                                                ctx->xbar32, ctx->xsum32, ps.partial32, 0, tpb, (int)it, nullptr,
                                                ctx->lo32);
        if (rs != PDHG_OK) return rs;
      } else {
        launch_primal_step_halpern<float>(ctx->At, ctx->At.v32, ctx->y32, ctx->ch32, ctx->x32, ctx->xbar32,
                                          ctx->xsum32, ctx->st, (int)it, grT, s, tpb, nullptr, 0, nullptr,
                                          ctx->lo32);
      }
    } else {
      pdhg_status rs = ctx->phase32 ? primal_step(ctx, true, ctx->y32, ctx->x32, ctx->xbar32, ctx->xsum32,
                                                  o.restarts, grT, tpb)
                                    : primal_step(ctx, false, yg64, ctx->x, ctx->xbar, ctx->xsum, o.restarts, grT,
                                                  tpb);
      if (rs != PDHG_OK) return rs;
    }
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 1], s));
    if (vu) {
      if (o.halpern)
        launch_dual_step_halpern<double, float>(ctx->A, ctx->A.u32, ctx->xbar, ctx->bh, ctx->y, ctx->yr, ctx->st,
                                                (int)it, grA, s, tpb, nullptr, ctx->dr, ctx->yg);
      else
        launch_dual_step_u(ctx->A, ctx->xbar, ctx->bh, ctx->y, ctx->ysum, ctx->st, o.restarts, grA, s, tpb, ctx->dr,
                           ctx->yg);
    } else if (o.halpern && !ctx->phase32) {
      if (hot > 0)
        launch_dual_step_hot<double>(ctx->A, ctx->A.v, ctx->xbar, hot, ctx->bh, ctx->y, ctx->yr, ctx->st, 0,
                                     ctx->sms, s, (int)it);
      else
        launch_dual_step_halpern<double>(ctx->A, ctx->A.v, ctx->xbar, ctx->bh, ctx->y, ctx->yr, ctx->st, (int)it,
                                         grA, s, tpb);
    } else if (o.halpern) {
      if (hot > 0)
        launch_dual_step_hot<float>(ctx->A, ctx->A.v32, ctx->xbar32, hot, ctx->bh32, ctx->y32, ctx->ysum32, ctx->st,
                                    0, ctx->sms, s, (int)it);
      else
        launch_dual_step_halpern<float>(ctx->A, ctx->A.v32, ctx->xbar32, ctx->bh32, ctx->y32, ctx->ysum32, ctx->st,
                                        (int)it, grA, s, tpb);
    } else if (ctx->phase32) {
      if (hot > 0)
        launch_dual_step_hot<float>(ctx->A, ctx->A.v32, ctx->xbar32, hot, ctx->bh32, ctx->y32, ctx->ysum32, ctx->st,
                                    o.restarts, ctx->sms, s);
      else
        launch_dual_step32(ctx->A, ctx->xbar32, ctx->bh32, ctx->y32, ctx->ysum32, ctx->st, o.restarts, grA, s, tpb);
    } else if (hot > 0) {
      launch_dual_step_hot<double>(ctx->A, ctx->A.v, ctx->xbar, hot, ctx->bh, ctx->y, ctx->ysum, ctx->st, o.restarts,
                                   ctx->sms, s);
    } else {
      launch_dual_step(ctx->A, ctx->xbar, ctx->bh, ctx->y, ctx->ysum, ctx->st, o.restarts, grA, s, nullptr, tpb);
    }
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 2], s));
  }
  launch_add_counters(ctx->st, nb, s);
  ctx->launches += 2 * nb + 1;
  CK(ctx, cudaGetLastError());
  return PDHG_OK;
}

// One evaluation: candidate measures, decisions, their application, and the
// copy of the state struct to pinned host memory (the host waits for it).
pdhg_status enqueue_eval(pdhg_ctx* ctx) {
  Range nvtx_range("pdhg/evaluation");
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int n = (int)ctx->n, m = (int)ctx->m;
  const int gv = vec_grid(ctx, std::max(n, m));
  const bool p32 = ctx->phase32;
  if (p32) {
    widen_current(ctx);
    ctx->launches += 2;
  }
  if (o.restarts && !o.halpern) {  // Halpern: no averages
    if (p32)
      average32(ctx);
    else
      launch_make_average(ctx->xsum, ctx->ysum, ctx->x, ctx->y, ctx->xavg, ctx->yavg, n, m, ctx->st, gv, s);
    eval_point(ctx, ctx->xavg, ctx->yavg, ctx->xr, ctx->yr, &ctx->st->avg);
  }
  if (o.restart_scheme == 1)
    eval_point_fp(ctx, &ctx->st->cur);
  else
    eval_point(ctx, ctx->x, ctx->y, ctx->xr, ctx->yr, &ctx->st->cur);
  launch_decide(ctx->st, ctx->trace, s);
  if (p32 && ctx->refine) {
    // a restart moves the FP64 reference and re-centres the FP32 iteration
    launch_apply32_delta(ctx->st, ctx->x32, ctx->y32, ctx->x, ctx->y, ctx->xavg, ctx->yavg, ctx->xr, ctx->yr,
                         ctx->xsum32, ctx->ysum32, n, m, gv, s);
    launch_recenter(ctx->A, ctx->At, ctx->xr, ctx->yr, ctx->bh, ctx->ch, ctx->bh32, ctx->ch32, ctx->lo32, ctx->st, 0,
                    stride_grid(ctx, ctx->A), stride_grid(ctx, ctx->At), s);
    ctx->launches += 2;
  } else if (p32)
    launch_apply32(ctx->st, ctx->x32, ctx->y32, ctx->x, ctx->y, ctx->xavg, ctx->yavg, ctx->xr, ctx->yr, ctx->xsum32,
                   ctx->ysum32, n, m, gv, s);
  else
    launch_apply(ctx->st, ctx->x, ctx->y, ctx->xavg, ctx->yavg, ctx->xr, ctx->yr, ctx->xsum, ctx->ysum, n, m, gv, s);
  ctx->launches += (o.restarts && !o.halpern ? 4 : 0) + 3 + 2 + (o.restart_scheme == 1 ? 1 : 0);
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * ctx->count, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaGetLastError());
  return PDHG_OK;
}

pdhg_status enqueue_block(pdhg_ctx* ctx, int64_t nb);
pdhg_status enqueue_steps_batch(pdhg_ctx* ctx, int64_t nb, bool timing);
pdhg_status enqueue_eval_batch(pdhg_ctx* ctx);

// A whole evaluation block (nb = eval_every iterations + evaluation) as a CUDA
// graph: captured on first use for the current precision phase, replayed
// after. Kernel arguments are fixed pointers and the step sizes, tolerance
// and counters live in device memory, so one capture serves every block.
pdhg_status run_block_graph(pdhg_ctx* ctx, int64_t nb) {
  Range nvtx_range("pdhg/evaluation_block_graph");
  const int slot = ctx->phase32 ? 1 : 0;
  if (!ctx->graph_exec[slot]) {
    const int64_t launches0 = ctx->launches;
    cudaGraph_t g = nullptr;
    CK(ctx, cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    pdhg_status rs = enqueue_block(ctx, nb);
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &g);
    if (rs != PDHG_OK) {
      if (g) cudaGraphDestroy(g);
      return rs;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&ctx->graph_exec[slot], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    ctx->graph_launches[slot] = ctx->launches - launches0;
    ctx->launches = launches0;
  }
  CK(ctx, cudaGraphLaunch(ctx->graph_exec[slot], ctx->stream));
  ctx->launches += ctx->graph_launches[slot];
  ctx->graph_replays += 1;
  return PDHG_OK;
}

pdhg_status enqueue_block(pdhg_ctx* ctx, int64_t nb) {
  pdhg_status rs = ctx->count > 1 ? enqueue_steps_batch(ctx, nb, false) : enqueue_steps(ctx, nb, false);
  if (rs != PDHG_OK) return rs;
  return ctx->count > 1 ? enqueue_eval_batch(ctx) : enqueue_eval(ctx);
}

// ---- batch -------------------------------------------------------------------

pdhg_status setup_batch(pdhg_ctx* ctx, int count, const pdhg_lp_desc* lps) {
  Range nvtx_range("pdhg/setup_batch");
  const pdhg_options& o = ctx->opt;
  ctx->count = count;
  ctx->xoff_h.assign(count + 1, 0);
  ctx->yoff_h.assign(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    ctx->xoff_h[i + 1] = ctx->xoff_h[i] + (int)lps[i].n;
    ctx->yoff_h[i + 1] = ctx->yoff_h[i] + (int)lps[i].m;
  }
  const int64_t m = ctx->m, n = ctx->n, nnz = ctx->nnz;
  cudaStream_t s = ctx->stream;
  Scratch sc(s);
  // the instances' arrays, concatenated on the device
  std::vector<long long> rpoff(count), zoff(count + 1, 0);
  for (int i = 0; i < count; ++i) {
    rpoff[i] = (long long)ctx->yoff_h[i] + i;
    zoff[i + 1] = zoff[i] + lps[i].nnz;
  }
  long long* lrp = nullptr;
  int* lci = nullptr;
  double *lv = nullptr, *lb = nullptr, *lc = nullptr;
  CK(ctx, sc.take(&lrp, m + count));
  CK(ctx, sc.take(&lci, nnz));
  CK(ctx, sc.take(&lv, nnz));
  CK(ctx, sc.take(&lb, m));
  CK(ctx, sc.take(&lc, n));
  for (int i = 0; i < count; ++i) {
    const pdhg_lp_desc& L = lps[i];
    CK(ctx, cudaMemcpyAsync(lrp + rpoff[i], L.row_ptr, sizeof(long long) * (L.m + 1), cudaMemcpyHostToDevice, s));
    if (L.nnz) {
      CK(ctx, cudaMemcpyAsync(lci + zoff[i], L.col_idx, sizeof(int) * L.nnz, cudaMemcpyHostToDevice, s));
      CK(ctx, cudaMemcpyAsync(lv + zoff[i], L.val, sizeof(double) * L.nnz, cudaMemcpyHostToDevice, s));
    }
    CK(ctx, cudaMemcpyAsync(lb + ctx->yoff_h[i], L.b, sizeof(double) * L.m, cudaMemcpyHostToDevice, s));
    CK(ctx, cudaMemcpyAsync(lc + ctx->xoff_h[i], L.c, sizeof(double) * L.n, cudaMemcpyHostToDevice, s));
  }
  pdhg_status rs = build_layouts(ctx, sc, lrp, lci, lv, rpoff, zoff);
  if (rs != PDHG_OK) return rs;
  {
    std::vector<int> ustart(count + 1);
    for (int i = 0; i <= count; ++i) ustart[i] = ctx->bstart_h[i] * ctx->wpb;
    CK(ctx, dalloc(ctx, &ctx->ustart, count + 1));
    CK(ctx, cudaMemcpyAsync(ctx->ustart, ustart.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
    CK(ctx, cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i)
      ctx->persist_smem = std::max(ctx->persist_smem, persistent_smem_bytes(lps[i].n, lps[i].m));
  }
  Hyb& A = ctx->A;
  Hyb& At = ctx->At;
  CK(ctx, dalloc(ctx, &ctx->xoff, count + 1));
  CK(ctx, dalloc(ctx, &ctx->yoff, count + 1));
  CK(ctx, dalloc(ctx, &ctx->bstart, count + 1));
  double** vecs_n[] = {&ctx->c, &ctx->ch, &ctx->dc, &ctx->idc, &ctx->x, &ctx->xbar, &ctx->xsum, &ctx->xavg,
                       &ctx->xr, &ctx->tmp_n, &ctx->tmp_n2};
  double** vecs_m[] = {&ctx->b, &ctx->bh, &ctx->dr, &ctx->idr, &ctx->y, &ctx->ysum, &ctx->yavg, &ctx->yr,
                       &ctx->tmp_m};
  for (double** p : vecs_n) CK(ctx, dalloc(ctx, p, n));
  for (double** p : vecs_m) CK(ctx, dalloc(ctx, p, m));
  ctx->nb_eval = ctx->nblocks;
  CK(ctx, dalloc(ctx, &ctx->partials, (size_t)ctx->nblocks * NQ));
  CK(ctx, dalloc(ctx, &ctx->scal, (size_t)8 * count));
  CK(ctx, dalloc(ctx, &ctx->st, count));
  CK(ctx, dalloc(ctx, &ctx->kkt_sums, 1));
  CK(ctx, dalloc(ctx, &ctx->trace, 1));
  CK(ctx, dalloc(ctx, &ctx->sol, 2 * n + m));
  if (o.eps_cross > 0.0 || o.snapshot_every > 0) CK(ctx, dalloc(ctx, &ctx->bsnap, 2 * n + m));
  CK(ctx, cudaMallocHost(&ctx->h_st, sizeof(DevState) * count));
  CK(ctx, cudaMallocHost(&ctx->h_kkt, sizeof(EvalSums)));
  for (int i = 0; i < 3 * EV_POOL; ++i) CK(ctx, cudaEventCreate(&ctx->ev[i]));
  prefer_l1_for_step_kernels();
  CK(ctx, cudaMemcpyAsync(ctx->xoff, ctx->xoff_h.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->yoff, ctx->yoff_h.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->bstart, ctx->bstart_h.data(), sizeof(int) * (count + 1), cudaMemcpyHostToDevice, s));
  launch_gather_double(lb, ctx->perm_y, m, ctx->b, s);
  launch_gather_double(lc, ctx->perm_x, n, ctx->c, s);

  // scaling: row and column factors are per row / column, so one pass over
  // the block-diagonal layouts scales every instance by its own factors
  const int gn = vec_grid(ctx, n), gm = vec_grid(ctx, m);
  const int grA = stride_grid(ctx, A), grT = stride_grid(ctx, At);
  launch_fill(ctx->dr, 1.0, m, gm, s);
  launch_fill(ctx->dc, 1.0, n, gn, s);
  double* r = ctx->tmp_m;
  double* sf = ctx->tmp_n;
  for (int it = 0; it < o.ruiz_iters; ++it) {
    launch_row_absmax(A, r, grA, s);
    launch_row_absmax(At, sf, grT, s);
    launch_inv_sqrt_or_one(r, r, (int)m, gm, s);
    launch_inv_sqrt_or_one(sf, sf, (int)n, gn, s);
    launch_scale(A, r, sf, 0, grA, s);
    launch_scale(At, r, sf, 1, grT, s);
    for (int k = 0; ctx->panels_on && k < (ctx->pan32 ? 2 : 1); ++k)
      launch_scale(ctx->pan[k].Pn, r, sf, 2, stride_grid(ctx, ctx->pan[k].Pn), s, ctx->pan[k].col, ctx->pan[k].base);
    launch_mul_inplace(ctx->dr, r, (int)m, gm, s);
    launch_mul_inplace(ctx->dc, sf, (int)n, gn, s);
  }
  if (o.pock_chambolle) {
    launch_row_abspow_sum(A, o.pc_alpha, r, grA, s);
    launch_row_abspow_sum(At, 2.0 - o.pc_alpha, sf, grT, s);
    launch_inv_sqrt_or_one(r, r, (int)m, gm, s);
    launch_inv_sqrt_or_one(sf, sf, (int)n, gn, s);
    launch_scale(A, r, sf, 0, grA, s);
    launch_scale(At, r, sf, 1, grT, s);
    for (int k = 0; ctx->panels_on && k < (ctx->pan32 ? 2 : 1); ++k)
      launch_scale(ctx->pan[k].Pn, r, sf, 2, stride_grid(ctx, ctx->pan[k].Pn), s, ctx->pan[k].col, ctx->pan[k].base);
    launch_mul_inplace(ctx->dr, r, (int)m, gm, s);
    launch_mul_inplace(ctx->dc, sf, (int)n, gn, s);
  }
  launch_mul(ctx->bh, ctx->dr, ctx->b, (int)m, gm, s);
  launch_mul(ctx->ch, ctx->dc, ctx->c, (int)n, gn, s);
  launch_reciprocal(ctx->idr, ctx->dr, (int)m, gm, s);
  launch_reciprocal(ctx->idc, ctx->dc, (int)n, gn, s);

  // power iteration, norms and step sizes per instance
  const int gx = std::max(1, std::min(64, (int)(n / count / TPB + 1)));
  double* v = ctx->tmp_n;
  double* w = ctx->tmp_n2;
  double* u = ctx->tmp_m;
  launch_fill(ctx->scal, 0.0, (long long)8 * count, vec_grid(ctx, 8 * count), s);
  launch_power_start(w, ctx->perm_x, ctx->xoff, count, (int)n, gx, s);
  launch_sumsq_b(w, ctx->xoff, count, ctx->scal + 6, 8, s);
  launch_div_by_norm_b(v, w, ctx->scal + 6, 8, ctx->xoff, count, gx, s);
  for (int it = 0; it < o.power_iters; ++it) {  // the last iteration's ||Ahat v|| per instance (as above)
    launch_spmv(A, v, u, grA, s);
    if (it == o.power_iters - 1) launch_sumsq_b(u, ctx->yoff, count, ctx->scal + 0, 8, s);
    launch_spmv(At, u, w, grT, s);
    launch_sumsq_b(w, ctx->xoff, count, ctx->scal + 5, 8, s);
    launch_div_by_norm_b(v, w, ctx->scal + 5, 8, ctx->xoff, count, gx, s);
  }
  launch_sumsq_b(ctx->ch, ctx->xoff, count, ctx->scal + 1, 8, s);
  launch_sumsq_b(ctx->bh, ctx->yoff, count, ctx->scal + 2, 8, s);
  launch_sumsq_b(ctx->b, ctx->yoff, count, ctx->scal + 3, 8, s);
  launch_sumsq_b(ctx->c, ctx->xoff, count, ctx->scal + 4, 8, s);
  CK(ctx, cudaGetLastError());
  DevState h{};
  h.eps_factor = o.eps_factor;
  h.beta_suff = o.beta_suff;
  h.beta_nec = o.beta_nec;
  h.beta_art = o.beta_art;
  h.theta = o.theta;
  h.restarts_on = o.restarts;
  h.primal_weight_on = o.primal_weight;
  h.halpern = o.halpern;
  h.rho = o.halpern_reflect;
  h.gap_tol = o.gap_tol;
  h.eps_target = o.eps_cross;  // Algorithm 1's schedule, per instance
  h.snapshot_every = o.snapshot_every;
  h.next_snapshot = o.snapshot_every;
  for (int i = 0; i < count; ++i) ctx->h_st[i] = h;
  CK(ctx, cudaMemcpyAsync(ctx->st, ctx->h_st, sizeof(DevState) * count, cudaMemcpyHostToDevice, s));
  launch_finish_setup_b(ctx->st, count, ctx->scal, 8, o.step_factor, o.primal_weight, s);

  // start at zero; the starting point is each instance's restart reference
  launch_fill(ctx->x, 0.0, n, gn, s);
  launch_fill(ctx->y, 0.0, m, gm, s);
  launch_fill(ctx->xsum, 0.0, n, gn, s);
  launch_fill(ctx->ysum, 0.0, m, gm, s);
  launch_fill(ctx->xr, 0.0, n, gn, s);
  launch_fill(ctx->yr, 0.0, m, gm, s);
  launch_fill(ctx->xavg, 0.0, n, gn, s);
  launch_fill(ctx->yavg, 0.0, m, gm, s);
  launch_eval_point(A, At, ctx->x, ctx->y, ctx->bh, ctx->ch, ctx->idr, ctx->idc, nullptr, nullptr, ctx->partials,
                    ctx->nblocks, s, ctx->st, ctx->binst, 32 * ctx->wpb);
  launch_eval_finalize_b(ctx->partials, ctx->bstart, count, &ctx->st->cur, sizeof(DevState), s);
  launch_init_restart_ref_b(ctx->st, count, s);
  CK(ctx, cudaGetLastError());
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  for (int i = 0; i < count; ++i)
    if (!std::isfinite(ctx->h_st[i].norm_est) || !std::isfinite(ctx->h_st[i].omega))
      return fail(ctx, PDHG_ERR_NUMERIC, "non-finite norm estimate or primal weight after scaling");
  return PDHG_OK;
}

// Evaluate the current and average points of every active instance.
void eval_batch(pdhg_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  const int count = ctx->count;
  const int gx = std::max(1, std::min(64, (int)(ctx->n / count / TPB + 1)));
  if (ctx->opt.restarts && !ctx->opt.halpern) {  // Halpern: no averages
    launch_make_average_b(ctx->xsum, ctx->ysum, ctx->x, ctx->y, ctx->xavg, ctx->yavg, ctx->xoff, ctx->yoff, ctx->st,
                          count, gx, s);
    launch_eval_point(ctx->A, ctx->At, ctx->xavg, ctx->yavg, ctx->bh, ctx->ch, ctx->idr, ctx->idc, ctx->xr, ctx->yr,
                      ctx->partials, ctx->nblocks, s, ctx->st, ctx->binst, 32 * ctx->wpb);
    launch_eval_finalize_b(ctx->partials, ctx->bstart, count, &ctx->st->avg, sizeof(DevState), s);
  }
  launch_eval_point(ctx->A, ctx->At, ctx->x, ctx->y, ctx->bh, ctx->ch, ctx->idr, ctx->idc, ctx->xr, ctx->yr,
                    ctx->partials, ctx->nblocks, s, ctx->st, ctx->binst, 32 * ctx->wpb);
  launch_eval_finalize_b(ctx->partials, ctx->bstart, count, &ctx->st->cur, sizeof(DevState), s);
  launch_decide_b(ctx->st, count, s);
  launch_apply_b(ctx->st, ctx->x, ctx->y, ctx->xavg, ctx->yavg, ctx->xr, ctx->yr, ctx->xsum, ctx->ysum, ctx->xoff,
                 ctx->yoff, count, gx, s);
  if (ctx->bsnap)
    launch_snap_b(ctx->At, ctx->st, ctx->binst, ctx->nblocks, ctx->perm_x, ctx->perm_y, ctx->x, ctx->y, ctx->xavg,
                  ctx->yavg, ctx->ch, ctx->dc, ctx->dr, ctx->bsnap, ctx->bsnap + ctx->n, ctx->bsnap + ctx->n + ctx->m,
                  ctx->yoff, count, gx, 32 * ctx->wpb, s);
}

pdhg_status enqueue_steps_batch(pdhg_ctx* ctx, int64_t nb, bool timing) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  for (int64_t it = 0; it < nb; ++it) {
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it], s));
    if (o.halpern)
      launch_primal_step_halpern<double>(ctx->At, ctx->At.v, ctx->y, ctx->ch, ctx->x, ctx->xbar, ctx->xr, ctx->st,
                                         (int)it, ctx->nblocks, s, 32 * ctx->wpb, ctx->binst);
    else
      launch_primal_step(ctx->At, ctx->y, ctx->ch, ctx->x, ctx->xbar, ctx->xsum, ctx->st, o.restarts, ctx->nblocks, s,
                         ctx->binst, 32 * ctx->wpb);
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 1], s));
    if (o.halpern)
      launch_dual_step_halpern<double>(ctx->A, ctx->A.v, ctx->xbar, ctx->bh, ctx->y, ctx->yr, ctx->st, (int)it,
                                       ctx->nblocks, s, 32 * ctx->wpb, ctx->binst);
    else
      launch_dual_step(ctx->A, ctx->xbar, ctx->bh, ctx->y, ctx->ysum, ctx->st, o.restarts, ctx->nblocks, s,
                       ctx->binst, 32 * ctx->wpb);
    if (timing) CK(ctx, cudaEventRecord(ctx->ev[3 * it + 2], s));
  }
  launch_add_counters_b(ctx->st, ctx->count, nb, s);
  ctx->launches += 2 * nb + 1;
  CK(ctx, cudaGetLastError());
  return PDHG_OK;
}

pdhg_status enqueue_eval_batch(pdhg_ctx* ctx) {
  Range nvtx_range("pdhg/evaluation_batch");
  eval_batch(ctx);
  ctx->launches += (ctx->opt.restarts ? 4 : 0) + 3 + 2 + (ctx->bsnap ? 2 : 0);
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * ctx->count, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaGetLastError());
  return PDHG_OK;
}

// pdhg_iterate with option persistent: the solve loop runs on the device, one
// block per LP; the host launches again only after a snapshot it has to take.
pdhg_status iterate_persistent(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int count = ctx->count;
  const bool batch = count > 1;
  for (int i = 0; i < count; ++i) {
    ctx->h_st[i].tol = tol;
    CK(ctx, cudaMemcpyAsync(&ctx->st[i].tol, &ctx->h_st[i].tol, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  PersistentArgs a{};
  a.eval_every = o.eval_every;
  a.evaluating = batch || o.restarts || tol > 0.0 || o.eps_cross > 0.0 || o.snapshot_every > 0;
  a.restarts = o.restarts;
  a.batch = batch;
  a.n = (int)ctx->n;
  a.m = (int)ctx->m;
  a.xoff = batch ? ctx->xoff : nullptr;
  a.yoff = batch ? ctx->yoff : nullptr;
  a.ustart = batch ? ctx->ustart : nullptr;
  a.x = ctx->x;
  a.xbar = ctx->xbar;
  a.xsum = ctx->xsum;
  a.xr = ctx->xr;
  a.xavg = ctx->xavg;
  a.y = ctx->y;
  a.ysum = ctx->ysum;
  a.yr = ctx->yr;
  a.yavg = ctx->yavg;
  a.ch = ctx->ch;
  a.idc = ctx->idc;
  a.bh = ctx->bh;
  a.idr = ctx->idr;
  ctx->converged = false;
  int64_t done = 0;
  while (done < max_iters) {
    a.max_iters = max_iters - done;
    CK(ctx, launch_solve_block(ctx->A, ctx->At, a, count, ctx->persist_smem, ctx->st, batch ? nullptr : ctx->trace,
                               s));
    ctx->launches += 1;
    CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * count, cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    int64_t k_new = ctx->k;
    bool all_done = true;
    for (int i = 0; i < count; ++i) {
      const DevState& h = ctx->h_st[i];
      if (h.numeric && !(batch && h.frozen)) {
        if (iters_done) *iters_done = done;
        return fail(ctx, PDHG_ERR_NUMERIC,
                    batch ? "NaN or Inf in the iterates of instance " + std::to_string(i) : "NaN or Inf in the iterates");
      }
      k_new = std::max<int64_t>(k_new, h.k);
      all_done = all_done && (batch ? h.frozen != 0 : h.converged != 0);
    }
    const int64_t step = k_new - ctx->k;
    ctx->k = k_new;
    done += step;
    if (!batch && ctx->h_st->snapshot_flag) {
      pdhg_status rs = take_snapshot(ctx);
      if (rs != PDHG_OK) return rs;
      ctx->launches += 2;
    }
    if (all_done) {
      ctx->converged = true;
      break;
    }
    if (batch || step == 0) break;  // a batch launch runs every instance to its end
  }
  if (iters_done) *iters_done = done;
  if (ctx->converged || tol == 0.0) return PDHG_OK;
  return fail(ctx, PDHG_ERR_NOT_CONVERGED, "iteration limit reached before the tolerance");
}

// The launch (plus the copies around it) of one pdhg_iterate call on a batch
// with persistent = 2: the control block to the device, the cooperative solve,
// the states and the control block back.
pdhg_status enqueue_batch_solve(pdhg_ctx* ctx) {
  cudaStream_t s = ctx->stream;
  BatchArgs a{};
  a.A = ctx->A;
  a.At = ctx->At;
  a.binst = ctx->binst;
  a.bstart = ctx->bstart;
  a.xoff = ctx->xoff;
  a.yoff = ctx->yoff;
  a.nvb = ctx->nblocks;
  a.count = ctx->count;
  a.eval_every = ctx->opt.eval_every;
  a.restarts = ctx->opt.restarts;
  a.halpern = ctx->opt.halpern;
  a.x = ctx->x;
  a.xbar = ctx->xbar;
  a.xsum = ctx->xsum;
  a.xr = ctx->xr;
  a.xavg = ctx->xavg;
  a.y = ctx->y;
  a.ysum = ctx->ysum;
  a.yr = ctx->yr;
  a.yavg = ctx->yavg;
  a.ch = ctx->ch;
  a.bh = ctx->bh;
  a.idc = ctx->idc;
  a.idr = ctx->idr;
  a.part_avg = ctx->partials_avg;
  a.part_cur = ctx->partials;
  a.sts = ctx->st;
  a.ctl = ctx->bctl;
  if (ctx->bsnap) {
    a.snap_x = ctx->bsnap;
    a.snap_y = ctx->bsnap + ctx->n;
    a.snap_z = ctx->bsnap + ctx->n + ctx->m;
    a.perm_x = ctx->perm_x;
    a.perm_y = ctx->perm_y;
    a.dc = ctx->dc;
    a.dr = ctx->dr;
  }
  CK(ctx, cudaMemcpyAsync(ctx->bctl, ctx->h_bctl, sizeof(BatchCtl), cudaMemcpyHostToDevice, s));
  CK(ctx, launch_batch_solve(a, ctx->bgrid, 32 * ctx->wpb, s));
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * ctx->count, cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(ctx->h_bctl, ctx->bctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, s));
  return PDHG_OK;
}

// pdhg_iterate for a batch with persistent = 2: ONE cooperative launch runs
// every active instance until it meets the tolerance, or max_iters
// iterations; the varying inputs (iteration count so far, budget) sit in the
// device control block, so a captured CUDA graph of the launch and its copies
// serves every call. A barrier wait that gives up ends the launch with
// PDHG_ERR_TIMEOUT (the context's iterates are then partly updated, but the
// context still answers queries).
pdhg_status iterate_batch_coop(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done) {
  Range nvtx_range("pdhg/batch_cooperative_launch");
  cudaStream_t s = ctx->stream;
  const int count = ctx->count;
  for (int i = 0; i < count; ++i) ctx->h_st[i].tol = tol;
  for (int i = 0; i < count; ++i)
    CK(ctx, cudaMemcpyAsync(&ctx->st[i].tol, &ctx->h_st[i].tol, sizeof(double), cudaMemcpyHostToDevice, s));
  if (!ctx->bctl) {
    CK(ctx, dalloc(ctx, &ctx->bctl, 1));
    CK(ctx, dalloc(ctx, &ctx->partials_avg, (size_t)ctx->nblocks * NQ));
    CK(ctx, cudaMallocHost(&ctx->h_bctl, sizeof(BatchCtl)));
    memset(ctx->h_bctl, 0, sizeof(BatchCtl));
    CK(ctx, batch_solve_grid(32 * ctx->wpb, &ctx->bgrid));
  }
  int active = 0;
  for (int i = 0; i < count; ++i) active += ctx->h_st[i].frozen ? 0 : 1;
  if (iters_done) *iters_done = 0;
  if (active == 0 || max_iters == 0) {
    CK(ctx, cudaStreamSynchronize(s));
    ctx->converged = active == 0;
    return ctx->converged || tol == 0.0 ? PDHG_OK
                                        : fail(ctx, PDHG_ERR_NOT_CONVERGED, "iteration limit reached before every "
                                                                            "instance met the tolerance");
  }
  BatchCtl& h = *ctx->h_bctl;
  h.k0 = ctx->k;
  h.max_iters = max_iters;
  h.budget = ctx->opt.barrier_cycles > 0 ? ctx->opt.barrier_cycles : (1LL << 31);
  h.done = -1;
  h.arrive = 0;
  h.gen = 0;
  h.error = BATCH_ERR_NONE;
  h.where = 0;
  h.active = active;
  bool replayed = false;
  if (ctx->opt.use_graphs && !ctx->bgraph_failed) {
    if (!ctx->bgraph) {
      // capture once; if the cooperative launch cannot be captured, launch it
      // directly from then on
      cudaGraph_t g = nullptr;
      CK(ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      pdhg_status rs = enqueue_batch_solve(ctx);
      cudaError_t e = cudaStreamEndCapture(s, &g);
      if (rs == PDHG_OK && e == cudaSuccess) e = cudaGraphInstantiate(&ctx->bgraph, g, 0);
      if (g) cudaGraphDestroy(g);
      if (rs != PDHG_OK || e != cudaSuccess) {
        ctx->bgraph = nullptr;
        ctx->bgraph_failed = true;
        cudaGetLastError();  // clear a capture error; the direct launch below reports its own
      }
    }
    if (ctx->bgraph) {
      CK(ctx, cudaGraphLaunch(ctx->bgraph, s));
      ctx->graph_replays += 1;
      replayed = true;
    }
  }
  if (!replayed) {
    pdhg_status rs = enqueue_batch_solve(ctx);
    if (rs != PDHG_OK) return rs;
  }
  ctx->launches += 1;
  CK(ctx, cudaStreamSynchronize(s));
  int64_t done = h.done;
  if (done < 0) {  // the launch ended early: the iterations the instances ran
    done = 0;
    for (int i = 0; i < count; ++i) done = std::max<int64_t>(done, ctx->h_st[i].k - ctx->k);
  }
  ctx->k += done;
  if (iters_done) *iters_done = done;
  if (h.error == BATCH_ERR_TIMEOUT)
    return fail(ctx, PDHG_ERR_TIMEOUT,
                "a grid-barrier wait of the cooperative batch launch gave up (barrier " + std::to_string(h.where) +
                    " of the launch, after " + std::to_string((long long)h.budget) + " clock cycles)");
  bool all_done = true;
  for (int i = 0; i < count; ++i) {
    if (ctx->h_st[i].numeric && !ctx->h_st[i].frozen)
      return fail(ctx, PDHG_ERR_NUMERIC, "NaN or Inf in the iterates of instance " + std::to_string(i));
    all_done = all_done && ctx->h_st[i].frozen;
  }
  ctx->converged = all_done;
  if (all_done || tol == 0.0) return PDHG_OK;
  return fail(ctx, PDHG_ERR_NOT_CONVERGED, "iteration limit reached before every instance met the tolerance");
}

pdhg_status iterate_batch(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done) {
  const pdhg_options& o = ctx->opt;
  cudaStream_t s = ctx->stream;
  const int count = ctx->count;
  // tolerance of every instance (the rest of the state stays on the device)
  for (int i = 0; i < count; ++i) ctx->h_st[i].tol = tol;
  for (int i = 0; i < count; ++i)
    CK(ctx, cudaMemcpyAsync(&ctx->st[i].tol, &ctx->h_st[i].tol, sizeof(double), cudaMemcpyHostToDevice, s));
  const bool graphs = o.use_graphs && !o.kernel_timing;
  int64_t done = 0;
  bool all_done = false;
  while (done < max_iters && !all_done) {
    const int64_t nb = std::min<int64_t>(o.eval_every - (ctx->k % o.eval_every), max_iters - done);
    const bool timing = o.kernel_timing && nb <= EV_POOL;
    const bool eval_now = (ctx->k + nb) % o.eval_every == 0;
    pdhg_status rs;
    if (graphs && eval_now && nb == o.eval_every) {
      rs = run_block_graph(ctx, nb);
    } else {
      rs = enqueue_steps_batch(ctx, nb, timing);
      if (rs == PDHG_OK && eval_now) rs = enqueue_eval_batch(ctx);
    }
    if (rs != PDHG_OK) return rs;
    ctx->k += nb;
    done += nb;
    if (timing) {
      CK(ctx, cudaEventSynchronize(ctx->ev[3 * (nb - 1) + 2]));
      for (int64_t it = 0; it < nb; ++it) {
        float a = 0.f, bms = 0.f;
        CK(ctx, cudaEventElapsedTime(&a, ctx->ev[3 * it], ctx->ev[3 * it + 1]));
        CK(ctx, cudaEventElapsedTime(&bms, ctx->ev[3 * it + 1], ctx->ev[3 * it + 2]));
        ctx->ms_primal += a;
        ctx->ms_dual += bms;
      }
      ctx->launches_primal += nb;
      ctx->launches_dual += nb;
    }
    if (eval_now) {
      CK(ctx, cudaStreamSynchronize(s));
      all_done = true;
      for (int i = 0; i < count; ++i) {
        if (ctx->h_st[i].numeric && !ctx->h_st[i].frozen) {
          if (iters_done) *iters_done = done;
          return fail(ctx, PDHG_ERR_NUMERIC, "NaN or Inf in the iterates of instance " + std::to_string(i));
        }
        all_done = all_done && ctx->h_st[i].frozen;
      }
    }
  }
  CK(ctx, cudaStreamSynchronize(s));
  if (iters_done) *iters_done = done;
  ctx->converged = all_done;
  if (all_done || tol == 0.0) return PDHG_OK;
  return fail(ctx, PDHG_ERR_NOT_CONVERGED, "iteration limit reached before every instance met the tolerance");
}


// ---- feasibility polishing -----------------------------------------------------

// Whole evaluation blocks of a polishing phase until its test is met (the
// decision kernel's converged flag) or `budget` iterations; a NaN/Inf ends the
// phase as not met.
pdhg_status polish_phase_run(pdhg_ctx* ctx, int64_t budget, bool graphs, int64_t* iters, bool* met) {
  const int64_t E = ctx->opt.eval_every;
  *iters = 0;
  *met = false;
  while (*iters < budget) {
    pdhg_status rs = graphs ? run_block_graph(ctx, E) : enqueue_block(ctx, E);
    if (rs != PDHG_OK) return rs;
    ctx->k += E;
    *iters += E;
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->h_st->numeric) break;
    if (ctx->h_st->converged) {
      *met = true;
      break;
    }
  }
  return PDHG_OK;
}

// Set up a phase: the current (x, y) is its start and restart reference, the
// averages are empty, and the start is evaluated on the phase's problem.
pdhg_status polish_phase_begin(pdhg_ctx* ctx, int term_mode) {
  const int64_t n = ctx->n, m = ctx->m;
  cudaStream_t s = ctx->stream;
  CK(ctx, cudaMemsetAsync(ctx->xsum, 0, sizeof(double) * n, s));
  CK(ctx, cudaMemsetAsync(ctx->ysum, 0, sizeof(double) * m, s));
  CK(ctx, cudaMemcpyAsync(ctx->xr, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(ctx, cudaMemcpyAsync(ctx->yr, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
  eval_point(ctx, ctx->x, ctx->y, nullptr, nullptr, &ctx->st->cur);
  launch_polish_begin(ctx->st, term_mode, s);
  ctx->launches += 3;
  CK(ctx, cudaGetLastError());
  ctx->k = 0;
  return PDHG_OK;
}

// One attempt of feasibility polishing after an evaluation of the main solve
// (h_st holds its decisions): a primal phase (chat = 0) from (x_c, 0) until
// rel_p <= tol, then a dual phase (bhat = 0) from (0, y_c) until rel_d <= tol,
// each for at most `budget` iterations, with the main solve's scaling, step
// and current primal weight. The main state (iterates, sums, restart point,
// device state, iteration count) is saved before and restored after; when the
// pair (x_p, y_d) passes the termination test on the LP as given, it becomes
// the current iterate and *solved is set.
pdhg_status feas_polish(pdhg_ctx* ctx, double tol, int64_t budget, bool graphs, bool* solved) {
  Range nvtx_range("pdhg/feasibility_polishing");
  *solved = false;
  const int64_t n = ctx->n, m = ctx->m;
  cudaStream_t s = ctx->stream;
  if (!ctx->fp_buf) CK(ctx, dalloc(ctx, &ctx->fp_buf, (size_t)6 * (n + m)));
  double *sx = ctx->fp_buf, *sxs = sx + n, *sxr = sx + 2 * n, *xc = sx + 3 * n, *xp = sx + 4 * n, *sch = sx + 5 * n;
  double *sy = ctx->fp_buf + 6 * n, *sys = sy + m, *syr = sy + 2 * m, *yc = sy + 3 * m, *yd = sy + 4 * m,
         *sbh = sy + 5 * m;
  const DevState saved = *ctx->h_st;
  const int64_t k_saved = ctx->k;
  const bool avg = saved.candidate == KIND_AVG;
  const size_t bn = sizeof(double) * n, bm = sizeof(double) * m;
  const cudaMemcpyKind d2d = cudaMemcpyDeviceToDevice;
  double* save_n[][2] = {{sx, ctx->x}, {sxs, ctx->xsum}, {sxr, ctx->xr}, {xc, avg ? ctx->xavg : ctx->x},
                         {sch, ctx->ch}};
  double* save_m[][2] = {{sy, ctx->y}, {sys, ctx->ysum}, {syr, ctx->yr}, {yc, avg ? ctx->yavg : ctx->y},
                         {sbh, ctx->bh}};
  for (auto& p : save_n) CK(ctx, cudaMemcpyAsync(p[0], p[1], bn, d2d, s));
  for (auto& p : save_m) CK(ctx, cudaMemcpyAsync(p[0], p[1], bm, d2d, s));
  pdhg_polish_rec rec{};
  rec.iteration = k_saved;
  rec.budget = budget;
  rec.rel_kkt = rec.rel_gap = INFINITY;

  // primal phase: objective 0, start (x_c, 0)
  CK(ctx, cudaMemsetAsync(ctx->ch, 0, bn, s));
  CK(ctx, cudaMemcpyAsync(ctx->x, xc, bn, d2d, s));
  CK(ctx, cudaMemsetAsync(ctx->y, 0, bm, s));
  pdhg_status rs = polish_phase_begin(ctx, TERM_PRIMAL);
  if (rs != PDHG_OK) return rs;
  bool okp = false, okd = false;
  rs = polish_phase_run(ctx, budget, graphs, &rec.primal_iters, &okp);
  if (rs != PDHG_OK) return rs;
  rec.primal_ok = okp;
  CK(ctx, cudaMemcpyAsync(xp, ctx->x, bn, d2d, s));
  CK(ctx, cudaMemcpyAsync(ctx->ch, sch, bn, d2d, s));
  if (okp) {
    // dual phase: right-hand side 0, start (0, y_c)
    CK(ctx, cudaMemsetAsync(ctx->bh, 0, bm, s));
    CK(ctx, cudaMemsetAsync(ctx->x, 0, bn, s));
    CK(ctx, cudaMemcpyAsync(ctx->y, yc, bm, d2d, s));
    rs = polish_phase_begin(ctx, TERM_DUAL);
    if (rs != PDHG_OK) return rs;
    rs = polish_phase_run(ctx, budget, graphs, &rec.dual_iters, &okd);
    if (rs != PDHG_OK) return rs;
    rec.dual_ok = okd;
    CK(ctx, cudaMemcpyAsync(yd, ctx->y, bm, d2d, s));
    CK(ctx, cudaMemcpyAsync(ctx->bh, sbh, bm, d2d, s));
  }
  ctx->fp_iters += rec.primal_iters + rec.dual_iters;
  double rel_p = INFINITY, rel_d = INFINITY;
  if (okp && okd) {
    // the pair on the LP as given
    eval_point(ctx, xp, yd, nullptr, nullptr, ctx->kkt_sums);
    ctx->launches += 2;
    CK(ctx, cudaGetLastError());
    CK(ctx, cudaMemcpyAsync(ctx->h_kkt, ctx->kkt_sums, sizeof(EvalSums), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    const double* q = ctx->h_kkt->q;
    rel_p = sqrt(q[Q_RP2U]) / (1.0 + saved.b_norm);
    rel_d = sqrt(q[Q_RD2U]) / (1.0 + saved.c_norm);
    rec.rel_gap = fabs(q[Q_CX] - q[Q_BY]) / (1.0 + fabs(q[Q_CX]) + fabs(q[Q_BY]));
    rec.rel_kkt = std::max(rel_p, std::max(rel_d, rec.rel_gap));
  }
  const double gtol = ctx->opt.gap_tol > 0.0 ? ctx->opt.gap_tol : tol;
  *solved = okp && okd && rel_p <= tol && rel_d <= tol && rec.rel_gap <= gtol;
  ctx->fp_log.push_back(rec);

  // restore the main solve, or end it with the polished pair
  for (auto& p : save_n)
    if (p[1] != ctx->xavg && p[1] != ctx->ch) CK(ctx, cudaMemcpyAsync(p[1], p[0], bn, d2d, s));
  for (auto& p : save_m)
    if (p[1] != ctx->yavg && p[1] != ctx->bh) CK(ctx, cudaMemcpyAsync(p[1], p[0], bm, d2d, s));
  *ctx->h_st = saved;
  if (*solved) {
    CK(ctx, cudaMemcpyAsync(ctx->x, xp, bn, d2d, s));
    CK(ctx, cudaMemcpyAsync(ctx->y, yd, bm, d2d, s));
    ctx->h_st->converged = 1;
    ctx->h_st->cand_rel_kkt = rec.rel_kkt;
    ctx->h_st->cand_rel_gap = rec.rel_gap;
    ctx->fp_polished = true;
  }
  CK(ctx, cudaMemcpyAsync(ctx->st, ctx->h_st, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(ctx, cudaStreamSynchronize(s));
  ctx->k = k_saved;
  return PDHG_OK;
}

}  // namespace

extern "C" {

void pdhg_default_options(pdhg_options* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = PDHG_FP64;
  o->ruiz_iters = 10;
  o->pock_chambolle = 1;
  o->pc_alpha = 1.0;
  o->power_iters = 100;
  o->step_factor = 0.9;
  o->restarts = 1;
  o->primal_weight = 1;
  o->eval_every = 64;
  o->beta_suff = 0.2;
  o->beta_nec = 0.8;
  o->beta_art = 0.36;
  o->theta = 0.5;
  o->eps_cross = 0.0;
  o->eps_factor = 0.1;
  o->snapshot_every = 0;
  o->inputs_on_device = 0;
  o->use_graphs = 1;
  o->kernel_timing = 0;
  o->polish_switch = -1.0;
  o->long_row_min = 128;
  o->rows_per_thread = 4;
  o->dual_hot_cols = 0;
  o->singleton_order = 1;
  o->panel_min_len = 0;
  o->barrier_cycles = 0;
  o->restart_scheme = 0;
  o->values32 = -1;
  o->pid_kp = 0.99;
  o->pid_ki = 0.01;
  o->pid_kd = 0.0;
  o->record_for_backward = 0;
  o->checkpoint_every = 50;
  o->step_block = 256;
  o->primal_panels = -1;
  o->panel_rows = 0;
  o->halpern = 0;
  o->halpern_reflect = 1.0;
  o->gap_tol = 0.0;
  o->feas_polish = 0;
  o->polish_div = 8;
  o->stream_steps = 0;
  o->stream_warps = 0;
  o->stream_depth = 3;
  o->refine32 = -1;
  o->panel_overlap = -1;
  o->panel_balance = -1;
}

pdhg_status pdhg_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                        const double* val, const double* b, const double* c, const double* x0, const double* y0,
                        const pdhg_options* opt, void* cuda_stream, pdhg_ctx** out) {
  if (!out) return fail(nullptr, PDHG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (m < 1 || n < 1 || m >= (1LL << 31) - 1 || n >= (1LL << 31) - 1)
    return fail(nullptr, PDHG_ERR_INVALID, "m and n must be in [1, 2^31 - 1)");
  if (nnz < 0 || nnz >= (1LL << 31) - 1) return fail(nullptr, PDHG_ERR_INVALID, "nnz must be in [0, 2^31 - 1)");
  if (!row_ptr || (nnz > 0 && (!col_idx || !val)) || !b || !c)
    return fail(nullptr, PDHG_ERR_INVALID, "NULL array argument");
  pdhg_options o;
  if (opt)
    o = *opt;
  else
    pdhg_default_options(&o);
  if (o.precision != PDHG_FP64 && o.precision != PDHG_FP32 && o.precision != PDHG_MIXED)
    return fail(nullptr, PDHG_ERR_INVALID, "precision must be PDHG_FP64, PDHG_FP32 or PDHG_MIXED");
  if (o.record_for_backward &&
      (o.restarts || o.primal_weight || o.precision == PDHG_MIXED || o.checkpoint_every < 1))
    return fail(nullptr, PDHG_ERR_INVALID,
                "record_for_backward needs restarts = 0, primal_weight = 0 (fixed steps), precision FP64 or FP32 "
                "and checkpoint_every >= 1");
  if (o.eval_every < 1 || o.ruiz_iters < 0 || o.power_iters < 1 || !(o.step_factor > 0.0) || o.pc_alpha < 0.0 ||
      o.pc_alpha > 2.0 || o.long_row_min < 1 || o.dual_hot_cols < 0 || o.dual_hot_cols > HOT_MAX ||
      !(o.rows_per_thread == 1 || o.rows_per_thread == 2 || o.rows_per_thread == 4) || o.snapshot_every < 0 ||
      o.eps_cross < 0.0 || !(o.eps_factor > 0.0 && o.eps_factor < 1.0))
    return fail(nullptr, PDHG_ERR_INVALID, "option out of range");
  if (o.singleton_order < 0 || o.singleton_order > 1)
    return fail(nullptr, PDHG_ERR_INVALID, "singleton_order must be 0 or 1");
  if (o.panel_min_len < 0) return fail(nullptr, PDHG_ERR_INVALID, "panel_min_len must be >= 0");
  if (!(o.step_block == 0 || o.step_block == 128 || o.step_block == 256 || o.step_block == 512))
    return fail(nullptr, PDHG_ERR_INVALID, "step_block must be 128, 256 or 512");
  // a context that only ever runs FP32 steps (PDHG_FP32) can hold twice the
  // entries of y in a panel
  const long long panel_max = PANEL_SMEM_MAX / (o.precision == PDHG_FP32 ? 4 : 8);
  if (o.primal_panels < -1 || o.primal_panels > 1 || o.panel_rows < 0 || o.panel_rows > panel_max)
    return fail(nullptr, PDHG_ERR_INVALID,
                "primal_panels must be -1, 0 or 1 and panel_rows in [0, 28160] (56320 with precision PDHG_FP32)");
  if (o.persistent && o.primal_panels == 1)
    return fail(nullptr, PDHG_ERR_INVALID, "persistent = 1 and primal_panels = 1 exclude each other");
  if (o.halpern != 0 && (o.halpern != 1 || o.persistent || o.record_for_backward || !(o.halpern_reflect >= 0.0) ||
                         !(o.halpern_reflect <= 1.0)))
    return fail(nullptr, PDHG_ERR_INVALID,
                "halpern = 1 needs halpern_reflect in [0, 1], and no persistent loop or recording");
  if (o.persistent == 2)
    return fail(nullptr, PDHG_ERR_INVALID, "persistent = 2 (one cooperative launch) is for batches");
  if (o.persistent) {
    if (o.persistent != 1 || o.precision != PDHG_FP64 || o.record_for_backward || o.kernel_timing ||
        o.dual_hot_cols)
      return fail(nullptr, PDHG_ERR_INVALID,
                  "persistent = 1 needs precision FP64 and no recording, kernel timing or hot columns");
    if (7 * n + 6 * m > PERSIST_MAX_DOUBLES)
      return fail(nullptr, PDHG_ERR_INVALID,
                  "persistent: the LP's vectors (7n + 6m doubles) exceed one block's shared memory (28672)");
  }

  if (!(o.gap_tol >= 0.0) || o.feas_polish < 0 || o.feas_polish > 1 || o.polish_div < 1)
    return fail(nullptr, PDHG_ERR_INVALID, "gap_tol must be >= 0, feas_polish 0 or 1 and polish_div >= 1");
  if (o.feas_polish && (o.persistent || o.record_for_backward))
    return fail(nullptr, PDHG_ERR_INVALID, "feas_polish = 1 needs no persistent loop and no recording");
  if (o.restart_scheme < 0 || o.restart_scheme > 1 ||
      (o.restart_scheme == 1 && (o.halpern != 1 || o.feas_polish || o.persistent)) || !std::isfinite(o.pid_kp) ||
      !std::isfinite(o.pid_ki) || !std::isfinite(o.pid_kd))
    return fail(nullptr, PDHG_ERR_INVALID,
                "restart_scheme must be 0 or 1 (1: with halpern = 1, no feasibility polishing or persistent loop) "
                "and the PID gains finite");
  if (o.values32 < -1 || o.values32 > 1 ||
      (o.values32 == 1 && (o.precision == PDHG_FP32 || o.persistent || o.record_for_backward)))
    return fail(nullptr, PDHG_ERR_INVALID,
                "values32 must be -1, 0 or 1 (1: precision FP64 or MIXED, no persistent loop, no recording)");
  if (o.stream_steps < 0 || o.stream_steps > 1 || o.stream_warps < 0 || o.stream_warps > STREAM_TPB_MAX / 32 ||
      o.stream_depth < 2 || o.stream_depth > 8 || (o.stream_steps && (o.persistent || o.dual_hot_cols)))
    return fail(nullptr, PDHG_ERR_INVALID,
                "stream_steps must be 0 or 1 (1: no persistent loop or hot columns), stream_warps in [0, 16] and "
                "stream_depth in [2, 8]");
  if (o.refine32 < -1 || o.refine32 > 1 ||
      (o.refine32 == 1 && (o.precision == PDHG_FP64 || o.record_for_backward || o.persistent)))
    return fail(nullptr, PDHG_ERR_INVALID,
                "refine32 must be -1, 0 or 1 (1: precision FP32 or MIXED, no recording or persistent loop)");
  if (o.panel_overlap < -1 || o.panel_overlap > 1)
    return fail(nullptr, PDHG_ERR_INVALID, "panel_overlap must be -1, 0 or 1");
  if (o.panel_balance < -1 || o.panel_balance > 1)
    return fail(nullptr, PDHG_ERR_INVALID, "panel_balance must be -1, 0 or 1");
  if (!(o.polish_switch >= 0.0 || o.polish_switch == -1.0))
    return fail(nullptr, PDHG_ERR_INVALID, "polish_switch must be >= 0 or -1 (automatic)");

  // Checks of host inputs (CSR structure, finite data). With a GPU they run on
  // the device, on the uploaded copies, before setup reads them (on the host
  // they took ~23 ms of the 1e6 x 3e6 LP's set-up beside the upload, and
  // slowed the upload). Without one (no device or no driver), or when the
  // device set-up fails before the upload, they run on host threads, so a
  // malformed LP gets INVALID / NUMERIC whether or not a GPU is present; on
  // host threads they run beside the context's set-up: stream creation,
  // allocations and the upload depend only on the sizes, and setup reads
  // nothing it uploaded before the checks have passed, and their failure takes
  // precedence over any later error. Device inputs are checked on the device.
  auto run_checks = [=]() {
    const char* msg = "";
    pdhg_status st = check_lp(m, n, nnz, row_ptr, col_idx, val, b, c, &msg);
    if (st == PDHG_OK && ((x0 && !all_finite(x0, n)) || (y0 && !all_finite(y0, m)))) {
      st = PDHG_ERR_NUMERIC;
      msg = "NaN or Inf in the input data";
    }
    return std::make_pair(st, msg);
  };
  std::future<std::pair<pdhg_status, const char*>> checks;
  std::pair<pdhg_status, const char*> checked{PDHG_OK, ""};
  int ndev = 0;
  const bool dev_checks = !o.inputs_on_device && cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0;
  if (!o.inputs_on_device && !dev_checks) {
    try {
      checks = std::async(std::launch::async, run_checks);
    } catch (...) {  // no thread to be had: check here, before any device work
      checked = run_checks();
      if (checked.first != PDHG_OK) return fail(nullptr, checked.first, checked.second);
    }
  }
  std::function<pdhg_status()> await_checks = [&]() {
    if (checks.valid()) checked = checks.get();
    return checked.first;
  };

  pdhg_ctx* ctx = new (std::nothrow) pdhg_ctx();
  if (!ctx) {
    if (await_checks() != PDHG_OK) return fail(nullptr, checked.first, checked.second);
    return fail(nullptr, PDHG_ERR_OOM, "host allocation of the context failed");
  }
  ctx->m = m;
  ctx->n = n;
  ctx->nnz = nnz;
  ctx->opt = o;
  ctx->check_on_device = dev_checks;
  ctx->wpb = (o.step_block ? o.step_block : TPB) / 32;
  // auto: only where the matrix stream dwarfs the panels' copies of y (every
  // block copies one panel, ~H entries, per step)
  ctx->panels_on = !o.persistent && (o.primal_panels == 1 || (o.primal_panels < 0 && m >= (1 << 18) &&
                                                                nnz >= (1 << 23)));
  // PDHG_MIXED keeps a second, FP32-tuned panel layout for its FP32 phase
  ctx->pan32 = ctx->panels_on && o.precision == PDHG_MIXED;
  for (int k = 0; ctx->panels_on && k < (ctx->pan32 ? 2 : 1); ++k) {
    // panel rows: as many as fit in shared memory in the precision of the
    // layout's steps, a multiple of 16 entries, which keeps every panel's
    // start 16-byte aligned for the asynchronous copies of y
    const bool fp32_steps = k == 1 || o.precision == PDHG_FP32;
    const long long hmax = PANEL_SMEM_MAX / (fp32_steps ? 4LL : 8LL);
    const long long P0 = (m + hmax - 1) / hmax;
    const long long H = o.panel_rows > 0 ? o.panel_rows : std::min(hmax, ((m + P0 - 1) / P0 + 15) / 16 * 16);
    ctx->pan[k].pl.m = (int)m;
    ctx->pan[k].pl.rows = (int)H;
    ctx->pan[k].pl.panels = (int)((m + H - 1) / H);
  }
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    if (dev_checks) checked = run_checks();  // the input's errors come first
    const pdhg_status v = await_checks();
    pdhg_status st = v != PDHG_OK ? fail(nullptr, v, checked.second) : cuda_fail(nullptr, e, "device/stream setup");
    pdhg_destroy(ctx);
    return st;
  }
  pdhg_status st = setup(ctx, row_ptr, col_idx, val, b, c, x0, y0, await_checks);
  if (st == PDHG_OK) st = read_check(ctx);
  if (st != PDHG_OK) {
    if (await_checks() != PDHG_OK)
      st = fail(nullptr, checked.first, checked.second);
    else
      g_create_error = ctx->err;
    pdhg_destroy(ctx);
    return st;
  }
  // the per-evaluation log (off unless PDHG_LOG names a file; a file that
  // cannot be opened leaves it off)
  const char* log_path = getenv("PDHG_LOG");
  if (log_path && *log_path) ctx->log = fopen(log_path, "a");
  *out = ctx;
  return PDHG_OK;
}

void pdhg_destroy(pdhg_ctx* ctx) {
  if (!ctx) return;
  if (ctx->log) fclose(ctx->log);
  int cur = -1;
  if (cudaGetDevice(&cur) == cudaSuccess && cur != ctx->device) cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->side) cudaStreamSynchronize(ctx->side);
  for (void* p : ctx->allocs) cudaFree(p);
  for (int s = 0; s < SNAP_SLOTS; ++s) {
    if (ctx->snap_host[s]) cudaFreeHost(ctx->snap_host[s]);
    if (ctx->snap_packed[s]) cudaEventDestroy(ctx->snap_packed[s]);
    if (ctx->snap_done[s]) cudaEventDestroy(ctx->snap_done[s]);
  }
  for (int i = 0; i < 3 * EV_POOL; ++i)
    if (ctx->ev[i]) cudaEventDestroy(ctx->ev[i]);
  for (int g = 0; g < 2; ++g)
    if (ctx->graph_exec[g]) cudaGraphExecDestroy(ctx->graph_exec[g]);
  if (ctx->bgraph) cudaGraphExecDestroy(ctx->bgraph);
  if (ctx->h_bctl) cudaFreeHost(ctx->h_bctl);
  if (ctx->h_st) cudaFreeHost(ctx->h_st);
  if (ctx->h_kkt) cudaFreeHost(ctx->h_kkt);
  if (ctx->side) cudaStreamDestroy(ctx->side);
  if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

static pdhg_status iterate_impl(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done);

// One JSON line per evaluation (PDHG_LOG): the evaluation's candidate on the
// problem as given - Section 2's relative residuals and gap, their maximum -
// and the decisions taken there, from the state copy the host reads anyway.
void log_evaluation(pdhg_ctx* ctx) {
  const DevState& h = *ctx->h_st;
  const EvalSums& e = h.candidate == KIND_AVG ? h.avg : h.cur;
  const double cx = e.q[Q_CX], by = e.q[Q_BY];
  const double rel_p = sqrt(e.q[Q_RP2U]) / (1.0 + h.b_norm);
  const double rel_d = sqrt(e.q[Q_RD2U]) / (1.0 + h.c_norm);
  const double rel_g = fabs(cx - by) / (1.0 + fabs(cx) + fabs(by));
  const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - ctx->t_create).count();
  static const char* const kinds[] = {"none", "current", "average", "step"};
  static const char* const applies[] = {"none", "restart_current", "restart_average", "take_average",
                                        "restart_step"};
  fprintf(ctx->log,
          "{\"iteration\": %lld, \"rel_p\": %.17g, \"rel_d\": %.17g, \"rel_gap\": %.17g, \"rel_kkt\": %.17g, "
          "\"primal_obj\": %.17g, \"dual_obj\": %.17g, \"candidate\": \"%s\", \"restart\": \"%s\", "
          "\"restarts\": %lld, \"omega\": %.17g, \"precision\": \"%s\", \"converged\": %d, "
          "\"elapsed_s\": %.6f}\n",
          (long long)h.k, rel_p, rel_d, rel_g, h.cand_rel_kkt, cx, by,
          kinds[h.candidate >= 0 && h.candidate <= 3 ? h.candidate : 0],
          applies[h.apply_mode >= 0 && h.apply_mode <= 4 ? h.apply_mode : 0], (long long)h.restarts, h.omega,
          ctx->phase32 ? "fp32" : "fp64", h.converged, sec);
  fflush(ctx->log);
}

pdhg_status pdhg_iterate(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done) {
  Range nvtx_range("pdhg/iterate");
  pdhg_status rs = iterate_impl(ctx, max_iters, tol, iters_done);
  if (ctx && (rs == PDHG_OK || rs == PDHG_ERR_NOT_CONVERGED)) {
    const pdhg_status cs = read_check(ctx);  // checked build only
    if (cs != PDHG_OK) return cs;
  }
  return rs;
}

static pdhg_status iterate_impl(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done) {
  if (iters_done) *iters_done = 0;
  if (!ctx) return PDHG_ERR_INVALID;
  if (max_iters < 0 || !(tol >= 0.0)) return fail(ctx, PDHG_ERR_INVALID, "max_iters < 0 or tol < 0");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  if (ctx->opt.persistent == 2) return iterate_batch_coop(ctx, max_iters, tol, iters_done);
  if (ctx->opt.persistent) return iterate_persistent(ctx, max_iters, tol, iters_done);
  if (ctx->count > 1) return iterate_batch(ctx, max_iters, tol, iters_done);
  const pdhg_options& o = ctx->opt;
  const bool evaluating = o.restarts || tol > 0.0 || o.eps_cross > 0.0 || o.snapshot_every > 0;
  const int n = (int)ctx->n, m = (int)ctx->m;
  cudaStream_t s = ctx->stream;
  CK(ctx, cudaMemcpyAsync(&ctx->st->tol, &tol, sizeof(double), cudaMemcpyHostToDevice, s));
  const bool graphs = o.use_graphs && evaluating && !o.kernel_timing && !o.record_for_backward;
  ctx->converged = false;
  int64_t done = 0;
  while (done < max_iters) {
    int64_t nb;
    if (evaluating)
      nb = std::min<int64_t>(o.eval_every - (ctx->k % o.eval_every), max_iters - done);
    else
      nb = std::min<int64_t>(max_iters - done, o.kernel_timing ? EV_POOL : (1 << 20));
    const bool timing = o.kernel_timing && nb <= EV_POOL;
    const bool eval_now = evaluating && (ctx->k + nb) % o.eval_every == 0;
    if (graphs && eval_now && nb == o.eval_every) {
      rs = run_block_graph(ctx, nb);
    } else {
      rs = enqueue_steps(ctx, nb, timing);
      if (rs == PDHG_OK && eval_now) rs = enqueue_eval(ctx);
    }
    if (rs != PDHG_OK) return rs;
    ctx->k += nb;
    done += nb;
    if (timing) {
      CK(ctx, cudaEventSynchronize(ctx->ev[3 * (nb - 1) + 2]));
      for (int64_t it = 0; it < nb; ++it) {
        float a = 0.f, bms = 0.f;
        CK(ctx, cudaEventElapsedTime(&a, ctx->ev[3 * it], ctx->ev[3 * it + 1]));
        CK(ctx, cudaEventElapsedTime(&bms, ctx->ev[3 * it + 1], ctx->ev[3 * it + 2]));
        ctx->ms_primal += a;
        ctx->ms_dual += bms;
      }
      ctx->launches_primal += nb;
      ctx->launches_dual += nb;
    }
    if (eval_now) {
      CK(ctx, cudaStreamSynchronize(s));  // the state copy of the evaluation has landed
      if (ctx->h_st->wait_err) {
        if (iters_done) *iters_done = done;
        return fail(ctx, PDHG_ERR_TIMEOUT, "a bounded wait of a streamed step kernel ran out");
      }
      if (ctx->h_st->numeric) {
        if (iters_done) *iters_done = done;
        return fail(ctx, PDHG_ERR_NUMERIC, "NaN or Inf in the iterates");
      }
      if (ctx->log) log_evaluation(ctx);
      if (ctx->h_st->snapshot_flag) {
        rs = take_snapshot(ctx);
        if (rs != PDHG_OK) return rs;
        ctx->launches += 2;
      }
      if (ctx->h_st->converged) {
        ctx->converged = true;
        break;
      }
      if (o.feas_polish && tol > 0.0 && !ctx->phase32 && ctx->k >= ctx->fp_next &&
          ctx->h_st->cand_rel_gap <= (o.gap_tol > 0.0 ? o.gap_tol : tol)) {
        // feasibility polishing; the next attempt once the iteration count has doubled
        ctx->fp_next = 2 * ctx->k;
        const int64_t per = (int64_t)o.polish_div * o.eval_every;
        const int64_t budget = o.eval_every * std::max<int64_t>(1, (ctx->k + per - 1) / per);
        bool solved = false;
        rs = feas_polish(ctx, tol, budget, graphs, &solved);
        if (rs != PDHG_OK) return rs;
        if (solved) {
          ctx->converged = true;
          break;
        }
      }
      bool stalled = false;
      if (ctx->phase32) {
        // FP32 stall: the best relative KKT of the FP32 phase has not
        // improved by 10% over the last STALL_ITERS iterations
        const double r = ctx->h_st->cand_rel_kkt;
        if (r < 0.9 * ctx->best32) {
          ctx->best32 = r;
          ctx->best32_k = ctx->k;
        }
        stalled = ctx->k - ctx->best32_k >= (ctx->refine ? STALL_ITERS_REFINED : STALL_ITERS);
      }
      const double pswitch = o.polish_switch >= 0.0 ? o.polish_switch : (ctx->refine ? 0.0 : 1e-5);
      if (ctx->phase32 && o.precision == PDHG_MIXED && (ctx->h_st->cand_rel_kkt <= pswitch || stalled)) {
        // FP64 polishing phase: continue in FP64 from the FP32 iterate (held
        // exactly in x, y), keeping D_r, D_c, eta and omega.
        if (!o.halpern) {
          // PDLP-style restarts: the same restart epoch goes on - the
          // restart reference (xr, yr, its norms) and the count since the
          // last restart stay, and the running sums carry over from FP32 -
          // so the switch is no restart (one would drop the average)
          if (ctx->refine) {  // sums of corrections: t terms of the reference each
            launch_widen_sum_delta(ctx->xsum, ctx->xr, ctx->xsum32, n, ctx->st, vec_grid(ctx, n), s);
            launch_widen_sum_delta(ctx->ysum, ctx->yr, ctx->ysum32, m, ctx->st, vec_grid(ctx, m), s);
          } else {
            launch_widen(ctx->xsum, ctx->xsum32, n, vec_grid(ctx, n), s);
            launch_widen(ctx->ysum, ctx->ysum32, m, vec_grid(ctx, m), s);
          }
          ctx->launches += 2;
        } else {
          // reflected Halpern forms: the iterate becomes the anchor and the
          // restart reference, and the Halpern count starts over
          if (o.restart_scheme == 1)
            eval_point_fp(ctx, &ctx->st->cur);  // the fixed-point residual at the switch
          else
            eval_point(ctx, ctx->x, ctx->y, nullptr, nullptr, &ctx->st->cur);
          launch_promote_state(ctx->st, s);
          CK(ctx, cudaMemcpyAsync(ctx->xr, ctx->x, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
          CK(ctx, cudaMemcpyAsync(ctx->yr, ctx->y, sizeof(double) * m, cudaMemcpyDeviceToDevice, s));
          ctx->launches += 2;
        }
        CK(ctx, cudaGetLastError());
        ctx->phase32 = false;
        ctx->promoted_at = ctx->k;
      }
    }
  }
  if (ctx->stream_on) {  // a bounded wait that ran out after the last evaluation
    unsigned werr = 0;
    CK(ctx, cudaMemcpyAsync(&werr, &ctx->st->wait_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(ctx, cudaStreamSynchronize(s));
    if (werr) {
      if (iters_done) *iters_done = done;
      return fail(ctx, PDHG_ERR_TIMEOUT, "a bounded wait of a streamed step kernel ran out");
    }
  }
  CK(ctx, cudaStreamSynchronize(s));
  if (iters_done) *iters_done = done;
  if (ctx->converged || tol == 0.0) return PDHG_OK;
  return fail(ctx, PDHG_ERR_NOT_CONVERGED, "iteration limit reached before the tolerance");
}

pdhg_status pdhg_kkt(pdhg_ctx* ctx, int which, pdhg_kkt_info* out) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (ctx->count > 1) return fail(ctx, PDHG_ERR_STATE, "batch context: use pdhg_batch_info");
  if (!out) return fail(ctx, PDHG_ERR_INVALID, "out is NULL");
  if (which < PDHG_CURRENT || which > PDHG_LAST_RESTART) return fail(ctx, PDHG_ERR_INVALID, "bad point selector");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  const double *px, *py;
  point_of(ctx, which, &px, &py);
  eval_point(ctx, px, py, nullptr, nullptr, ctx->kkt_sums);
  CK(ctx, cudaGetLastError());
  CK(ctx, cudaMemcpyAsync(ctx->h_kkt, ctx->kkt_sums, sizeof(EvalSums), cudaMemcpyDeviceToHost, ctx->stream));
  rs = read_state(ctx);
  if (rs != PDHG_OK) return rs;
  const double* q = ctx->h_kkt->q;
  out->rp_norm2 = sqrt(q[Q_RP2U]);
  out->rp_norminf = q[Q_RPINF];
  out->rd_norm2 = sqrt(q[Q_RD2U]);
  out->rd_norminf = q[Q_RDINF];
  out->primal_obj = q[Q_CX];
  out->dual_obj = q[Q_BY];
  out->gap = fabs(q[Q_CX] - q[Q_BY]);
  out->complementarity = q[Q_XZ];
  out->rel_p = out->rp_norm2 / (1.0 + ctx->h_st->b_norm);
  out->rel_d = out->rd_norm2 / (1.0 + ctx->h_st->c_norm);
  out->rel_gap = out->gap / (1.0 + fabs(out->primal_obj) + fabs(out->dual_obj));
  out->rel_kkt = max3_nan(out->rel_p, out->rel_d, out->rel_gap);
  out->iteration = ctx->h_st->k;
  return PDHG_OK;
}

pdhg_status pdhg_get_solution(pdhg_ctx* ctx, int which, double* x, double* y, double* z, int on_device) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (ctx->count > 1) return fail(ctx, PDHG_ERR_STATE, "batch context: use pdhg_batch_solution");
  if (which < PDHG_CURRENT || which > PDHG_LAST_RESTART) return fail(ctx, PDHG_ERR_INVALID, "bad point selector");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  const double *px, *py;
  point_of(ctx, which, &px, &py);
  double* ox = ctx->sol;
  double* oy = ctx->sol + ctx->n;
  double* oz = ctx->sol + ctx->n + ctx->m;
  launch_pack_solution(ctx->At, ctx->perm_x, ctx->perm_y, px, py, ctx->ch, ctx->dc, ctx->dr, x ? ox : nullptr,
                       y ? oy : nullptr, z ? oz : nullptr, stride_grid(ctx, ctx->At), ctx->stream);
  CK(ctx, cudaGetLastError());
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (x) CK(ctx, cudaMemcpyAsync(x, ox, sizeof(double) * ctx->n, kind, ctx->stream));
  if (y) CK(ctx, cudaMemcpyAsync(y, oy, sizeof(double) * ctx->m, kind, ctx->stream));
  if (z) CK(ctx, cudaMemcpyAsync(z, oz, sizeof(double) * ctx->n, kind, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

pdhg_status pdhg_snapshot_poll(pdhg_ctx* ctx, int64_t* count, int* ready) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (count) *count = ctx->snap_count;
  if (ready) {
    *ready = 0;
    if (ctx->snap_count > 0) {
      cudaError_t e = cudaEventQuery(ctx->snap_done[(ctx->snap_count - 1) % SNAP_SLOTS]);
      if (e == cudaSuccess)
        *ready = 1;
      else if (e != cudaErrorNotReady)
        return cuda_fail(ctx, e, "cudaEventQuery");
    }
  }
  return PDHG_OK;
}

pdhg_status pdhg_snapshot(pdhg_ctx* ctx, double* x, double* y, double* z, int64_t* iteration, double* rel_kkt) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (ctx->snap_count == 0) return fail(ctx, PDHG_ERR_STATE, "no snapshot has been taken");
  const int slot = (int)((ctx->snap_count - 1) % SNAP_SLOTS);
  CK(ctx, cudaEventSynchronize(ctx->snap_done[slot]));
  const double* h = ctx->snap_host[slot];
  if (x) memcpy(x, h, sizeof(double) * ctx->n);
  if (y) memcpy(y, h + ctx->n, sizeof(double) * ctx->m);
  if (z) memcpy(z, h + ctx->n + ctx->m, sizeof(double) * ctx->n);
  if (iteration) *iteration = ctx->snap_iter[slot];
  if (rel_kkt) *rel_kkt = ctx->snap_rel[slot];
  return PDHG_OK;
}

pdhg_status pdhg_snapshot_wait(pdhg_ctx* ctx, int64_t after, int64_t timeout_ms, double* x, double* y, double* z,
                               int64_t* index, int64_t* iteration, double* rel_kkt) {
  if (!ctx || after < 0 || timeout_ms < 0) return PDHG_ERR_INVALID;
  int slot = -1;
  int64_t seq = 0;
  {
    std::unique_lock<std::mutex> lk(ctx->snap_mu);
    // the slot of the newest complete snapshot numbered above `after`. A slot
    // being rewritten holds 0, so when the newest complete snapshot's slot is
    // reused before its successors land, this waits for a successor.
    auto newest = [&] {
      slot = -1;
      for (int s = 0; s < SNAP_SLOTS; ++s)
        if (ctx->snap_seq[s] > after && (slot < 0 || ctx->snap_seq[s] > ctx->snap_seq[slot])) slot = s;
      return slot >= 0;
    };
    if (!ctx->snap_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), newest)) return PDHG_ERR_TIMEOUT;
    seq = ctx->snap_seq[slot];
    ctx->snap_readers[slot] += 1;
  }
  const double* h = ctx->snap_host[slot];
  if (x) memcpy(x, h, sizeof(double) * ctx->n);
  if (y) memcpy(y, h + ctx->n, sizeof(double) * ctx->m);
  if (z) memcpy(z, h + ctx->n + ctx->m, sizeof(double) * ctx->n);
  if (iteration) *iteration = ctx->snap_iter[slot];
  if (rel_kkt) *rel_kkt = ctx->snap_rel[slot];
  if (index) *index = seq;
  {
    std::lock_guard<std::mutex> lk(ctx->snap_mu);
    ctx->snap_readers[slot] -= 1;
  }
  ctx->snap_cv.notify_all();
  return PDHG_OK;
}

pdhg_status pdhg_get_info(pdhg_ctx* ctx, pdhg_info* out) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (!out) return fail(ctx, PDHG_ERR_INVALID, "out is NULL");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  rs = read_state(ctx);
  if (rs != PDHG_OK) return rs;
  const DevState& h = *ctx->h_st;
  memset(out, 0, sizeof(*out));
  out->norm_estimate = h.norm_est;
  out->eta = h.eta;
  out->omega = h.omega;
  out->tau = h.tau;
  out->sigma = h.sigma;
  out->iterations = h.k;
  out->since_restart = h.t;
  out->restarts = h.restarts;
  out->evaluations = h.evals;
  out->snapshots = ctx->snap_count;
  out->last_rel_kkt = h.cand_rel_kkt;
  out->precision_now = ctx->phase32 ? PDHG_FP32 : PDHG_FP64;
  out->polish_started_at = ctx->promoted_at;
  out->converged = ctx->converged ? 1 : 0;
  out->kernel_ms_primal = ctx->ms_primal;
  out->kernel_ms_dual = ctx->ms_dual;
  out->kernel_launches_primal = ctx->launches_primal;
  out->kernel_launches_dual = ctx->launches_dual;
  out->kernel_launches = ctx->launches;
  out->feas_polish_attempts = (int64_t)ctx->fp_log.size();
  out->feas_polish_iterations = ctx->fp_iters;
  out->feas_polished = ctx->fp_polished ? 1 : 0;
  out->persistent_grid = ctx->bgrid;
  out->graph_launches = ctx->graph_replays;
  out->values32 = ctx->vals_u ? 1 : 0;
  out->stream_steps = ctx->stream_on ? 1 : 0;
  out->refine32 = ctx->refine ? 1 : 0;
  out->panels = !ctx->panels_on ? 0 : ctx->pan[ctx->phase32 && ctx->pan32 ? 1 : 0].pl.panels;
  return PDHG_OK;
}

pdhg_status pdhg_get_polish_log(pdhg_ctx* ctx, pdhg_polish_rec* recs, int64_t cap, int64_t* count) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (cap < 0 || (cap > 0 && !recs)) return fail(ctx, PDHG_ERR_INVALID, "bad record buffer");
  const int64_t total = (int64_t)ctx->fp_log.size();
  for (int64_t i = 0; i < std::min(cap, total); ++i) recs[i] = ctx->fp_log[i];
  if (count) *count = total;
  return PDHG_OK;
}

pdhg_status pdhg_get_trace(pdhg_ctx* ctx, pdhg_trace_rec* recs, int64_t cap, int64_t* count) {
  if (!ctx) return PDHG_ERR_INVALID;
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  rs = read_state(ctx);
  if (rs != PDHG_OK) return rs;
  const int64_t stored = std::min<int64_t>(ctx->h_st->evals, TRACE_CAP);
  const int64_t k = std::min<int64_t>(stored, cap < 0 ? 0 : cap);
  if (count) *count = stored;
  if (k > 0 && recs) {
    static_assert(sizeof(TraceRec) == sizeof(pdhg_trace_rec), "trace record layout");
    CK(ctx, cudaMemcpy(recs, ctx->trace, sizeof(TraceRec) * k, cudaMemcpyDeviceToHost));
  }
  return PDHG_OK;
}

pdhg_status pdhg_backward(pdhg_ctx* ctx, const double* dL_dxK, const double* dL_dyK, double* dL_dc, double* dL_db,
                          int on_device) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (!ctx->opt.record_for_backward)
    return fail(ctx, PDHG_ERR_STATE, "the context was not created with record_for_backward = 1");
  if (!dL_dxK || !dL_dc || !dL_db) return fail(ctx, PDHG_ERR_INVALID, "NULL argument");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  cudaStream_t s = ctx->stream;
  const int64_t n = ctx->n, m = ctx->m;
  // inputs into device scratch (tmp_n, tmp_m), outputs through sol
  const cudaMemcpyKind in_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(ctx, cudaMemcpyAsync(ctx->tmp_n, dL_dxK, sizeof(double) * n, in_kind, s));
  if (dL_dyK) CK(ctx, cudaMemcpyAsync(ctx->tmp_m, dL_dyK, sizeof(double) * m, in_kind, s));
  double* out_c = ctx->sol;
  double* out_b = ctx->sol + n;
  rs = ctx->opt.precision == PDHG_FP32
           ? backward_impl<float>(ctx, ctx->tmp_n, dL_dyK ? ctx->tmp_m : nullptr, out_c, out_b)
           : backward_impl<double>(ctx, ctx->tmp_n, dL_dyK ? ctx->tmp_m : nullptr, out_c, out_b);
  if (rs != PDHG_OK) return rs;
  const cudaMemcpyKind out_kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CK(ctx, cudaMemcpyAsync(dL_dc, out_c, sizeof(double) * n, out_kind, s));
  CK(ctx, cudaMemcpyAsync(dL_db, out_b, sizeof(double) * m, out_kind, s));
  CK(ctx, cudaStreamSynchronize(s));
  return PDHG_OK;
}

pdhg_status pdhg_create_batch(int count, const pdhg_lp_desc* lps, const pdhg_options* opt, void* cuda_stream,
                              pdhg_ctx** out) {
  if (!out) return fail(nullptr, PDHG_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (count < 1 || !lps) return fail(nullptr, PDHG_ERR_INVALID, "count < 1 or lps is NULL");
  pdhg_options o;
  if (opt)
    o = *opt;
  else
    pdhg_default_options(&o);
  if (o.precision != PDHG_FP64 || o.record_for_backward || o.inputs_on_device || o.dual_hot_cols ||
      o.eval_every < 1 || o.ruiz_iters < 0 || o.power_iters < 1 || !(o.step_factor > 0.0) || o.long_row_min < 1 ||
      !(o.rows_per_thread == 1 || o.rows_per_thread == 2 || o.rows_per_thread == 4) || o.snapshot_every < 0 ||
      o.eps_cross < 0.0 || !(o.eps_factor > 0.0 && o.eps_factor < 1.0))
    return fail(nullptr, PDHG_ERR_INVALID,
                "batch: FP64, host inputs, no recording, no shared-memory hot columns, valid options");
  if (o.persistent == 1 && (o.eps_cross > 0.0 || o.snapshot_every > 0))
    return fail(nullptr, PDHG_ERR_INVALID, "batch snapshots need persistent = 0 or 2");
  if (!(o.step_block == 0 || o.step_block == 128 || o.step_block == 256 || o.step_block == 512))
    return fail(nullptr, PDHG_ERR_INVALID, "step_block must be 128, 256 or 512");
  if (o.primal_panels == 1)
    return fail(nullptr, PDHG_ERR_INVALID, "primal_panels = 1 is for single LPs (batches use the direct primal step)");
  if (o.halpern && (o.persistent == 1 || !(o.halpern_reflect >= 0.0) || !(o.halpern_reflect <= 1.0)))
    return fail(nullptr, PDHG_ERR_INVALID,
                "halpern = 1 needs halpern_reflect in [0, 1] and no single-block loop (persistent = 1)");
  if (o.persistent < 0 || o.persistent > 2 || (o.persistent && o.kernel_timing) || o.barrier_cycles < 0)
    return fail(nullptr, PDHG_ERR_INVALID,
                "persistent must be 0, 1 or 2 and excludes kernel timing; barrier_cycles must be >= 0");
  if (o.feas_polish || !(o.gap_tol >= 0.0) || o.restart_scheme != 0 || o.values32 == 1 || o.values32 < -1 ||
      o.stream_steps || o.refine32 == 1)
    return fail(nullptr, PDHG_ERR_INVALID,
                "batch: no feasibility polishing, fixed-point restart scheme, values32 or stream_steps (single LPs "
                "only), gap_tol >= 0");
  int64_t mt = 0, nt = 0, zt = 0;
  for (int i = 0; i < count; ++i) {
    const pdhg_lp_desc& L = lps[i];
    pdhg_status vs = validate_lp(L.m, L.n, L.nnz, L.row_ptr, L.col_idx, L.val, L.b, L.c);
    if (vs != PDHG_OK) {
      g_create_error = "instance " + std::to_string(i) + ": " + g_create_error;
      return vs;
    }
    mt += L.m;
    nt += L.n;
    zt += L.nnz;
    if (o.persistent == 1 && 7 * L.n + 6 * L.m > PERSIST_MAX_DOUBLES)
      return fail(nullptr, PDHG_ERR_INVALID,
                  "persistent: the vectors of instance " + std::to_string(i) +
                      " (7n + 6m doubles) exceed one block's shared memory (28672)");
  }
  if (mt >= (1LL << 31) - 1 || nt >= (1LL << 31) - 1 || zt >= (1LL << 31) - 1)
    return fail(nullptr, PDHG_ERR_INVALID, "batch totals of m, n and nnz must be below 2^31 - 1");
  pdhg_ctx* ctx = new (std::nothrow) pdhg_ctx();
  if (!ctx) return fail(nullptr, PDHG_ERR_OOM, "host allocation of the context failed");
  ctx->m = mt;
  ctx->n = nt;
  ctx->nnz = zt;
  ctx->opt = o;
  ctx->wpb = (o.step_block ? o.step_block : TPB) / 32;
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      ctx->stream = (cudaStream_t)cuda_stream;
    } else {
      e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
      ctx->own_stream = true;
    }
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    pdhg_status st = cuda_fail(nullptr, e, "device/stream setup");
    pdhg_destroy(ctx);
    return st;
  }
  pdhg_status st = setup_batch(ctx, count, lps);
  if (st == PDHG_OK) st = read_check(ctx);
  if (st != PDHG_OK) {
    g_create_error = ctx->err;
    pdhg_destroy(ctx);
    return st;
  }
  *out = ctx;
  return PDHG_OK;
}

pdhg_status pdhg_batch_info(pdhg_ctx* ctx, int64_t* iterations, int* converged, double* rel_kkt, int64_t* restarts) {
  if (!ctx) return PDHG_ERR_INVALID;
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  CK(ctx, cudaMemcpyAsync(ctx->h_st, ctx->st, sizeof(DevState) * ctx->count, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  for (int i = 0; i < ctx->count; ++i) {
    const DevState& h = ctx->h_st[i];
    if (iterations) iterations[i] = h.k;
    if (converged) converged[i] = ctx->count > 1 ? h.frozen : (ctx->converged ? 1 : 0);
    if (rel_kkt) rel_kkt[i] = h.cand_rel_kkt;
    if (restarts) restarts[i] = h.restarts;
  }
  return PDHG_OK;
}

pdhg_status pdhg_batch_kkt(pdhg_ctx* ctx, int instance, int which, pdhg_kkt_info* out) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (!out) return fail(ctx, PDHG_ERR_INVALID, "out is NULL");
  if (instance < 0 || instance >= ctx->count) return fail(ctx, PDHG_ERR_INVALID, "instance out of range");
  if (which < PDHG_CURRENT || which > PDHG_LAST_RESTART) return fail(ctx, PDHG_ERR_INVALID, "bad point selector");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  if (ctx->count == 1) return pdhg_kkt(ctx, which, out);
  const double* px = which == PDHG_AVERAGE ? ctx->xavg : (which == PDHG_LAST_RESTART ? ctx->xr : ctx->x);
  const double* py = which == PDHG_AVERAGE ? ctx->yavg : (which == PDHG_LAST_RESTART ? ctx->yr : ctx->y);
  // the instance's units form a contiguous range of both layouts (whole blocks)
  const int b0 = ctx->bstart_h[instance], nb = ctx->bstart_h[instance + 1] - b0;
  Hyb Ai = ctx->A, Ti = ctx->At;
  for (Hyb* H : {&Ai, &Ti}) {
    H->uoff += (size_t)b0 * ctx->wpb;
    H->uinfo += (size_t)b0 * ctx->wpb;
    H->n_units = nb * ctx->wpb;
  }
  cudaStream_t s = ctx->stream;
  launch_eval_point(Ai, Ti, px, py, ctx->bh, ctx->ch, ctx->idr, ctx->idc, nullptr, nullptr, ctx->partials, nb, s,
                    nullptr, nullptr, 32 * ctx->wpb);
  launch_eval_finalize(ctx->partials, nb, ctx->kkt_sums, s);
  CK(ctx, cudaGetLastError());
  CK(ctx, cudaMemcpyAsync(ctx->h_kkt, ctx->kkt_sums, sizeof(EvalSums), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaMemcpyAsync(ctx->h_st + instance, ctx->st + instance, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(ctx, cudaStreamSynchronize(s));
  const double* q = ctx->h_kkt->q;
  const DevState& h = ctx->h_st[instance];
  out->rp_norm2 = sqrt(q[Q_RP2U]);
  out->rp_norminf = q[Q_RPINF];
  out->rd_norm2 = sqrt(q[Q_RD2U]);
  out->rd_norminf = q[Q_RDINF];
  out->primal_obj = q[Q_CX];
  out->dual_obj = q[Q_BY];
  out->gap = fabs(q[Q_CX] - q[Q_BY]);
  out->complementarity = q[Q_XZ];
  out->rel_p = out->rp_norm2 / (1.0 + h.b_norm);
  out->rel_d = out->rd_norm2 / (1.0 + h.c_norm);
  out->rel_gap = out->gap / (1.0 + fabs(out->primal_obj) + fabs(out->dual_obj));
  out->rel_kkt = max3_nan(out->rel_p, out->rel_d, out->rel_gap);
  out->iteration = h.k;
  return PDHG_OK;
}

pdhg_status pdhg_batch_solution(pdhg_ctx* ctx, int instance, double* x, double* y, double* z) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (instance < 0 || instance >= ctx->count) return fail(ctx, PDHG_ERR_INVALID, "instance out of range");
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  double* ox = ctx->sol;
  double* oy = ctx->sol + ctx->n;
  double* oz = ctx->sol + ctx->n + ctx->m;
  launch_pack_solution(ctx->At, ctx->perm_x, ctx->perm_y, ctx->x, ctx->y, ctx->ch, ctx->dc, ctx->dr, ox, oy, oz,
                       stride_grid(ctx, ctx->At), ctx->stream);
  CK(ctx, cudaGetLastError());
  const int x0 = ctx->count > 1 ? ctx->xoff_h[instance] : 0;
  const int y0 = ctx->count > 1 ? ctx->yoff_h[instance] : 0;
  const int64_t ni = ctx->count > 1 ? ctx->xoff_h[instance + 1] - x0 : ctx->n;
  const int64_t mi = ctx->count > 1 ? ctx->yoff_h[instance + 1] - y0 : ctx->m;
  if (x) CK(ctx, cudaMemcpyAsync(x, ox + x0, sizeof(double) * ni, cudaMemcpyDeviceToHost, ctx->stream));
  if (y) CK(ctx, cudaMemcpyAsync(y, oy + y0, sizeof(double) * mi, cudaMemcpyDeviceToHost, ctx->stream));
  if (z) CK(ctx, cudaMemcpyAsync(z, oz + x0, sizeof(double) * ni, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return PDHG_OK;
}

pdhg_status pdhg_snapshot_i(pdhg_ctx* ctx, int instance, double* x, double* y, double* z, int64_t* iteration,
                            double* rel_kkt, int64_t* count) {
  if (!ctx) return PDHG_ERR_INVALID;
  if (instance < 0 || instance >= ctx->count) return fail(ctx, PDHG_ERR_INVALID, "instance out of range");
  if (ctx->count == 1) {
    if (count) {
      pdhg_status rs = pdhg_snapshot_poll(ctx, count, nullptr);
      if (rs != PDHG_OK) return rs;
    }
    return pdhg_snapshot(ctx, x, y, z, iteration, rel_kkt);
  }
  pdhg_status rs = set_device(ctx);
  if (rs != PDHG_OK) return rs;
  if (!ctx->bsnap) return fail(ctx, PDHG_ERR_STATE, "no snapshot schedule (eps_cross, snapshot_every) was set");
  CK(ctx, cudaMemcpyAsync(ctx->h_st + instance, ctx->st + instance, sizeof(DevState), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  const DevState& h = ctx->h_st[instance];
  if (count) *count = h.snapshots;
  if (h.snapshots == 0) return fail(ctx, PDHG_ERR_STATE, "instance has no snapshot yet");
  const int x0 = ctx->xoff_h[instance], y0 = ctx->yoff_h[instance];
  const int64_t ni = ctx->xoff_h[instance + 1] - x0, mi = ctx->yoff_h[instance + 1] - y0;
  const double* b = ctx->bsnap;
  if (x) CK(ctx, cudaMemcpyAsync(x, b + x0, sizeof(double) * ni, cudaMemcpyDeviceToHost, ctx->stream));
  if (y) CK(ctx, cudaMemcpyAsync(y, b + ctx->n + y0, sizeof(double) * mi, cudaMemcpyDeviceToHost, ctx->stream));
  if (z)
    CK(ctx, cudaMemcpyAsync(z, b + ctx->n + ctx->m + x0, sizeof(double) * ni, cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (iteration) *iteration = h.snap_k;
  if (rel_kkt) *rel_kkt = h.snap_rel;
  return PDHG_OK;
}

const char* pdhg_last_error(const pdhg_ctx* ctx) { return ctx ? ctx->err.c_str() : g_create_error.c_str(); }

}  // extern "C"
