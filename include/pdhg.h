/*
 * pdhg.h - C ABI of the B300 (sm_103a) PDHG engine for the standard-form LP
 *
 *     min c^T x   s.t.  A x = b,  x >= 0        (primal)
 *     max b^T y   s.t.  A^T y + z = c,  z >= 0  (dual)
 *
 * as stated in Section 2 ("Background") of "Concurrent Crossover for PDHG"
 * (Rothberg, 2025). The engine runs the PDLP-style PDHG iteration on one GPU
 * (the "Perform PDHG iteration" step of Algorithm 1, Section 3.1), reports the
 * residuals r_P = b - A x and r_D = A^T y + z - c, the objective gap and
 * complementarity (Section 2), and hands out snapshot iterates (x, y, z) at the
 * points where Algorithm 1 would launch a crossover thread (Section 3.1).
 *
 * General rules for every call:
 *   - Every call returns a pdhg_status; nothing aborts, traps or exits.
 *     pdhg_last_error() gives a one-line description of the last failure.
 *     A NULL context gives PDHG_ERR_INVALID (with no message). A failed CUDA
 *     call gives PDHG_ERR_CUDA, or PDHG_ERR_OOM for a failed allocation; its
 *     message names the call. Host-side checks run before any device work, so
 *     a call that fails them leaves the context unchanged.
 *   - A pdhg_ctx is not thread-safe: one host thread at a time per context.
 *     Different contexts are independent.
 *   - Pointers passed in are borrowed for the duration of the call only; the
 *     library copies what it keeps. Output buffers are owned by the caller.
 *   - Matrices are CSR with rows = constraints, 0-based, column indices strictly
 *     increasing within each row (so no duplicates). Sizes: 1 <= m, n < 2^31,
 *     0 <= nnz < 2^31.
 *   - Vectors are dense float64 arrays: x, c, z have length n; y, b length m.
 *   - The CUDA stream argument is a cudaStream_t (for example
 *     torch.cuda.current_stream().cuda_stream) or NULL for a stream the library
 *     creates. All device work of the context is ordered on that stream.
 */
#ifndef PDHG_H
#define PDHG_H

#include <stdint.h>

#if defined(__GNUC__)
#define PDHG_API __attribute__((visibility("default")))
#else
#define PDHG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pdhg_ctx pdhg_ctx;

typedef enum {
  PDHG_OK = 0,
  PDHG_ERR_INVALID = 1,       /* bad argument or malformed CSR */
  PDHG_ERR_CUDA = 2,          /* a CUDA runtime call failed */
  PDHG_ERR_OOM = 3,           /* device or pinned host allocation failed */
  PDHG_ERR_TIMEOUT = 4,       /* a bounded device wait gave up */
  PDHG_ERR_NUMERIC = 5,       /* NaN or Inf in the data or in the iterates */
  PDHG_ERR_STATE = 6,         /* call not valid in the context's state */
  PDHG_ERR_NOT_CONVERGED = 7  /* iteration limit reached before the tolerance */
} pdhg_status;

/* arithmetic of the iteration */
enum { PDHG_FP64 = 0, PDHG_FP32 = 1, PDHG_MIXED = 2 };

/* which point pdhg_kkt / pdhg_get_solution look at */
enum { PDHG_CURRENT = 0, PDHG_AVERAGE = 1, PDHG_LAST_RESTART = 2 };

/* restart kinds in the evaluation trace (PDHG_RESTART_TO_PDHG_STEP: the
 * fixed-point residual scheme's restart at T(z) of the current point) */
enum { PDHG_NO_RESTART = 0, PDHG_RESTART_TO_CURRENT = 1, PDHG_RESTART_TO_AVERAGE = 2, PDHG_RESTART_TO_PDHG_STEP = 3 };

/* Options (pdhg_default_options gives the values in parentheses). Scaling,
 * step size, restarts and the primal weight follow the PDLP line of work that
 * the paper's solver follows (Section 1, Section 4.1). The paper fixes none of
 * them, so they and their defaults (PDLP's published ones) are readings.
 * eps_cross and eps_factor are Algorithm 1's snapshot thresholds (Section 3.1).
 * feas_polish and gap_tol follow Section 5 and Section 2. The other options
 * choose the engine's form (precision, layout, launch shape, recording); the
 * paper has no counterpart for them. */
typedef struct {
  int precision;          /* PDHG_FP64 (default); PDHG_FP32: both half-steps in FP32 (matrix values,
                             vectors, accumulation) with FP64 evaluation and restart decisions;
                             PDHG_MIXED: as PDHG_FP32 (on corrections to an FP64 restart point, see
                             refine32) until rel. KKT <= polish_switch or the FP32 phase stalls, then FP64 */
  int ruiz_iters;         /* Ruiz equilibration passes (10) */
  int pock_chambolle;     /* 1: one Pock-Chambolle pass after Ruiz (1) */
  double pc_alpha;        /* Pock-Chambolle alpha in [0, 2] (1.0) */
  int power_iters;        /* power iterations for ||Ahat||_2 (100) */
  double step_factor;     /* eta = step_factor / ||Ahat||_2 (0.9) */
  int restarts;           /* 1: averaging + adaptive restarts (1) */
  int primal_weight;      /* 1: omega0 = ||chat||/||bhat|| and updates at restarts (1) */
  int eval_every;         /* iterations between evaluations (64) */
  double beta_suff;       /* sufficient-decay restart factor (0.2) */
  double beta_nec;        /* necessary-decay restart factor (0.8) */
  double beta_art;        /* artificial restart fraction (0.36) */
  double theta;           /* primal-weight smoothing (0.5) */
  double eps_cross;       /* Algorithm 1: first snapshot target; 0 = off (0) */
  double eps_factor;      /* Algorithm 1: target shrink factor (0.1) */
  int64_t snapshot_every; /* periodic snapshots every this many iterations; 0 = off */
  int inputs_on_device;   /* 1: pointers given to pdhg_create are device pointers */
  int use_graphs;         /* 1: replay evaluation blocks as CUDA graphs (1) */
  int kernel_timing;      /* 1: time the two step kernels with CUDA events (0) */
  double polish_switch;   /* PDHG_MIXED: rel. KKT at which FP64 iterations take over; they also take over
                             when the FP32 phase stalls (no 10% gain in 16384 iterations, 65536 when the
                             phase is refined). -1 = automatic:
                             0 (on a stall only) when the FP32 phase is refined (refine32), else 1e-5 (-1) */
  int long_row_min;       /* rows with at least this many entries get a warp each (128) */
  int rows_per_thread;    /* most rows one thread reduces at once in short rows: 1, 2 or 4 (4) */
  int dual_hot_cols;      /* entries of xbar (the first ones, i.e. the longest columns of A) the dual step
                             stages in shared memory: 0 = off; at most 56320, and at most 28160 are staged in
                             FP64 phases (0) */
  int record_for_backward; /* 1: keep checkpoints for pdhg_backward; needs restarts = 0, primal_weight = 0,
                              precision FP64 or FP32 (0) */
  int64_t checkpoint_every; /* iterations between adjoint checkpoints (50) */
  int persistent;         /* 1: run the solve loop of each LP in one thread block: a single launch does the
                             iterations, evaluations, restarts and termination test with the LP's vectors in
                             shared memory (LPs with 7n + 6m <= 28672, i.e. up to ~224 KiB of vectors; FP64,
                             no recording, no kernel timing); 2 (batches): one cooperative launch over the whole
                             GPU runs every instance's iterations, evaluations, restarts and termination test,
                             the phases separated by grid-wide barriers whose waits are bounded by
                             barrier_cycles (replayed from a CUDA graph when use_graphs = 1; no kernel timing);
                             0: two launches per iteration (0) */
  int step_block;         /* threads per block of the step and evaluation kernels: 128, 256 or 512 (256) */
  int primal_panels;      /* panel-tiled primal half-step: y is cut into panels that fit in shared memory and
                             the long rows of A^T (columns with >= long_row_min entries) into per-panel
                             segments whose partial sums are added per column, while the other columns take
                             the direct step; 1 = on, 0 = off, -1 = on for single LPs with m >= 2^18 and
                             nnz >= 2^23 (-1) */
  int panel_rows;         /* entries of y per panel; 0 = as many as fit in shared memory (0; at most 28160, or
                             56320 with precision PDHG_FP32, whose panels hold FP32 entries only) */
  int halpern;            /* 1: reflected Halpern iteration (the cuPDLP+ line, Section 4.1): z <- w ((1 + rho)
                             T(z) - rho z) + (1 - w) z_r with T the PDHG map, w = (t + 1) / (t + 2), t the
                             iterations since the last restart, z_r the last restart point; no averaging (the
                             current iterate is the restart candidate). Single LPs, every precision, not
                             persistent (0) */
  double halpern_reflect; /* rho in [0, 1] (1.0) */
  double gap_tol;         /* relative-gap tolerance of the termination test: converged when rel_p <= tol,
                             rel_d <= tol and rel_gap <= gap_tol; 0 = tol (Section 2's single eps) (0) */
  int feas_polish;        /* 1: feasibility polishing, the PDLP variant Section 5 describes (PDHG iterations
                             with a zero objective inside the main solve): at an evaluation whose candidate has
                             rel_gap <= gap_tol but fails the test, at most once until the iteration count has
                             doubled, run PDHG with c = 0 from (x_c, 0) until rel_p <= tol, then with b = 0 from
                             (0, y_c) until rel_d <= tol, each phase with the current scaling, step and primal
                             weight and at most polish_div-th of the iterations so far (whole evaluation
                             periods); the solve ends with (x_p, y_d) if that pair passes the test, otherwise it
                             goes on unchanged. Single LPs, FP64 phases only (in PDHG_MIXED after the switch),
                             not persistent, no recording (0) */
  int polish_div;         /* polishing phase budget divisor (8) */
  int singleton_order;    /* 1: number the columns with one entry by the row of that entry (single LPs), so
                             that the step kernels gather them nearly in order; 0: by the caller's order (1) */
  int panel_min_len;      /* panel-tiled primal step: columns whose units (see long_row_min, rows_per_thread)
                             hold only columns with at least this many entries go to the panels; 0 = 32 for
                             the layout of FP32 steps and long_row_min for FP64 steps (0). PDHG_FP32 layouts
                             also take twice the rows per panel (FP32 entries of y); PDHG_MIXED keeps one
                             layout of each kind, for its FP32 and its FP64 phase */
  int64_t barrier_cycles; /* persistent = 2: clock cycles one grid-barrier wait may last before the launch
                             gives up with PDHG_ERR_TIMEOUT; 0 = 2^31 (about a second) (0) */
  int restart_scheme;     /* 0: PDLP's restarts on the weighted KKT error (0); 1 (with halpern = 1, single
                             LPs, no feasibility polishing): the cuPDLP+ scheme the paper's solver follows
                             (Section 4.1, which gives no formula; readings): the three restart rules on the
                             fixed-point residual r(z) = ||z - T(z)||_M of the current point (T the PDHG map, M
                             the metric ||(dx,dy)||^2 = ||dx||^2/tau + 2 dy^T Ahat dx + ||dy||^2/sigma); a
                             restart moves the iterate and the anchor to T(z); the primal weight takes a PID
                             step on e = ln(omega dx / dy), dx and dy the moves of the restart point */
  int values32;           /* FP64 steps on FP32 copies of A's unscaled values, read with FP64 arithmetic: the
                             values are then exact when every value of A is an FP32 number (checked at
                             create), and the steps stream 4 bytes less per entry; they apply the scaling
                             D_r, D_c per row and column and gather D_c xbar and D_r y. -1 = on for PDHG_MIXED
                             (its FP64 phase) when A's values are all FP32 numbers, off otherwise; 0 = off;
                             1 = on (PDHG_FP64 or PDHG_MIXED; PDHG_ERR_INVALID if a value of A is not an FP32
                             number). Single LPs, not persistent, no recording; the dual step then stages no
                             entries of xbar (dual_hot_cols) in FP64 phases (-1) */
  double pid_kp, pid_ki, pid_kd; /* restart_scheme = 1: PID gains of the primal weight (0.99, 0.01, 0) */
  int stream_steps;       /* 1: the half-steps of single LPs run as streamed kernels: every warp keeps the
                             next pieces of its matrix units and its rows of the step's vectors in flight in
                             a ring of shared-memory slots filled by bulk copies (TMA), and issues only the
                             gathers from registers; same arithmetic in the same order as the direct step
                             kernels, so bit-identical results. A bounded wait that runs out ends the call
                             with PDHG_ERR_TIMEOUT. Not with persistent, dual_hot_cols or batches; the
                             range-checked build ignores it (0) */
  int stream_warps;       /* stream_steps: warps per block, 1..16 (8) */
  int stream_depth;       /* stream_steps: shared-memory slots per warp, 2..8; the block's shared memory,
                             warps x depth x (512 x (4 + value bytes) + 544 x vector bytes + 8), must stay
                             within 227 KB (3) */
  int refine32;           /* 1 (precision FP32 or MIXED): the FP32 iteration runs on FP32 corrections to the
                             last restart point, which is held in FP64: a restart moves that point (in FP64)
                             and recomputes, with FP64 sparse products, the FP32 iteration's costs - the
                             residuals chat - Ahat^T y_r and bhat - Ahat x_r at the point - and the bounds
                             -x_r of the primal corrections; the FP32 rounding then scales with the corrections,
                             which shrink as the solve converges, rather than with the iterate. Single LPs,
                             no recording or persistent loop. 0 = off; -1 = on for PDHG_MIXED, off for
                             PDHG_FP32 (-1) */
  int panel_overlap;      /* panel-tiled primal step: 1 = the short-column step is a programmatic dependent
                             launch of the panel pass, so its blocks start on SMs as the panel pass's blocks
                             finish; only its per-column combine of the panels' partial sums waits for the
                             whole pass (same results); 0 = the two launches in sequence; -1 = 1 for FP32
                             steps, 0 for FP64 steps (where it measured slower) (-1) */
  int panel_balance;      /* panel-tiled primal step: 1 = panel heights follow the long columns' entries, so
                             that every panel gets a whole number of the panel pass's blocks (one wave) with
                             equal entries per block, each panel at most panel_rows rows (or as many as fit in
                             shared memory when panel_rows = 0); 0 = every panel panel_rows rows; -1 = 1 when
                             panel_rows = 0, else 0 (-1). Results differ from equal heights by rounding only
                             (the partial sums are cut at other rows) */
} pdhg_options;

/* Per-evaluation log: when the environment variable PDHG_LOG names a file at
 * pdhg_create, the context appends one JSON line per evaluation of
 * pdhg_iterate (single LPs): iteration, the candidate's rel_p, rel_d, rel_gap
 * and rel_kkt (Section 2's relative termination test), its objectives, the
 * candidate kind, the restart decision, the restart count, omega, the
 * arithmetic of the iteration (fp32 / fp64), converged, and the seconds since
 * create. A file that cannot be opened leaves the log off. Off by default. */

/* Scalars of one point on the problem as given (unscaled), all FP64.
 * r_P = b - A x, r_D = A^T y + z - c with z = max(0, c - A^T y) (Section 2);
 * rel_* are the three ratios of the relative termination test (Section 2) and
 * rel_kkt is their maximum ("maxresid" of Algorithm 1). */
typedef struct {
  double rp_norm2, rp_norminf;
  double rd_norm2, rd_norminf;
  double primal_obj;      /* c^T x */
  double dual_obj;        /* b^T y */
  double gap;             /* |c^T x - b^T y| */
  double complementarity; /* x^T z */
  double rel_p, rel_d, rel_gap, rel_kkt;
  int64_t iteration;
} pdhg_kkt_info;

/* Engine scalars after setup / during the solve. */
typedef struct {
  double norm_estimate;   /* power-iteration estimate of ||Ahat||_2 */
  double eta, omega, tau, sigma;
  int64_t iterations;     /* total PDHG iterations so far */
  int64_t since_restart;
  int64_t restarts;
  int64_t evaluations;
  int64_t snapshots;      /* scheduled snapshots taken so far */
  double last_rel_kkt;    /* rel_kkt of the last evaluation's candidate */
  int precision_now;      /* arithmetic currently used by the iteration */
  int converged;
  double kernel_ms_primal, kernel_ms_dual; /* summed event times (kernel_timing) */
  int64_t kernel_launches_primal, kernel_launches_dual;
  int64_t kernel_launches; /* all kernels launched by pdhg_iterate so far */
  int64_t polish_started_at; /* PDHG_MIXED: iteration where FP64 took over, -1 if not (yet) */
  int64_t feas_polish_attempts;   /* feasibility polishing attempts so far */
  int64_t feas_polish_iterations; /* iterations run in polishing phases (not counted in `iterations`) */
  int feas_polished;              /* 1: the current iterate is a polished pair (x_p, y_d) that passed the test */
  int persistent_grid;            /* persistent = 2: blocks of the cooperative launch (0 before the first) */
  int64_t graph_launches;         /* CUDA-graph launches by pdhg_iterate so far */
  int values32;                   /* 1: FP64 steps read the FP32 copies of A's unscaled values (option values32) */
  int stream_steps;               /* 1: the half-steps run as streamed kernels (option stream_steps) */
  int refine32;                   /* 1: FP32 phases run on corrections to an FP64 point (option refine32) */
  int panels;                     /* panels of the panel-tiled primal step's layout for the phase in use (0: the
                                     direct step over every column) */
} pdhg_info;

/* One feasibility polishing attempt. */
typedef struct {
  int64_t iteration;     /* main iteration count at the attempt */
  int64_t budget;        /* iteration limit of each phase */
  int64_t primal_iters, dual_iters;
  int32_t primal_ok, dual_ok; /* the phase reached rel_p <= tol (rel_d <= tol) */
  double rel_kkt, rel_gap;    /* of the pair (x_p, y_d) on the problem as given; +inf if a phase failed */
} pdhg_polish_rec;

/* One record per evaluation. */
typedef struct {
  int64_t iteration;
  int32_t kind;       /* PDHG_NO_RESTART / _TO_CURRENT / _TO_AVERAGE */
  int32_t candidate;  /* PDHG_RESTART_TO_CURRENT or _TO_AVERAGE */
  double omega;       /* primal weight after this evaluation */
  double rel_kkt;     /* candidate's rel_kkt on the problem as given */
} pdhg_trace_rec;

/* Fill *opt with the defaults listed above. */
PDHG_API void pdhg_default_options(pdhg_options* opt);

/* Create a solver for one LP, the primal/dual pair of Section 2. A (m x n,
 * CSR: row_ptr[m+1], col_idx[nnz], val[nnz]), b[m], c[n]; x0[n] and y0[m] are
 * an optional warm start (NULL = zeros). Host pointers, or device pointers when
 * opt->inputs_on_device = 1; all are borrowed for the call (the context keeps
 * its own copies). opt NULL = the defaults. Setup: copy, transpose, Ruiz +
 * Pock-Chambolle scaling, power iteration for eta, primal weight omega0, and
 * the evaluation of the starting point. Errors: INVALID for sizes out of range,
 * NULL arrays, malformed CSR or options out of range; NUMERIC for NaN/Inf in
 * A, b, c or the warm start; CUDA / OOM from the device. On failure *out is
 * NULL and pdhg_last_error(NULL) describes the failure (per host thread). */
PDHG_API pdhg_status pdhg_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row_ptr, const int32_t* col_idx,
                                 const double* val, const double* b, const double* c, const double* x0,
                                 const double* y0, const pdhg_options* opt, void* cuda_stream, pdhg_ctx** out);

/* Free all device and pinned memory of the context. NULL-safe. */
PDHG_API void pdhg_destroy(pdhg_ctx* ctx);

/* Run PDHG iterations (Algorithm 1, "Perform PDHG iteration") until the
 * candidate passes the termination test at an evaluation (rel_kkt <= tol; with
 * gap_tol set, rel_p <= tol, rel_d <= tol and rel_gap <= gap_tol), or
 * max_iters more iterations (feasibility polishing phases not counted).
 * Evaluations happen every eval_every iterations (counted from the first
 * iteration of the context) when tol > 0, restarts are on, or a snapshot
 * schedule is set. tol = 0 with restarts off runs exactly max_iters plain
 * iterations. Returns PDHG_OK when converged (or tol == 0), else
 * PDHG_ERR_NOT_CONVERGED; *iters_done (nullable) gets the count run. */
PDHG_API pdhg_status pdhg_iterate(pdhg_ctx* ctx, int64_t max_iters, double tol, int64_t* iters_done);

/* KKT measures (see pdhg_kkt_info; Section 2's residuals, gap and the three
 * relative ratios of its termination test) of the current iterate, the running
 * average or the last restart point (which = PDHG_CURRENT, PDHG_AVERAGE,
 * PDHG_LAST_RESTART), in FP64 on the problem as given; *out is caller-owned.
 * INVALID for a NULL out or another selector, STATE on a batch context. */
PDHG_API pdhg_status pdhg_kkt(pdhg_ctx* ctx, int which, pdhg_kkt_info* out);

/* Copy (x, y, z) of the chosen point (selector as in pdhg_kkt), on the
 * problem as given (Section 2's variables), into caller buffers x[n], y[m],
 * z[n] (any may be NULL). Host pointers unless on_device != 0.
 * z = max(0, c - A^T y). Synchronous. INVALID for another selector, STATE on
 * a batch context. */
PDHG_API pdhg_status pdhg_get_solution(pdhg_ctx* ctx, int which, double* x, double* y, double* z, int on_device);

/* Scheduled snapshots (Algorithm 1, Section 3.1: thresholds
 * eps_cross * eps_factor^j, and/or every snapshot_every iterations): the
 * evaluation's candidate point, unscaled, packed on the GPU and copied to
 * pinned host memory on a side stream while the iteration continues. *count
 * gets the number taken so far, *ready whether the latest copy has landed
 * (both nullable). Non-blocking; CUDA if the copy's event reports an error. */
PDHG_API pdhg_status pdhg_snapshot_poll(pdhg_ctx* ctx, int64_t* count, int* ready);

/* Copy the latest scheduled snapshot (Algorithm 1's (x_k, y_k, z_k)) into
 * caller-owned host buffers x[n], y[m], z[n] (any may be NULL) and its
 * iteration and rel_kkt (nullable); waits for its copy to land. STATE if none
 * was taken. */
PDHG_API pdhg_status pdhg_snapshot(pdhg_ctx* ctx, double* x, double* y, double* z, int64_t* iteration,
                                   double* rel_kkt);

/* Algorithm 1's hand-off to a concurrent consumer (a crossover thread): blocks
 * until a snapshot newer than number `after` (1-based count of snapshots taken;
 * 0 = any) has reached pinned host memory, then copies the newest one into the
 * caller's host buffers x (n), y (m), z (n) (any may be NULL) and returns its
 * number (index), iteration and rel_kkt. It may be called from threads other
 * than the one running pdhg_iterate, concurrently with it; the snapshot being
 * copied is protected from reuse until the copy is done (the iterating thread
 * waits for it, at most 60 s, before overwriting that ring slot). Returns
 * PDHG_ERR_TIMEOUT when no newer snapshot completes within timeout_ms (a host
 * wait: nothing waits on the GPU) and INVALID for after < 0 or
 * timeout_ms < 0; does not update pdhg_last_error. The
 * context must outlive the calls (destroy it only after its consumers have
 * returned). */
PDHG_API pdhg_status pdhg_snapshot_wait(pdhg_ctx* ctx, int64_t after, int64_t timeout_ms, double* x, double* y,
                                        double* z, int64_t* index, int64_t* iteration, double* rel_kkt);

/* Reverse pass through every iteration run so far (all of them plain
 * fixed-step PDHG iterations: the context must have been created with
 * record_for_backward = 1). Given dL/dx_K[n] and optionally dL/dy_K[m] (NULL =
 * 0) for the current iterate on the problem as given, writes dL/dc[n] and
 * dL/db[m], holding the scaling, eta and omega fixed (they depend on A only).
 * Checkpoints of (x, y) every checkpoint_every iterations are kept during
 * pdhg_iterate; each segment is recomputed from its checkpoint and reversed
 * with one A^T and one A SpMV per iteration, in the context's precision. The
 * derivative of max(u, 0) at u = 0 is taken as 0. Pointers are host memory
 * unless on_device != 0. STATE if recording is off. */
PDHG_API pdhg_status pdhg_backward(pdhg_ctx* ctx, const double* dL_dxK, const double* dL_dyK, double* dL_dc,
                                   double* dL_db, int on_device);

/* Engine scalars (iteration counts, restarts, step sizes, primal weight,
 * precision in use, polishing counts; see pdhg_info) into the caller-owned
 * *out. INVALID for a NULL out. */
PDHG_API pdhg_status pdhg_get_info(pdhg_ctx* ctx, pdhg_info* out);

/* Copy up to cap evaluation records (oldest first: at each evaluation the
 * candidate's rel_kkt, the restart decision and the primal weight) into the caller-owned
 * host array recs; *count gets the number stored (at most 65536 are kept). */
PDHG_API pdhg_status pdhg_get_trace(pdhg_ctx* ctx, pdhg_trace_rec* recs, int64_t cap, int64_t* count);

/* Feasibility polishing (the PDLP variant Section 5 describes; see the
 * feas_polish option): copy up to cap attempt records, oldest first, into the
 * caller-owned host array recs (NULL allowed when cap = 0); *count (nullable)
 * gets the number of attempts so far. INVALID if cap < 0, or recs is NULL with
 * cap > 0. Host-only, no device work. */
PDHG_API pdhg_status pdhg_get_polish_log(pdhg_ctx* ctx, pdhg_polish_rec* recs, int64_t cap, int64_t* count);

/* KKT measures (as pdhg_kkt) of a point (x, y), z = max(0, c - A^T y), of an LP
 * the caller keeps on the device, computed WITHOUT ALLOCATING ANY MEMORY. The
 * paper has no counterpart; this entry point exists for callers that cannot
 * let a library allocate: applications whose device memory belongs to their
 * own pool or framework allocator, services held to a fixed memory budget, and
 * latency-critical code where cudaMalloc/cudaFree would synchronize the device.
 *   Inputs (all DEVICE pointers, borrowed for the call): A as CSR
 *   (a_row_ptr[m+1] int64, a_col_idx[nnz] int32, a_val[nnz]) and its transpose
 *   as CSR (at_row_ptr[n+1], at_col_idx[nnz], at_val[nnz]); b[m], c[n], x[n],
 *   y[m]. Indices are not checked and must be in range. Output: *out in HOST
 *   memory (iteration = -1). Work runs on cuda_stream (NULL = legacy default
 *   stream); the call waits for it to finish.
 *   blocks: blocks per pass, 0 = 4 per SM; at most 1024, because the partial
 *   sums live in one fixed 96 KiB array in device memory that the library
 *   declares statically (every GPU that loads the library holds it until the
 *   process exits). Larger values return PDHG_ERR_INVALID.
 *   The first call on a device looks up that array's device address (once per
 *   device) and keeps it for the life of the process; make that first call
 *   before any stream capture. The kept address does not survive a
 *   cudaDeviceReset, nor a switch to a context other than the device's
 *   primary one: after either, do not call this entry point again.
 *   All calls on a device share the array and leave their partial sums in it;
 *   each call overwrites what it reads, so nothing needs clearing, but calls
 *   that overlap on the GPU (unordered streams or threads) race and return
 *   wrong values: order them on one stream.
 *   Errors: INVALID (bad sizes, NULL pointers, blocks > 1024), CUDA, NUMERIC
 *   (non-finite result); pdhg_last_error(NULL) describes the failure. */
PDHG_API pdhg_status pdhg_kkt_noalloc(int64_t m, int64_t n, const int64_t* a_row_ptr, const int32_t* a_col_idx,
                                      const double* a_val, const int64_t* at_row_ptr, const int32_t* at_col_idx,
                                      const double* at_val, const double* b, const double* c, const double* x,
                                      const double* y, int blocks, void* cuda_stream, pdhg_kkt_info* out);

/* One LP of a batch (host pointers, borrowed for the call; same CSR rules as
 * pdhg_create). */
typedef struct {
  int64_t m, n, nnz;
  const int64_t* row_ptr;
  const int32_t* col_idx;
  const double* val;
  const double* b;
  const double* c;
} pdhg_lp_desc;

/* A batch of independent LPs of uneven sizes solved together: every PDHG
 * half-step is one launch over all instances (their matrices laid out block-
 * diagonally, each instance renumbered on its own and padded to whole thread
 * blocks), while scaling, step sizes, primal weight, averages, restarts and
 * termination are per instance; an instance that has converged stops (its
 * blocks return at once). FP64, host inputs, starting point zero; recording
 * and warm starts are not available for batches, and snapshots are taken per
 * instance (pdhg_snapshot_i; not with persistent = 1). Use pdhg_iterate (runs
 * until every instance meets tol, or max_iters), pdhg_batch_info,
 * pdhg_batch_kkt, pdhg_batch_solution and pdhg_snapshot_i; pdhg_kkt and
 * pdhg_get_solution return STATE.
 * Errors: INVALID for count < 1, a NULL lps, an instance that fails
 * pdhg_create's checks (the message names it), totals of m, n or nnz at or
 * above 2^31 - 1, or options a batch does not take (primal_panels = 1,
 * feas_polish); NUMERIC for NaN/Inf in an instance; CUDA / OOM from the
 * device. On failure *out is NULL. */
PDHG_API pdhg_status pdhg_create_batch(int count, const pdhg_lp_desc* lps, const pdhg_options* opt,
                                       void* cuda_stream, pdhg_ctx** out);

/* Per-instance arrays of length count, caller-owned host memory (any may be
 * NULL): iterations run, converged (rel_kkt <= tol at an evaluation), last
 * candidate rel_kkt, restarts. Also valid for a single-LP context
 * (count = 1). */
PDHG_API pdhg_status pdhg_batch_info(pdhg_ctx* ctx, int64_t* iterations, int* converged, double* rel_kkt,
                                     int64_t* restarts);

/* pdhg_kkt for one instance of a batch (the same measures, on that instance's
 * problem as given): its current, average or last-restart point. INVALID for
 * a NULL out, an instance outside [0, count) or another selector. */
PDHG_API pdhg_status pdhg_batch_kkt(pdhg_ctx* ctx, int instance, int which, pdhg_kkt_info* out);

/* (x, y, z) of one instance on its problem as given, into caller-owned host
 * buffers of its n, m, n (any may be NULL). INVALID for an instance outside
 * [0, count). */
PDHG_API pdhg_status pdhg_batch_solution(pdhg_ctx* ctx, int instance, double* x, double* y, double* z);

/* Algorithm 1's hand-off (Section 3.1) for each LP of a batch: with eps_cross
 * and/or snapshot_every set at pdhg_create_batch, every evaluation at which an
 * instance's candidate meets its own schedule (the thresholds
 * eps_cross * eps_factor^j of its rel_kkt, or its periodic mark) packs that
 * instance's candidate (x, y, z), on its problem as given, into a device copy
 * kept per instance (the latest one), inside the same launches (or the same
 * cooperative launch) as the iteration. This copies instance `instance`'s
 * latest snapshot into caller-owned host buffers x[n_i], y[m_i], z[n_i] (any
 * may be NULL) and its iteration, rel_kkt and the number of snapshots the
 * instance has taken (nullable). Synchronous: waits for the context's stream;
 * call it between pdhg_iterate calls. On a single-LP context it returns
 * pdhg_snapshot's latest snapshot (instance 0). INVALID for an instance outside
 * [0, count); STATE when no schedule was set or the instance has taken no
 * snapshot yet (*count is then still written). */
PDHG_API pdhg_status pdhg_snapshot_i(pdhg_ctx* ctx, int instance, double* x, double* y, double* z, int64_t* iteration,
                                     double* rel_kkt, int64_t* count);

/* Layout autotuner (no counterpart in the paper: a tuning aid for the step
 * kernels). Times the two step kernels with CUDA events on this LP (count = 1)
 * or batch (count > 1) for candidate layouts, by coordinate search over
 * long_row_min in {32, 64, 128, 256, 512}, then rows_per_thread in {1, 2, 4},
 * then step_block in {128, 256, 512}, each starting from the best so far, and
 * writes into *tuned a copy of *opt (defaults if NULL) with the fastest three.
 * With cache_path != NULL, a choice stored there for an LP of the same profile
 * (see pdhg_profile_key) is returned without any device work (*from_cache = 1;
 * from_cache may be NULL), and a newly timed choice is appended as one line
 * "key step_block rows_per_thread long_row_min ms_per_iteration". Host inputs
 * only; each candidate builds and frees its own context on cuda_stream.
 * Errors: INVALID for a NULL tuned, device inputs, or bad sizes, row
 * pointers or column indices; otherwise the first failing candidate's
 * status from pdhg_create or pdhg_iterate (for example INVALID for unsorted
 * columns, NUMERIC, CUDA, OOM). */
PDHG_API pdhg_status pdhg_autotune(int count, const pdhg_lp_desc* lps, const pdhg_options* opt,
                                   const char* cache_path, void* cuda_stream, pdhg_options* tuned,
                                   int* from_cache);

/* The profile under which pdhg_autotune stores its choice, into buf (at most
 * cap bytes including the terminating NUL): precision, the number of
 * instances, m, n and nnz on a log2 scale in steps of 1/2, and the share of
 * the rows of A and of A^T in each power-of-two length class, rounded to 10%.
 * Host logic only. INVALID for a NULL buf, cap < 1, a key longer than
 * cap - 1, or bad sizes, row pointers or column indices. */
PDHG_API pdhg_status pdhg_profile_key(int count, const pdhg_lp_desc* lps, int precision, char* buf, int64_t cap);

/* The current device's FP64 fused multiply-add throughput (no counterpart in
 * the paper: a measurement aid). The FP64 iteration issues one FP64 FMA per
 * stored matrix entry and a few FP64 operations per row and column, and this
 * GPU runs FP64 at a small fraction of its FP32 rate, so the FP64 pipe is a
 * second bound of the FP64 step kernels beside HBM bandwidth. A full-occupancy
 * grid runs independent FMA chains for a fixed count (about 0.1 s on a B300),
 * timed with CUDA events on cuda_stream (NULL = legacy default stream); the
 * call waits for it. *fma_per_s gets FMAs (lane operations) per second, *ms
 * (nullable) the kernel's time. Allocates no device memory. INVALID for a
 * NULL fma_per_s, CUDA from the device; pdhg_last_error(NULL) describes the
 * failure. */
PDHG_API pdhg_status pdhg_fp64_fma_rate(void* cuda_stream, double* fma_per_s, double* ms);

/* Description of the last failure of ctx, or of the last failed context-free
 * call (pdhg_create, pdhg_kkt_noalloc, pdhg_fp64_fma_rate) when ctx is NULL. Never
 * NULL. */
PDHG_API const char* pdhg_last_error(const pdhg_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PDHG_H */
