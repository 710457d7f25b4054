"""Python binding of libpdhg.so (the C ABI in include/pdhg.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels. Functions carry the C names (``pdhg_create``, ``pdhg_iterate``,
``pdhg_kkt``, ``pdhg_snapshot`` ...); ``Solver`` wraps one context.

Arrays may be numpy arrays (host) or torch tensors (host or CUDA). PyTorch is
used for device memory and streams only. There is no CPU fallback: if the
library is missing or fails to load, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpdhg.so")

(PDHG_OK, PDHG_ERR_INVALID, PDHG_ERR_CUDA, PDHG_ERR_OOM, PDHG_ERR_TIMEOUT, PDHG_ERR_NUMERIC, PDHG_ERR_STATE,
 PDHG_ERR_NOT_CONVERGED) = range(8)
STATUS_NAMES = ["OK", "INVALID", "CUDA", "OOM", "TIMEOUT", "NUMERIC", "STATE", "NOT_CONVERGED"]
PDHG_FP64, PDHG_FP32, PDHG_MIXED = 0, 1, 2
PDHG_CURRENT, PDHG_AVERAGE, PDHG_LAST_RESTART = 0, 1, 2
PDHG_NO_RESTART, PDHG_RESTART_TO_CURRENT, PDHG_RESTART_TO_AVERAGE, PDHG_RESTART_TO_PDHG_STEP = 0, 1, 2, 3


class pdhg_options(C.Structure):
    _fields_ = [
        ("precision", C.c_int),
        ("ruiz_iters", C.c_int),
        ("pock_chambolle", C.c_int),
        ("pc_alpha", C.c_double),
        ("power_iters", C.c_int),
        ("step_factor", C.c_double),
        ("restarts", C.c_int),
        ("primal_weight", C.c_int),
        ("eval_every", C.c_int),
        ("beta_suff", C.c_double),
        ("beta_nec", C.c_double),
        ("beta_art", C.c_double),
        ("theta", C.c_double),
        ("eps_cross", C.c_double),
        ("eps_factor", C.c_double),
        ("snapshot_every", C.c_int64),
        ("inputs_on_device", C.c_int),
        ("use_graphs", C.c_int),
        ("kernel_timing", C.c_int),
        ("polish_switch", C.c_double),
        ("long_row_min", C.c_int),
        ("rows_per_thread", C.c_int),
        ("dual_hot_cols", C.c_int),
        ("record_for_backward", C.c_int),
        ("checkpoint_every", C.c_int64),
        ("persistent", C.c_int),
        ("step_block", C.c_int),
        ("primal_panels", C.c_int),
        ("panel_rows", C.c_int),
        ("halpern", C.c_int),
        ("halpern_reflect", C.c_double),
        ("gap_tol", C.c_double),
        ("feas_polish", C.c_int),
        ("polish_div", C.c_int),
        ("singleton_order", C.c_int),
        ("panel_min_len", C.c_int),
        ("barrier_cycles", C.c_int64),
        ("restart_scheme", C.c_int),
        ("values32", C.c_int),
        ("pid_kp", C.c_double),
        ("pid_ki", C.c_double),
        ("pid_kd", C.c_double),
        ("stream_steps", C.c_int),
        ("stream_warps", C.c_int),
        ("stream_depth", C.c_int),
        ("refine32", C.c_int),
        ("panel_overlap", C.c_int),
        ("panel_balance", C.c_int),
    ]


class pdhg_kkt_info(C.Structure):
    _fields_ = [(k, C.c_double) for k in (
        "rp_norm2", "rp_norminf", "rd_norm2", "rd_norminf", "primal_obj", "dual_obj", "gap", "complementarity",
        "rel_p", "rel_d", "rel_gap", "rel_kkt")] + [("iteration", C.c_int64)]


class pdhg_info(C.Structure):
    _fields_ = [
        ("norm_estimate", C.c_double), ("eta", C.c_double), ("omega", C.c_double), ("tau", C.c_double),
        ("sigma", C.c_double), ("iterations", C.c_int64), ("since_restart", C.c_int64), ("restarts", C.c_int64),
        ("evaluations", C.c_int64), ("snapshots", C.c_int64), ("last_rel_kkt", C.c_double),
        ("precision_now", C.c_int), ("converged", C.c_int), ("kernel_ms_primal", C.c_double),
        ("kernel_ms_dual", C.c_double), ("kernel_launches_primal", C.c_int64), ("kernel_launches_dual", C.c_int64),
        ("kernel_launches", C.c_int64),
        ("polish_started_at", C.c_int64),
        ("feas_polish_attempts", C.c_int64), ("feas_polish_iterations", C.c_int64), ("feas_polished", C.c_int),
        ("persistent_grid", C.c_int), ("graph_launches", C.c_int64), ("values32", C.c_int),
        ("stream_steps", C.c_int), ("refine32", C.c_int), ("panels", C.c_int),
    ]


class pdhg_polish_rec(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("budget", C.c_int64), ("primal_iters", C.c_int64),
                ("dual_iters", C.c_int64), ("primal_ok", C.c_int32), ("dual_ok", C.c_int32), ("rel_kkt", C.c_double),
                ("rel_gap", C.c_double)]


class pdhg_trace_rec(C.Structure):
    _fields_ = [("iteration", C.c_int64), ("kind", C.c_int32), ("candidate", C.c_int32), ("omega", C.c_double),
                ("rel_kkt", C.c_double)]


class pdhg_lp_desc(C.Structure):
    _fields_ = [("m", C.c_int64), ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p), ("b", C.c_void_p), ("c", C.c_void_p)]


class PDHGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"PDHG_{name}: {msg}")


_lib = None
_P = C.c_void_p

# every exported symbol of include/pdhg.h with its ctypes signature
SIGNATURES = {
    "pdhg_default_options": (None, [C.POINTER(pdhg_options)]),
    "pdhg_create": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, _P, C.POINTER(pdhg_options), _P,
                              C.POINTER(_P)]),
    "pdhg_destroy": (None, [_P]),
    "pdhg_iterate": (C.c_int, [_P, C.c_int64, C.c_double, C.POINTER(C.c_int64)]),
    "pdhg_kkt": (C.c_int, [_P, C.c_int, C.POINTER(pdhg_kkt_info)]),
    "pdhg_get_solution": (C.c_int, [_P, C.c_int, _P, _P, _P, C.c_int]),
    "pdhg_snapshot_poll": (C.c_int, [_P, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "pdhg_snapshot": (C.c_int, [_P, _P, _P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "pdhg_snapshot_wait": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "pdhg_get_info": (C.c_int, [_P, C.POINTER(pdhg_info)]),
    "pdhg_backward": (C.c_int, [_P, _P, _P, _P, _P, C.c_int]),
    "pdhg_get_trace": (C.c_int, [_P, C.POINTER(pdhg_trace_rec), C.c_int64, C.POINTER(C.c_int64)]),
    "pdhg_get_polish_log": (C.c_int, [_P, C.POINTER(pdhg_polish_rec), C.c_int64, C.POINTER(C.c_int64)]),
    "pdhg_last_error": (C.c_char_p, [_P]),
    "pdhg_create_batch": (C.c_int, [C.c_int, C.POINTER(pdhg_lp_desc), C.POINTER(pdhg_options), _P, C.POINTER(_P)]),
    "pdhg_batch_info": (C.c_int, [_P, _P, _P, _P, _P]),
    "pdhg_batch_solution": (C.c_int, [_P, C.c_int, _P, _P, _P]),
    "pdhg_batch_kkt": (C.c_int, [_P, C.c_int, C.c_int, C.POINTER(pdhg_kkt_info)]),
    "pdhg_kkt_noalloc": (C.c_int, [C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, C.c_int, _P,
                                   C.POINTER(pdhg_kkt_info)]),
    "pdhg_autotune": (C.c_int, [C.c_int, C.POINTER(pdhg_lp_desc), C.POINTER(pdhg_options), C.c_char_p, _P,
                                C.POINTER(pdhg_options), C.POINTER(C.c_int)]),
    "pdhg_profile_key": (C.c_int, [C.c_int, C.POINTER(pdhg_lp_desc), C.c_int, C.c_char_p, C.c_int64]),
    "pdhg_fp64_fma_rate": (C.c_int, [_P, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "pdhg_snapshot_i": (C.c_int, [_P, C.c_int, _P, _P, _P, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                  C.POINTER(C.c_int64)]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    """Load libpdhg.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libpdhg.so not built ({path}); run __graft_entry__.build() or "
                           "python paper_2510_24429_b300/build.py")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, ctx=None):
    if status != PDHG_OK:
        raise PDHGError(status, load().pdhg_last_error(ctx).decode())


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _prep(a, dtype, keep: list):
    """Return (pointer, on_device) for an input array; keeps converted copies alive."""
    if a is None:
        return None, False
    if _is_torch(a):
        import torch

        tdt = {np.float64: torch.float64, np.int64: torch.int64, np.int32: torch.int32}[dtype]
        t = a.to(tdt).contiguous()
        keep.append(t)
        return t.data_ptr(), t.is_cuda
    arr = np.ascontiguousarray(a, dtype=dtype)
    keep.append(arr)
    return arr.ctypes.data, False


def _out_ptr(a):
    if a is None:
        return None, False
    if _is_torch(a):
        import torch

        if not a.is_contiguous() or a.dtype != torch.float64:
            raise ValueError("output tensors must be contiguous float64")
        return a.data_ptr(), a.is_cuda
    if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
        raise ValueError("output arrays must be contiguous float64 numpy arrays")
    return a.ctypes.data, False


# ---------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------

def pdhg_default_options(**overrides) -> pdhg_options:
    o = pdhg_options()
    load().pdhg_default_options(C.byref(o))
    for k, v in overrides.items():
        if not hasattr(o, k) or k.startswith("reserved"):
            raise KeyError(f"unknown option {k}")
        setattr(o, k, v)
    return o


def pdhg_create(m, n, row_ptr, col_idx, val, b, c, x0=None, y0=None, opt: pdhg_options | None = None,
                stream=None) -> int:
    lib = load()
    keep: list = []
    ptrs = [_prep(row_ptr, np.int64, keep), _prep(col_idx, np.int32, keep), _prep(val, np.float64, keep),
            _prep(b, np.float64, keep), _prep(c, np.float64, keep), _prep(x0, np.float64, keep),
            _prep(y0, np.float64, keep)]
    dev = {d for p, d in ptrs if p is not None}
    if len(dev) > 1:
        raise ValueError("inputs must be all on the host or all on the device")
    if opt is None:
        opt = pdhg_default_options()
    opt.inputs_on_device = int(dev == {True})
    nnz = int(len(val))
    if stream is None and opt.inputs_on_device:
        import torch

        stream = torch.cuda.current_stream().cuda_stream
    out = C.c_void_p()
    st = lib.pdhg_create(int(m), int(n), nnz, *[p for p, _ in ptrs], C.byref(opt),
                         C.c_void_p(stream) if stream else None, C.byref(out))
    _check(st, None)
    return out.value


def pdhg_destroy(ctx):
    if ctx:
        load().pdhg_destroy(ctx)


def pdhg_iterate(ctx, max_iters: int, tol: float = 0.0, raise_on_not_converged: bool = False):
    """Returns (status, iterations run)."""
    done = C.c_int64()
    st = load().pdhg_iterate(ctx, int(max_iters), float(tol), C.byref(done))
    if st not in (PDHG_OK, PDHG_ERR_NOT_CONVERGED) or (raise_on_not_converged and st != PDHG_OK):
        _check(st, ctx)
    return st, done.value


def pdhg_kkt(ctx, which: int = PDHG_CURRENT) -> dict:
    info = pdhg_kkt_info()
    _check(load().pdhg_kkt(ctx, int(which), C.byref(info)), ctx)
    return {k: getattr(info, k) for k, _ in pdhg_kkt_info._fields_}


def pdhg_get_solution(ctx, which=PDHG_CURRENT, x=None, y=None, z=None):
    ptrs = [_out_ptr(a) for a in (x, y, z)]
    dev = {d for p, d in ptrs if p is not None}
    if len(dev) > 1:
        raise ValueError("outputs must be all on the host or all on the device")
    _check(load().pdhg_get_solution(ctx, int(which), *[p for p, _ in ptrs], int(dev == {True})), ctx)


def pdhg_snapshot_poll(ctx):
    cnt, ready = C.c_int64(), C.c_int()
    _check(load().pdhg_snapshot_poll(ctx, C.byref(cnt), C.byref(ready)), ctx)
    return cnt.value, bool(ready.value)


def pdhg_snapshot(ctx, x=None, y=None, z=None):
    ptrs = [_out_ptr(a) for a in (x, y, z)]
    if any(d for _, d in ptrs):
        raise ValueError("snapshot buffers are host arrays")
    it, rel = C.c_int64(), C.c_double()
    _check(load().pdhg_snapshot(ctx, *[p for p, _ in ptrs], C.byref(it), C.byref(rel)), ctx)
    return it.value, rel.value


def pdhg_snapshot_wait(ctx, after=0, timeout_ms=1000, x=None, y=None, z=None):
    """Newest snapshot numbered above ``after`` (blocks up to timeout_ms; may
    run in another thread while pdhg_iterate runs): (index, iteration,
    rel_kkt). Raises PDHGError(PDHG_ERR_TIMEOUT) if none completes in time."""
    ptrs = [_out_ptr(a) for a in (x, y, z)]
    if any(d for _, d in ptrs):
        raise ValueError("snapshot buffers are host arrays")
    idx, it, rel = C.c_int64(), C.c_int64(), C.c_double()
    st = load().pdhg_snapshot_wait(ctx, int(after), int(timeout_ms), *[p for p, _ in ptrs], C.byref(idx),
                                   C.byref(it), C.byref(rel))
    if st != PDHG_OK:
        raise PDHGError(st, "no newer snapshot within the timeout" if st == PDHG_ERR_TIMEOUT else "snapshot_wait failed")
    return idx.value, it.value, rel.value


def pdhg_backward(ctx, dL_dx, dL_dc, dL_db, dL_dy=None):
    """Gradients of a loss of the current iterate with respect to c and b
    (outputs dL_dc[n], dL_db[m] supplied by the caller, all host or all CUDA)."""
    keep: list = []
    px, dev = _prep(dL_dx, np.float64, keep)
    py, devy = _prep(dL_dy, np.float64, keep)
    pc, devc = _out_ptr(dL_dc)
    pb, devb = _out_ptr(dL_db)
    devs = {dev, devc, devb} | ({devy} if py is not None else set())
    if len(devs) != 1:
        raise ValueError("pdhg_backward: arrays must be all on the host or all on the device")
    _check(load().pdhg_backward(ctx, px, py, pc, pb, int(dev)), ctx)


def pdhg_get_info(ctx) -> dict:
    info = pdhg_info()
    _check(load().pdhg_get_info(ctx, C.byref(info)), ctx)
    return {k: getattr(info, k) for k, _ in pdhg_info._fields_}


def pdhg_get_trace(ctx) -> list[dict]:
    lib = load()
    cnt = C.c_int64()
    _check(lib.pdhg_get_trace(ctx, None, 0, C.byref(cnt)), ctx)
    recs = (pdhg_trace_rec * max(1, cnt.value))()
    _check(lib.pdhg_get_trace(ctx, recs, cnt.value, C.byref(cnt)), ctx)
    return [{k: getattr(r, k) for k, _ in pdhg_trace_rec._fields_} for r in recs[: cnt.value]]


def pdhg_get_polish_log(ctx) -> list[dict]:
    lib = load()
    cnt = C.c_int64()
    _check(lib.pdhg_get_polish_log(ctx, None, 0, C.byref(cnt)), ctx)
    recs = (pdhg_polish_rec * max(1, cnt.value))()
    _check(lib.pdhg_get_polish_log(ctx, recs, cnt.value, C.byref(cnt)), ctx)
    return [{k: getattr(r, k) for k, _ in pdhg_polish_rec._fields_} for r in recs[: cnt.value]]


def pdhg_last_error(ctx=None) -> str:
    return load().pdhg_last_error(ctx).decode()


def pdhg_kkt_noalloc(m, n, a_row_ptr, a_col_idx, a_val, at_row_ptr, at_col_idx, at_val, b, c, x, y, blocks=0,
                     stream=None) -> dict:
    """KKT measures of (x, y) for an LP held on the device as CSR of A and A^T,
    through the allocation-free entry point. Every array must already be a
    contiguous CUDA tensor of the right dtype (int64 row pointers, int32
    column indices, float64 values and vectors): nothing is converted or
    copied here, so the call allocates nothing."""
    import torch

    args = [a_row_ptr, a_col_idx, a_val, at_row_ptr, at_col_idx, at_val, b, c, x, y]
    want = [torch.int64, torch.int32, torch.float64] * 2 + [torch.float64] * 4
    for a, dt in zip(args, want):
        if not (_is_torch(a) and a.is_cuda and a.is_contiguous() and a.dtype == dt):
            raise ValueError("pdhg_kkt_noalloc takes contiguous CUDA tensors of the documented dtypes")
    # the kernels read the sizes given to them, so every length is checked
    # here (reading metadata only; nothing is allocated)
    m, n = int(m), int(n)
    lengths = {"a_row_ptr": (a_row_ptr, m + 1), "at_row_ptr": (at_row_ptr, n + 1), "b": (b, m), "y": (y, m),
               "c": (c, n), "x": (x, n)}
    for name, (a, want_len) in lengths.items():
        if a.numel() != want_len:
            raise ValueError(f"pdhg_kkt_noalloc: {name} has {a.numel()} entries, expected {want_len}")
    nnz = a_col_idx.numel()
    if not all(a.numel() == nnz for a in (a_val, at_col_idx, at_val)):
        raise ValueError("pdhg_kkt_noalloc: a_col_idx, a_val, at_col_idx and at_val must have the same length")
    dev = torch.cuda.current_device()
    if any(a.device.index != dev for a in args):
        raise ValueError(f"pdhg_kkt_noalloc: every tensor must be on the current device (cuda:{dev})")
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    info = pdhg_kkt_info()
    st = load().pdhg_kkt_noalloc(m, n, *[a.data_ptr() for a in args], int(blocks),
                                 C.c_void_p(stream) if stream else None, C.byref(info))
    _check(st, None)
    return {k: getattr(info, k) for k, _ in pdhg_kkt_info._fields_}


def _lp_descs(lps):
    """pdhg_lp_desc array for a sequence of (m, n, row_ptr, col_idx, val, b, c)
    tuples or objects with those attributes (host arrays); returns the array
    and the list of numpy arrays it points into (keep it alive)."""
    keep: list = []
    descs = (pdhg_lp_desc * len(lps))()
    for d, lp in zip(descs, lps):
        m, n, rp, ci, v, b, c = (lp if isinstance(lp, tuple) else
                                 (lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c))
        arrs = [np.ascontiguousarray(rp, np.int64), np.ascontiguousarray(ci, np.int32),
                np.ascontiguousarray(v, np.float64), np.ascontiguousarray(b, np.float64),
                np.ascontiguousarray(c, np.float64)]
        keep.extend(arrs)
        d.m, d.n, d.nnz = int(m), int(n), int(len(arrs[2]))
        d.row_ptr, d.col_idx, d.val, d.b, d.c = [a.ctypes.data for a in arrs]
    return descs, keep


def pdhg_autotune(lps, opt: pdhg_options | None = None, cache_path: str | None = None, stream=None):
    """Tuned layout options for one LP (a sequence of one) or a batch; returns
    (options, from_cache)."""
    descs, _keep = _lp_descs(lps)
    if opt is None:
        opt = pdhg_default_options()
    tuned, hit = pdhg_options(), C.c_int(0)
    _check(load().pdhg_autotune(len(lps), descs, C.byref(opt), cache_path.encode() if cache_path else None,
                                C.c_void_p(stream) if stream else None, C.byref(tuned), C.byref(hit)), None)
    return tuned, bool(hit.value)


def pdhg_fp64_fma_rate(stream=None) -> tuple[float, float]:
    """(FP64 FMAs per second, kernel milliseconds) measured on the current
    device."""
    rate, ms = C.c_double(0.0), C.c_double(0.0)
    _check(load().pdhg_fp64_fma_rate(C.c_void_p(stream) if stream else None, C.byref(rate), C.byref(ms)), None)
    return rate.value, ms.value


def pdhg_profile_key(lps, precision: int = 0) -> str:
    descs, _keep = _lp_descs(lps)
    buf = C.create_string_buffer(4096)
    _check(load().pdhg_profile_key(len(lps), descs, int(precision), buf, len(buf)), None)
    return buf.value.decode()


def pdhg_create_batch(lps, opt: pdhg_options | None = None, stream=None):
    """One context for many LPs; ``lps`` is a sequence of (m, n, row_ptr,
    col_idx, val, b, c) tuples or objects with those attributes (host arrays)."""
    descs, _keep = _lp_descs(lps)
    if opt is None:
        opt = pdhg_default_options()
    out = C.c_void_p()
    _check(load().pdhg_create_batch(len(lps), descs, C.byref(opt), C.c_void_p(stream) if stream else None,
                                    C.byref(out)), None)
    return out.value


def pdhg_batch_info(ctx, count):
    it, conv = np.zeros(count, np.int64), np.zeros(count, np.int32)
    rel, rs = np.zeros(count), np.zeros(count, np.int64)
    _check(load().pdhg_batch_info(ctx, it.ctypes.data, conv.ctypes.data, rel.ctypes.data, rs.ctypes.data), ctx)
    return dict(iterations=it, converged=conv.astype(bool), rel_kkt=rel, restarts=rs)


def pdhg_batch_solution(ctx, instance, m, n):
    x, y, z = np.empty(n), np.empty(m), np.empty(n)
    _check(load().pdhg_batch_solution(ctx, int(instance), x.ctypes.data, y.ctypes.data, z.ctypes.data), ctx)
    return x, y, z


class BatchSolver:
    """Many LPs solved together (see pdhg_create_batch in include/pdhg.h)."""

    def __init__(self, lps, stream=None, **options):
        self.sizes = [(lp.m, lp.n) if not isinstance(lp, tuple) else (lp[0], lp[1]) for lp in lps]
        self.ctx = None
        self.ctx = pdhg_create_batch(lps, pdhg_default_options(**options), stream)

    def iterate(self, max_iters, tol=0.0):
        return pdhg_iterate(self.ctx, max_iters, tol)

    def info(self):
        return pdhg_batch_info(self.ctx, len(self.sizes))

    def kkt(self, i, which=PDHG_CURRENT):
        """KKT measures of instance i (pdhg_batch_kkt)."""
        info = pdhg_kkt_info()
        _check(load().pdhg_batch_kkt(self.ctx, int(i), int(which), C.byref(info)), self.ctx)
        return {k: getattr(info, k) for k, _ in pdhg_kkt_info._fields_}

    def solution(self, i):
        m, n = self.sizes[i]
        return pdhg_batch_solution(self.ctx, i, m, n)

    def engine_info(self):
        return pdhg_get_info(self.ctx)

    def snapshot(self, i):
        """Instance i's latest scheduled snapshot (pdhg_snapshot_i): dict with
        x, y, z on its problem as given, iteration, rel_kkt and count."""
        m, n = self.sizes[i] if 0 <= i < len(self.sizes) else (1, 1)  # out of range: the library says INVALID
        x, y, z = np.empty(n), np.empty(m), np.empty(n)
        it, rel, cnt = C.c_int64(), C.c_double(), C.c_int64()
        _check(load().pdhg_snapshot_i(self.ctx, int(i), x.ctypes.data, y.ctypes.data, z.ctypes.data, C.byref(it),
                                      C.byref(rel), C.byref(cnt)), self.ctx)
        return {"x": x, "y": y, "z": z, "iteration": it.value, "rel_kkt": rel.value, "count": cnt.value}

    def close(self):
        if self.ctx:
            pdhg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Solver:
    """One LP resident on the GPU: ``Solver(m, n, row_ptr, col_idx, val, b, c, **options)``."""

    def __init__(self, m, n, row_ptr, col_idx, val, b, c, x0=None, y0=None, stream=None, **options):
        self.m, self.n = int(m), int(n)
        self.ctx = None
        self.ctx = pdhg_create(m, n, row_ptr, col_idx, val, b, c, x0, y0, pdhg_default_options(**options), stream)

    @classmethod
    def from_lp(cls, lp, **options):
        return cls(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, **options)

    def iterate(self, max_iters, tol=0.0):
        return pdhg_iterate(self.ctx, max_iters, tol)

    def kkt(self, which=PDHG_CURRENT):
        return pdhg_kkt(self.ctx, which)

    def solution(self, which=PDHG_CURRENT):
        x, y, z = np.empty(self.n), np.empty(self.m), np.empty(self.n)
        pdhg_get_solution(self.ctx, which, x, y, z)
        return x, y, z

    def snapshot(self):
        x, y, z = np.empty(self.n), np.empty(self.m), np.empty(self.n)
        it, rel = pdhg_snapshot(self.ctx, x, y, z)
        return dict(iteration=it, rel_kkt=rel, x=x, y=y, z=z)

    def snapshot_poll(self):
        return pdhg_snapshot_poll(self.ctx)

    def snapshot_wait(self, after=0, timeout_ms=1000):
        """Thread-safe hand-off of the newest snapshot numbered above ``after``."""
        x, y, z = np.empty(self.n), np.empty(self.m), np.empty(self.n)
        idx, it, rel = pdhg_snapshot_wait(self.ctx, after, timeout_ms, x, y, z)
        return dict(index=idx, iteration=it, rel_kkt=rel, x=x, y=y, z=z)

    def info(self):
        return pdhg_get_info(self.ctx)

    def backward(self, dL_dx, dL_dy=None):
        """(dL/dc, dL/db) through every iteration run so far (needs
        record_for_backward=1). CUDA tensors in give CUDA tensors out."""
        if _is_torch(dL_dx) and dL_dx.is_cuda:
            import torch

            gc = torch.empty(self.n, dtype=torch.float64, device=dL_dx.device)
            gb = torch.empty(self.m, dtype=torch.float64, device=dL_dx.device)
        else:
            gc, gb = np.empty(self.n), np.empty(self.m)
        pdhg_backward(self.ctx, dL_dx, gc, gb, dL_dy)
        return gc, gb

    def trace(self):
        return pdhg_get_trace(self.ctx)

    def polish_log(self):
        """One record per feasibility polishing attempt."""
        return pdhg_get_polish_log(self.ctx)

    def close(self):
        if self.ctx:
            pdhg_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# differentiable unrolled PDHG
# ---------------------------------------------------------------------------

def _unroll_function():
    import torch

    class PDHGUnroll(torch.autograd.Function):
        """x_K(c, b): K fixed-step PDHG iterations (no restarts, omega = 1) from
        zero on the LP with matrix ``csr = (m, n, row_ptr, col_idx, val)``;
        backward runs the library's adjoint (pdhg_backward) with checkpoints
        every ``checkpoint_every`` iterations. Scaling and step size depend on A
        only and are held fixed."""

        @staticmethod
        def forward(fctx, c, b, csr, iters, options):
            m, n, row_ptr, col_idx, val = csr
            sol = Solver(m, n, row_ptr, col_idx, val, b.detach().cpu().numpy(), c.detach().cpu().numpy(),
                         record_for_backward=1, restarts=0, primal_weight=0, **(options or {}))
            sol.iterate(int(iters))
            x = torch.empty(n, dtype=torch.float64, device=c.device)
            if x.is_cuda:
                pdhg_get_solution(sol.ctx, PDHG_CURRENT, x=x)
            else:
                xn = np.empty(n)
                pdhg_get_solution(sol.ctx, PDHG_CURRENT, x=xn)
                x.copy_(torch.from_numpy(xn))
            fctx.solver = sol
            return x

        @staticmethod
        def backward(fctx, grad_x):
            gc, gb = fctx.solver.backward(grad_x.detach().to(torch.float64).contiguous())
            fctx.solver.close()
            if not _is_torch(gc):
                gc, gb = torch.from_numpy(gc), torch.from_numpy(gb)
            return gc.to(grad_x.device), gb.to(grad_x.device), None, None, None

    return PDHGUnroll


def pdhg_unroll(c, b, csr, iters, **options):
    """Differentiable x_K(c, b) (see PDHGUnroll)."""
    return _unroll_function().apply(c, b, csr, iters, options)
