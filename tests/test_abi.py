"""Host-side checks of the C ABI: the library loads, exports every function
include/pdhg.h declares, the ctypes structs match the C layout, and argument
validation rejects malformed input before any device work (no GPU needed)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2510_24429_b300 import build as B
from paper_2510_24429_b300 import pdhg as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pdhg.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return P.load()


def _declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"PDHG_API\s+[\w\s\*]+?\b(pdhg_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert len(declared) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pdhg_\w+)", out))
    assert set(declared) <= exported, set(declared) - exported
    assert set(declared) == set(P.SIGNATURES), set(declared) ^ set(P.SIGNATURES)
    for name in declared:
        assert hasattr(lib, name)


def test_struct_layouts_match_header(tmp_path):
    structs = {"pdhg_options": P.pdhg_options, "pdhg_kkt_info": P.pdhg_kkt_info, "pdhg_info": P.pdhg_info,
               "pdhg_trace_rec": P.pdhg_trace_rec, "pdhg_polish_rec": P.pdhg_polish_rec,
               "pdhg_lp_desc": P.pdhg_lp_desc}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pdhg.h"', "int main(void) {"]
    for sname, cls in structs.items():
        lines.append(f'printf("{sname} size %zu\\n", sizeof({sname}));')
        for f, _ in cls._fields_:
            lines.append(f'printf("{sname}.{f} %zu\\n", offsetof({sname}, {f}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                                   check=True).stdout.splitlines())
    for sname, cls in structs.items():
        assert int(got[f"{sname} size"]) == C.sizeof(cls), sname
        for f, _ in cls._fields_:
            assert int(got[f"{sname}.{f}"]) == getattr(cls, f).offset, (sname, f)


def test_default_options(lib):
    o = P.pdhg_default_options()
    assert (o.ruiz_iters, o.pock_chambolle, o.power_iters, o.eval_every) == (10, 1, 100, 64)
    assert (o.step_factor, o.beta_suff, o.beta_nec, o.beta_art, o.theta) == (0.9, 0.2, 0.8, 0.36, 0.5)
    assert o.precision == P.PDHG_FP64 and o.restarts == 1 and o.primal_weight == 1
    assert (o.halpern, o.halpern_reflect, o.primal_panels, o.long_row_min) == (0, 1.0, -1, 128)
    assert (o.feas_polish, o.polish_div, o.gap_tol, o.polish_switch) == (0, 8, 0.0, -1.0)
    assert (o.dual_hot_cols, o.singleton_order, o.barrier_cycles) == (0, 1, 0)
    assert (o.panel_min_len, o.restart_scheme, o.values32) == (0, 0, -1)
    assert (o.pid_kp, o.pid_ki, o.pid_kd) == (0.99, 0.01, 0.0)
    assert (o.stream_steps, o.stream_warps, o.stream_depth, o.refine32, o.panel_overlap, o.panel_balance) == (
        0, 0, 3, -1, -1, -1)
    with pytest.raises(KeyError):
        P.pdhg_default_options(no_such_option=1)


def _tiny_csr():
    # A = [[1, 2, 0], [0, 1, 1]]
    return (np.array([0, 2, 4], np.int64), np.array([0, 1, 1, 2], np.int32), np.array([1.0, 2.0, 1.0, 1.0]),
            np.array([3.0, 2.0]), np.array([1.0, 1.0, 1.0]))


@pytest.mark.parametrize("mutate,status", [
    (lambda rp, ci, v, b, c: (np.array([0, 2, 5], np.int64), ci, v, b, c), P.PDHG_ERR_INVALID),  # rp[m] != nnz
    (lambda rp, ci, v, b, c: (rp, np.array([0, 3, 1, 2], np.int32), v, b, c), P.PDHG_ERR_INVALID),  # col out of range
    (lambda rp, ci, v, b, c: (rp, np.array([1, 0, 1, 2], np.int32), v, b, c), P.PDHG_ERR_INVALID),  # unsorted
    (lambda rp, ci, v, b, c: (rp, np.array([1, 1, 1, 2], np.int32), v, b, c), P.PDHG_ERR_INVALID),  # duplicate
    (lambda rp, ci, v, b, c: (np.array([0, 3, 2], np.int64), ci, v, b, c), P.PDHG_ERR_INVALID),  # decreasing rp
    (lambda rp, ci, v, b, c: (rp, ci, v, b, np.array([1.0, np.nan, 1.0])), P.PDHG_ERR_NUMERIC),  # NaN in c
    (lambda rp, ci, v, b, c: (rp, ci, np.array([1.0, np.inf, 1.0, 1.0]), b, c), P.PDHG_ERR_NUMERIC),  # Inf in A
])
def test_invalid_input_rejected_before_device_work(lib, mutate, status):
    rp, ci, v, b, c = mutate(*_tiny_csr())
    with pytest.raises(P.PDHGError) as ei:
        P.pdhg_create(2, 3, rp, ci, v, b, c)
    assert ei.value.status == status
    assert P.pdhg_last_error(None)


def test_each_host_check_on_its_own(lib):
    """Each check of pdhg_create's host inputs, with the others passing."""
    # A = [[1, 2, 0], [0, 0, 0], [0, 1, 1]]-shaped data for a 3x3 LP
    ci, v = np.array([0, 1, 1, 2], np.int32), np.array([1.0, 2.0, 1.0, 1.0])
    b, c = np.array([3.0, 0.0, 2.0]), np.array([1.0, 1.0, 1.0])
    cases = [
        # row 1 ends before it starts; rows 0 and 2 are well formed on their own
        (np.array([0, 2, 1, 3], np.int64), np.array([0, 1, 2], np.int32), v[:3], b, c, None,
         P.PDHG_ERR_INVALID, "non-decreasing"),
        (np.array([0, 2, 2, 3], np.int64), ci, v, b, c, None, P.PDHG_ERR_INVALID, "row_ptr[m]"),
        (np.array([0, 2, 2, 4], np.int64), np.array([0, 1, -1, 2], np.int32), v, b, c, None,
         P.PDHG_ERR_INVALID, "out of range"),
        (np.array([0, 2, 2, 4], np.int64), ci, v, np.array([3.0, np.nan, 2.0]), c, None,
         P.PDHG_ERR_NUMERIC, "NaN"),
        (np.array([0, 2, 2, 4], np.int64), ci, v, b, c, np.array([0.0, np.inf, 0.0]),
         P.PDHG_ERR_NUMERIC, "NaN"),  # Inf in the warm start
    ]
    for rp, cc, vv, bb, cv, x0, status, msg in cases:
        with pytest.raises(P.PDHGError) as ei:
            P.pdhg_create(3, 3, rp, cc, vv, bb, cv, x0=x0)
        assert ei.value.status == status, (rp, cc, bb, x0)
        assert msg in P.pdhg_last_error(None), (msg, P.pdhg_last_error(None))


def test_bad_sizes_and_options(lib):
    rp, ci, v, b, c = _tiny_csr()
    with pytest.raises(P.PDHGError) as ei:
        P.pdhg_create(0, 3, np.array([0], np.int64), ci[:0], v[:0], b[:0], c)
    assert ei.value.status == P.PDHG_ERR_INVALID
    for bad in (dict(eval_every=0), dict(eps_factor=1.5), dict(pc_alpha=3.0), dict(power_iters=0),
                dict(precision=7), dict(gap_tol=-1.0), dict(feas_polish=2), dict(polish_div=0),
                dict(feas_polish=1, persistent=1), dict(halpern=1, halpern_reflect=1.5), dict(primal_panels=3)):
        with pytest.raises(P.PDHGError) as ei:
            P.pdhg_create(2, 3, rp, ci, v, b, c, opt=P.pdhg_default_options(**bad))
        assert ei.value.status == P.PDHG_ERR_INVALID, bad


def test_null_context_is_safe(lib):
    lib.pdhg_destroy(None)
    assert lib.pdhg_iterate(None, 1, 0.0, None) == P.PDHG_ERR_INVALID
    assert lib.pdhg_kkt(None, 0, None) == P.PDHG_ERR_INVALID
    assert lib.pdhg_snapshot(None, None, None, None, None, None) == P.PDHG_ERR_INVALID


def test_missing_library_fails_loudly(tmp_path):
    """Without libpdhg.so the binding raises on first use: there is no CPU path."""
    pkg = tmp_path / "paper_2510_24429_b300"
    pkg.mkdir()
    for f in ("__init__.py", "pdhg.py", "lpgen.py"):
        (pkg / f).write_text(open(os.path.join(ROOT, "paper_2510_24429_b300", f)).read())
    code = (
        "from paper_2510_24429_b300 import lpgen, pdhg as P\n"
        "lp = lpgen.tiny_lp(0)\n"
        "try:\n"
        "    P.Solver.from_lp(lp)\n"
        "except RuntimeError as e:\n"
        "    print('RAISED', e)\n"
    )
    r = subprocess.run(["python", "-c", code], cwd=tmp_path, capture_output=True, text=True, timeout=300,
                       env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert r.returncode == 0, r.stderr
    assert "RAISED libpdhg.so not built" in r.stdout and str(pkg) in r.stdout, r.stdout


def test_header_and_library_from_plain_c(lib, tmp_path):
    """include/pdhg.h compiles as strict C99 and the library links and runs
    from a C program (tests/c_abi/from_c.c): defaults, host checks, NULL
    safety, and a short solve where a GPU is present."""
    import shutil

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "from_c"
    libdir = os.path.dirname(B.LIB)
    src = os.path.join(ROOT, "tests", "c_abi", "from_c.c")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                        src, "-o", str(exe), "-L", libdir, "-lpdhg", f"-Wl,-rpath,{libdir}", "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr


def test_noalloc_host_checks(lib):
    """pdhg_kkt_noalloc's argument checks run on the host before any device
    call: sizes out of range, NULL arrays, a NULL out and too many blocks are
    INVALID (the pointers below are never dereferenced)."""
    out = P.pdhg_kkt_info()
    fake = C.c_void_p(16)  # never read: every case fails a host check first
    arrays = [fake] * 10

    def call(m, n, arrs=arrays, blocks=0, o=C.byref(out)):
        return lib.pdhg_kkt_noalloc(m, n, *arrs, blocks, None, o)

    for m, n in ((0, 5), (5, 0), (-1, 5), (5, 2 ** 31), (2 ** 31, 5)):
        assert call(m, n) == P.PDHG_ERR_INVALID, (m, n)
        assert "2^31" in P.pdhg_last_error(None)
    for i in range(10):
        arrs = list(arrays)
        arrs[i] = None
        assert call(5, 5, arrs) == P.PDHG_ERR_INVALID, i
        assert "NULL" in P.pdhg_last_error(None)
    assert call(5, 5, blocks=1025) == P.PDHG_ERR_INVALID
    assert call(5, 5, blocks=-1) == P.PDHG_ERR_INVALID
    assert call(5, 5, o=None) == P.PDHG_ERR_INVALID


def test_fp64_rate_host_check(lib):
    assert lib.pdhg_fp64_fma_rate(None, None, None) == P.PDHG_ERR_INVALID
    assert "NULL" in P.pdhg_last_error(None)


def test_checked_library_exports_the_same_symbols():
    """The range-checked build (PDHG_CHECKED) is the same library with checks
    compiled in: it exports every declared entry point."""
    lib = B.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pdhg_\w+)", out))
    assert set(_declared_functions()) <= exported
