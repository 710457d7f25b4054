"""Build libpdhg.so in-tree with nvcc for sm_103a (B300)."""
from __future__ import annotations

import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libpdhg.so")
# the range-checked build (PDHG_CHECKED): every matrix unit's extent and rows and
# every gathered column index are checked before use; an index out of range
# sets a device error word (reported as PDHG_ERR_INVALID) and is skipped, so
# nothing traps. For tests on small cases, not for timing.
LIB_CHECKED = os.path.join(HERE, "libpdhg_checked.so")
SOURCES = ["kernels.cu", "stream.cu", "layout.cu", "persistent.cu", "pdhg_api.cu", "kkt_noalloc.cu", "autotune.cu",
           "fp64_rate.cu"]
HEADERS = ["common.cuh", "kernels.cuh", "decide.cuh", "step_ops.cuh"]
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "pdhg.h"))
    files.append(os.path.abspath(__file__))
    return files


def needs_build(lib: str = LIB) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(f) > t for f in _inputs())


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Compile the CUDA sources into paper_2510_24429_b300/libpdhg.so (or,
    with checked=True, the range-checked libpdhg_checked.so)."""
    lib = LIB_CHECKED if checked else LIB
    if not force and not needs_build(lib):
        return lib
    cmd = [
        _nvcc(), ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
        "-Xcompiler", "-fvisibility=hidden", "-I", os.path.join(ROOT, "include"), "-o", lib + ".tmp",
    ]
    if checked:
        cmd += ["-DPDHG_CHECKED=1"]
    if verbose:
        cmd += ["-Xptxas", "-v"]
    cmd += [os.path.join(CSRC, f) for f in SOURCES]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stdout + res.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    import sys

    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
