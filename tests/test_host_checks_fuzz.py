"""pdhg_create's host checks on generated inputs: small CSR matrices, well
formed or with one defect of a chosen kind (row pointers that do not start at
0, do not end at nnz or decrease; a column index out of range, out of order or
repeated; NaN/Inf in A, b or c). Every malformed input gets the status its
defect calls for (INVALID for structure, NUMERIC for non-finite data,
structure first), the checks never read outside the arrays (the process would
not survive), and a well-formed input passes them (it then gets a context on a
GPU, or PDHG_ERR_CUDA without one). The inputs come from a seeded generator,
an equal number per defect kind."""
import numpy as np
import pytest

from paper_2510_24429_b300 import build as B
from paper_2510_24429_b300 import pdhg as P

KINDS = ["none", "rp_first", "rp_last_low", "rp_last_high", "rp_decreasing_only", "rp_interior",
         "col_range", "col_order", "col_duplicate", "val", "b", "c"]
PER_KIND = 40


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()
    P.load()


def expected_status(m, n, rp, ci, v, b, c):
    """The classification written out from the CSR rules of the C ABI."""
    nnz = len(ci)
    if rp[0] != 0 or rp[m] != nnz or np.any(np.diff(rp) < 0):
        return P.PDHG_ERR_INVALID
    for i in range(m):
        row = ci[rp[i]:rp[i + 1]].astype(np.int64)
        if np.any(row < 0) or np.any(row >= n) or np.any(np.diff(row) <= 0):
            return P.PDHG_ERR_INVALID
    if not (np.all(np.isfinite(v)) and np.all(np.isfinite(b)) and np.all(np.isfinite(c))):
        return P.PDHG_ERR_NUMERIC
    return P.PDHG_OK


def make_lp(rng, kind):
    m = int(rng.integers(3 if kind == "rp_decreasing_only" else 1, 7))
    if kind == "rp_decreasing_only":
        # columns increasing along the whole entry array, so that rows that
        # overlap after the defect are still in order: the decrease is the only flaw
        lens = rng.integers(1, 3, size=m)
        nnz = int(lens.sum())
        n = nnz + int(rng.integers(0, 3))
        ci = np.sort(rng.choice(n, size=nnz, replace=False)).astype(np.int32)
    else:
        n = int(rng.integers(1, 7))
        lo = 2 if kind in ("col_order", "col_duplicate") and n >= 2 else (1 if kind != "none" else 0)
        rows = [np.sort(rng.choice(n, size=int(rng.integers(min(lo, n), n + 1)), replace=False)) for _ in range(m)]
        lens = np.array([len(r) for r in rows])
        ci = np.concatenate(rows).astype(np.int32) if lens.sum() else np.zeros(0, np.int32)
        nnz = int(lens.sum())
    rp = np.zeros(m + 1, np.int64)
    rp[1:] = np.cumsum(lens)
    v = rng.uniform(-10, 10, nnz)
    b, c = rng.uniform(-10, 10, m), rng.uniform(-10, 10, n)
    bad = [np.nan, np.inf, -np.inf][int(rng.integers(0, 3))]
    if kind == "rp_first":
        rp[0] = [1, -1][int(rng.integers(0, 2))]
    elif kind == "rp_last_low" and nnz:
        rp[m] -= 1
    elif kind == "rp_last_high":
        rp[m] += int(rng.choice([1, 2, 50]))
    elif kind == "rp_decreasing_only":
        i = int(rng.integers(1, m - 1))  # interior pointer, rows i-1 and i
        rp[i] = rp[i + 1] + 1  # row i-1 runs on into row i+1's first entry; row i ends before it starts
    elif kind == "rp_interior" and m >= 2:
        i = int(rng.integers(1, m))
        rp[i] += int(rng.choice([-3, -1, 1, 3]))
    elif kind == "col_range" and nnz:
        ci[int(rng.integers(0, nnz))] = int(rng.choice([-1, -7, n, n + 3, 2**31 - 1]))
    elif kind in ("col_order", "col_duplicate"):
        long_rows = [i for i in range(m) if rp[i + 1] - rp[i] >= 2]
        if long_rows:
            i = long_rows[int(rng.integers(0, len(long_rows)))]
            k = int(rp[i]) + int(rng.integers(0, rp[i + 1] - rp[i] - 1))
            if kind == "col_order":
                ci[k], ci[k + 1] = ci[k + 1], ci[k]
            else:
                ci[k + 1] = ci[k]
    elif kind == "val" and nnz:
        v[int(rng.integers(0, nnz))] = bad
    elif kind == "b":
        b[int(rng.integers(0, m))] = bad
    elif kind == "c":
        c[int(rng.integers(0, n))] = bad
    return m, n, rp, ci, v, b, c


@pytest.mark.parametrize("kind", KINDS)
def test_host_checks_classify_generated_inputs(kind):
    rng = np.random.default_rng(KINDS.index(kind))
    seen = set()
    for _ in range(PER_KIND):
        m, n, rp, ci, v, b, c = make_lp(rng, kind)
        if kind == "rp_decreasing_only":
            assert np.any(np.diff(rp) < 0) and rp[0] == 0 and rp[m] == len(ci)
        want = expected_status(m, n, rp, ci, v, b, c)
        seen.add(want)
        try:
            ctx = P.pdhg_create(m, n, rp, ci, v, b, c)
        except P.PDHGError as e:
            got = e.status
        else:
            P.pdhg_destroy(ctx)
            got = P.PDHG_OK
        if want == P.PDHG_OK:
            assert got in (P.PDHG_OK, P.PDHG_ERR_CUDA), (kind, got, P.pdhg_last_error(None))
        else:
            assert got == want, (kind, want, got, P.pdhg_last_error(None), rp, ci)
    # every defect kind produced its defect in most draws
    if kind == "none":
        assert seen == {P.PDHG_OK}
    else:
        assert (P.PDHG_ERR_NUMERIC if kind in ("val", "b", "c") else P.PDHG_ERR_INVALID) in seen
