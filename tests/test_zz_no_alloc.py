"""The allocation-free KKT entry point (pdhg_kkt_noalloc).

It exists for callers that must not let a library allocate device memory:
programs whose GPU memory is owned by their own pool or framework allocator,
services with a fixed memory budget, and latency-critical code where cudaMalloc
would synchronize the device. Its partial sums live in one static device array
shared by all calls, so these tests call it twice in a row (and with different
block counts, on the current stream, an explicit stream and the legacy default
stream) and check each result against the context-based pdhg_kkt, and check
that a NaN in the point is reported as PDHG_ERR_NUMERIC.

Kept in a file of its own, collected last, so that a run stopping at the first
failure has run every other test before this one.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P

pytestmark = pytest.mark.gpu

FIELDS = ("rp_norm2", "rp_norminf", "rd_norm2", "rd_norminf", "primal_obj", "dual_obj", "gap", "complementarity",
          "rel_p", "rel_d", "rel_gap", "rel_kkt")


@pytest.fixture(scope="module")
def setup():
    import torch

    from paper_2510_24429_b300 import build

    build.build()
    P.load()
    torch.cuda.set_device(0)
    lp = lpgen.generate(3001, 7919, 5, nnz_per_col=5, support=0.3)  # several tiles and a ragged tail
    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    At = sp.csr_matrix(A.T)
    dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")  # noqa: E731
    mats = (dev(A.indptr, torch.int64), dev(A.indices, torch.int32), dev(A.data, torch.float64),
            dev(At.indptr, torch.int64), dev(At.indices, torch.int32), dev(At.data, torch.float64),
            dev(lp.b, torch.float64), dev(lp.c, torch.float64))
    return lp, mats, dev


def _check_against_pdhg_kkt(ref, got):
    for key in FIELDS:
        assert got[key] == pytest.approx(ref[key], rel=1e-8, abs=1e-12), key


def test_noalloc_matches_pdhg_kkt_on_two_calls_in_a_row(setup):
    import torch

    lp, mats, dev = setup
    with P.Solver.from_lp(lp) as sol:
        for _ in range(2):
            sol.iterate(150)
            x, y, _ = sol.solution()
            ref = sol.kkt()
            got = P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, dev(x, torch.float64), dev(y, torch.float64))
            assert got["iteration"] == -1
            _check_against_pdhg_kkt(ref, got)


def test_noalloc_block_counts_agree_and_limit_is_enforced(setup):
    import torch

    lp, mats, dev = setup
    with P.Solver.from_lp(lp) as sol:
        sol.iterate(64)
        x, y, _ = sol.solution()
        ref = sol.kkt()
    xd, yd = dev(x, torch.float64), dev(y, torch.float64)
    for blocks in (1, 1024, 0, 7):
        _check_against_pdhg_kkt(ref, P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, xd, yd, blocks=blocks))
    with pytest.raises(P.PDHGError) as ei:
        P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, xd, yd, blocks=1025)
    assert ei.value.status == P.PDHG_ERR_INVALID
    assert "1024" in P.pdhg_last_error(None)


def test_noalloc_on_explicit_and_legacy_streams(setup):
    import torch

    lp, mats, dev = setup
    with P.Solver.from_lp(lp) as sol:
        sol.iterate(128)
        x, y, _ = sol.solution()
        ref = sol.kkt()
    xd, yd = dev(x, torch.float64), dev(y, torch.float64)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())  # inputs were written on the current stream
    with torch.cuda.stream(side):
        for _ in range(2):
            _check_against_pdhg_kkt(ref, P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, xd, yd, stream=side.cuda_stream))
    torch.cuda.synchronize()
    # stream 0: the legacy default stream, which orders itself after the others
    for _ in range(2):
        _check_against_pdhg_kkt(ref, P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, xd, yd, stream=0))


def test_noalloc_reports_nan_as_numeric(setup):
    """A NaN in y makes rel_d and rel_gap NaN while rel_p stays finite; the
    call must report PDHG_ERR_NUMERIC, not a finite rel_kkt."""
    import torch

    lp, mats, dev = setup
    x = np.zeros(lp.n)
    y = np.zeros(lp.m)
    y[17] = np.nan
    with pytest.raises(P.PDHGError) as ei:
        P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, dev(x, torch.float64), dev(y, torch.float64))
    assert ei.value.status == P.PDHG_ERR_NUMERIC
    # the next call on clean inputs is unaffected by the NaN left in the scratch
    y[17] = 0.0
    got = P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, dev(x, torch.float64), dev(y, torch.float64))
    assert np.isfinite(got["rel_kkt"])


def test_noalloc_wrapper_rejects_wrong_lengths(setup):
    import torch

    lp, mats, dev = setup
    x, y = dev(np.zeros(lp.n), torch.float64), dev(np.zeros(lp.m), torch.float64)
    with pytest.raises(ValueError, match="x has"):
        P.pdhg_kkt_noalloc(lp.m, lp.n, *mats, x[:-1], y)
    with pytest.raises(ValueError, match="a_row_ptr has"):
        P.pdhg_kkt_noalloc(lp.m + 1, lp.n, *mats, x, y)
    with pytest.raises(ValueError, match="same length"):
        P.pdhg_kkt_noalloc(lp.m, lp.n, mats[0], mats[1][:-1], *mats[2:], x, y)
