"""Streamed step kernels (option stream_steps): every warp fills a ring of
shared-memory slots with bulk copies (TMA) of its matrix pieces and of its
rows of the step's vectors, and issues only the gathers from registers.

The kernels perform the direct step kernels' arithmetic in the same order, so
every result must be bit-identical to the engine without the option: the
iterates after plain and restarted runs, the decision traces, the iteration
counts. The cases cover both half-steps in every form the engine runs (PDLP
style with averages, the reflected Halpern form, the cuPDLP+ restarts, FP32,
the refined FP32 iteration on corrections, the mixed form and its FP64 phase
on FP32 values), with and without the
panel-tiled primal step, long rows in A and A^T (warp-per-row pieces across
several slots), slices of 1, 2 and 4 rows per thread, several ring shapes, and
degenerate shapes. Agreement with the oracle then follows from the direct
engine's parity tests; one case checks it directly."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, TINY_PLAIN, assert_iterates_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.fixture(scope="module")
def zipf_lp():
    # Zipf-shaped column counts (columns of up to a few hundred entries), FP32
    # values so that the mixed form's FP64 phase reads the FP32 copies
    return lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                          support=0.3, fp32_values=True)


def _run(lp, iters, tol=0.0, **opts):
    with P.Solver.from_lp(lp, **opts) as s:
        st, done = s.iterate(iters, tol)
        out = {"status": st, "done": done, "info": s.info(), "trace": s.trace()}
        for which in (P.PDHG_CURRENT, P.PDHG_AVERAGE, P.PDHG_LAST_RESTART):
            out[which] = s.solution(which)
        out["kkt"] = s.kkt()
    return out


def _assert_identical(a, b):
    assert (a["status"], a["done"]) == (b["status"], b["done"])
    for which in (P.PDHG_CURRENT, P.PDHG_AVERAGE, P.PDHG_LAST_RESTART):
        for u, v in zip(a[which], b[which]):
            assert np.array_equal(u.view(np.uint64), v.view(np.uint64)), which
    assert a["trace"] == b["trace"]
    for key in ("iterations", "restarts", "omega", "tau", "sigma", "polish_started_at"):
        assert a["info"][key] == b["info"][key], key


FORMS = {
    "fp64": {},
    "fp64_halpern": dict(halpern=1),
    "cupdlp_plus": dict(halpern=1, restart_scheme=1),
    "fp32": dict(precision=P.PDHG_FP32),
    "fp32_halpern": dict(precision=P.PDHG_FP32, halpern=1),
    "fp32_refined": dict(precision=P.PDHG_FP32, refine32=1),
    "fp32_refined_halpern": dict(precision=P.PDHG_FP32, refine32=1, halpern=1, restart_scheme=1),
    "mixed": dict(precision=P.PDHG_MIXED, polish_switch=1e-3),
    "mixed_halpern": dict(precision=P.PDHG_MIXED, polish_switch=1e-3, halpern=1),
    "fp64_values32": dict(values32=1),
    "fp64_values32_halpern": dict(values32=1, halpern=1, restart_scheme=1),
}


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("panels", [1, 0])
def test_identical_to_direct_kernels(zipf_lp, form, panels):
    """Restarted runs of 1280 iterations (20 evaluations) on the Zipf LP: with
    panels the long columns (>= 32 entries) take the panel pass and the
    streamed launch combines them; without, they are long rows of A^T in the
    streamed launch (pieces over several slots)."""
    opts = dict(FORMS[form], primal_panels=panels, panel_rows=256, long_row_min=32)
    ref = _run(zipf_lp, 1280, 1e-12, **opts)
    got = _run(zipf_lp, 1280, 1e-12, stream_steps=1, **opts)
    assert got["info"]["stream_steps"] == 1 and ref["info"]["stream_steps"] == 0
    _assert_identical(got, ref)
    if form.startswith("mixed"):
        assert got["info"]["polish_started_at"] > 0  # both phases ran


@pytest.mark.parametrize("rpt", [1, 2, 4])
@pytest.mark.parametrize("lrm", [4, 8, 128])
def test_tiny_lp_slices_and_long_rows(tiny_lp, rpt, lrm):
    """The tiny LP (5 entries per column, ~12 per row): long_row_min 4 or 8
    makes long rows of A (and with 4 of A^T); slices of 1, 2 or 4 rows per
    thread. Plain fixed-step runs and restarted runs."""
    for extra in (dict(TINY_PLAIN), {}):
        opts = dict(extra, rows_per_thread=rpt, long_row_min=lrm)
        _assert_identical(_run(tiny_lp, 700, **opts), _run(tiny_lp, 700, stream_steps=1, **opts))


@pytest.mark.parametrize("shape", [(1, 2), (3, 8), (16, 2), (5, 5)])
def test_ring_shapes(zipf_lp, shape):
    """Warps per block and slots per warp change how the jobs are dealt out and
    how far ahead they are issued, never the result (FP32 and the FP64 phase of
    the mixed form, which take the most and the fewest warps)."""
    warps, depth = shape
    for prec in (P.PDHG_FP32, P.PDHG_MIXED):
        opts = dict(precision=prec, polish_switch=1e-3, primal_panels=1, panel_rows=256, long_row_min=32)
        # slot bytes: 512 (index + value bytes) + 544 vector bytes + an mbarrier;
        # the FP64 phase on FP32 values takes 8720 bytes per slot
        if prec == P.PDHG_MIXED and warps * depth * 8720 > 227 * 1024 - 256:
            continue  # more shared memory than a block has (rejected, see test_option_checks)
        ref = _run(zipf_lp, 640, 1e-12, **opts)
        got = _run(zipf_lp, 640, 1e-12, stream_steps=1, stream_warps=warps, stream_depth=depth, **opts)
        _assert_identical(got, ref)


def test_matches_oracle(tiny_lp):
    """100 plain FP64 iterations against the oracle at the parity bar (1e-10)."""
    oopt = O.Options(**TINY_PLAIN)
    orc = O.Oracle(tiny_lp.m, tiny_lp.n, tiny_lp.row_ptr, tiny_lp.col_idx, tiny_lp.val, tiny_lp.b, tiny_lp.c, oopt)
    orc.run(100)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    with P.Solver.from_lp(tiny_lp, stream_steps=1, **copts) as sol:
        assert sol.iterate(100) == (P.PDHG_OK, 100)
        assert_iterates_close(sol, orc, 1e-10)


def test_edge_shapes():
    for m, n, k in ((1, 1, 1), (1, 9, 1), (9, 1, 1), (5, 40, 3), (70, 3, 2)):
        lp = lpgen.generate(m, n, 11, nnz_per_col=k, support=0.3)
        for lrm in (1, 2, 128):
            for panels in (0, 1):
                opts = dict(TINY_PLAIN, long_row_min=lrm, primal_panels=panels, panel_rows=2)
                _assert_identical(_run(lp, 60, **opts), _run(lp, 60, stream_steps=1, **opts))


def test_option_checks(tiny_lp):
    bad = (dict(stream_steps=2), dict(stream_steps=1, stream_depth=1), dict(stream_steps=1, stream_depth=9),
           dict(stream_steps=1, stream_warps=17), dict(stream_steps=1, stream_warps=16, stream_depth=8),
           dict(stream_steps=1, persistent=1), dict(stream_steps=1, dual_hot_cols=64))
    for opts in bad:
        with pytest.raises(P.PDHGError):
            P.Solver.from_lp(tiny_lp, **opts)
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny_lp, tiny_lp], stream_steps=1)
