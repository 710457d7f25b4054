"""Panel-tiled primal half-step (option primal_panels): y staged in shared
memory panel by panel, per-(column, panel) partial sums added per column for
the long columns (at least long_row_min entries); the short columns take the
direct step in the same half-step. The tiny LP's columns all have 5 entries,
so long_row_min=4 puts every column in the panels; a Zipf-shaped LP mixes both.

The per-column sums are grouped by panel, so results differ from the direct
step at rounding level only; against the oracle the same bars as the parity
tests hold (1e-10 after 100 iterations, identical decision traces, converged
objectives within 1e-7 of f*). Small panel heights force many panels, partial
panels and segments of every length on the tiny LP; the large LP runs with
the shared-memory-sized panels the option picks by itself."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, TINY_PLAIN, assert_iterates_close, compare_traces, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _solvers(lp, engine_opts, **opts):
    oopt = O.Options(**opts)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    return orc, P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, **engine_opts, **copts)


@pytest.mark.parametrize("rows", [1, 7, 32, 200])
def test_plain_100_iterations_match_oracle(tiny_lp, rows):
    orc, sol = _solvers(tiny_lp, dict(primal_panels=1, panel_rows=rows, long_row_min=4), **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)


def test_panels_agree_with_direct_step(tiny_lp):
    _, sp = _solvers(tiny_lp, dict(primal_panels=1, panel_rows=32, long_row_min=4), **TINY_PLAIN)
    _, sd = _solvers(tiny_lp, dict(primal_panels=0), **TINY_PLAIN)
    sp.iterate(2000)
    sd.iterate(2000)
    for a, b in zip(sp.solution(), sd.solution()):
        assert rel_err(a, b) <= 1e-12


def test_restarted_run_matches_oracle(tiny_lp):
    orc, sol = _solvers(tiny_lp, dict(primal_panels=1, panel_rows=32, long_row_min=4))
    orc.run(100)
    sol.iterate(100)
    assert [r["kind"] for r in sol.trace()] == [r.kind for r in orc.trace] != [0]
    assert_iterates_close(sol, orc, 1e-10)
    assert_iterates_close(sol, orc, 1e-10, P.PDHG_AVERAGE)
    orc2, sol2 = _solvers(tiny_lp, dict(primal_panels=1, panel_rows=32, long_row_min=4))
    orc2.run(3000, 1e-10)
    sol2.iterate(3000, 1e-10)
    assert compare_traces(sol2.trace(), orc2.trace) >= 20


def test_converges_to_known_optimum(tiny_lp):
    _, sol = _solvers(tiny_lp, dict(primal_panels=1, panel_rows=50, long_row_min=4))
    st, _ = sol.iterate(200000, 1e-8)
    assert st == P.PDHG_OK
    k = sol.kkt()
    assert k["rel_kkt"] <= 1e-8
    assert k["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=1e-7)
    x, _, _ = sol.solution()
    assert rel_err(x, tiny_lp.x_star) <= 1e-6


@pytest.mark.parametrize("prec", [P.PDHG_FP32, P.PDHG_MIXED])
def test_fp32_and_mixed_with_panels(tiny_lp, prec):
    with P.Solver.from_lp(tiny_lp, precision=prec, primal_panels=1, panel_rows=40, long_row_min=4) as sp, \
            P.Solver.from_lp(tiny_lp, precision=prec, primal_panels=0) as sd:
        sp.iterate(640)
        sd.iterate(640)
        xp, xd = sp.solution()[0], sd.solution()[0]
        assert rel_err(xp, xd) <= 1e-4  # FP32 sums grouped differently
        if prec == P.PDHG_MIXED:
            st, _ = sp.iterate(200000, 1e-8)
            assert st == P.PDHG_OK
            assert sp.kkt()["primal_obj"] == pytest.approx(tiny_lp.f_star, rel=1e-7)


def test_adjoint_with_panels(tiny_lp):
    """The recorded forward and the reverse pass's recompute both use the
    panel-tiled step, so the gradient matches the direct engine's."""
    base = dict(restarts=0, primal_weight=0, record_for_backward=1, checkpoint_every=7)
    rng = np.random.default_rng(5)
    gx = rng.standard_normal(tiny_lp.n)
    grads = []
    for opts in (dict(primal_panels=1, panel_rows=16, long_row_min=4), dict(primal_panels=0, long_row_min=4)):
        with P.Solver.from_lp(tiny_lp, **base, **opts) as s:
            s.iterate(60)
            grads.append(s.backward(gx))
    for a, b in zip(grads[0], grads[1]):
        assert rel_err(a, b) <= 1e-11


def test_edge_shapes():
    for m, n, k in ((1, 1, 1), (1, 9, 1), (9, 1, 1), (5, 40, 3)):
        lp = lpgen.generate(m, n, 11, nnz_per_col=k, support=0.3)
        for lrm in (1, 2, 128):  # every column, the longer ones, none in the panels
            orc, sol = _solvers(lp, dict(primal_panels=1, panel_rows=2, long_row_min=lrm), **TINY_PLAIN)
            orc.run(50)
            sol.iterate(50)
            assert_iterates_close(sol, orc, 1e-10)


@pytest.mark.parametrize("prec", [P.PDHG_FP64, P.PDHG_FP32])
def test_long_and_short_columns_mixed(prec):
    """Zipf-shaped column counts: columns with >= 32 entries in the panels, the
    rest in the direct step of the same half-step; against the oracle (FP64)
    or the direct FP32 engine."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3, fp32_values=True)
    eng = dict(primal_panels=1, panel_rows=256, long_row_min=32, precision=prec)
    if prec == P.PDHG_FP64:
        orc, sol = _solvers(lp, eng, **TINY_PLAIN)
        orc.run(100)
        assert sol.iterate(100) == (P.PDHG_OK, 100)
        assert_iterates_close(sol, orc, 1e-10)
        orc2, sol2 = _solvers(lp, eng)
        orc2.run(2000, 1e-9)
        sol2.iterate(2000, 1e-9)
        assert compare_traces(sol2.trace(), orc2.trace) >= 10
    else:
        with P.Solver.from_lp(lp, **eng) as sp, P.Solver.from_lp(lp, precision=prec, primal_panels=0) as sd:
            sp.iterate(640)
            sd.iterate(640)
            assert rel_err(sp.solution()[0], sd.solution()[0]) <= 1e-4


@pytest.mark.parametrize("prec", [P.PDHG_FP64, P.PDHG_FP32])
def test_balanced_panel_heights(prec):
    """panel_balance = 1: panel heights cut where the long columns' entries
    fill a whole number of the panel pass's blocks (panel_rows the tallest
    allowed). Against the oracle at 1e-10 after 100 iterations (FP64) and
    against equal heights at rounding level (FP32); the panel count is
    reported in the info."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3, fp32_values=True)
    for rows in (64, 256):
        eng = dict(primal_panels=1, panel_rows=rows, long_row_min=32, precision=prec)
        if prec == P.PDHG_FP64:
            orc, sol = _solvers(lp, dict(eng, panel_balance=1), **TINY_PLAIN)
            with sol:
                assert sol.info()["panels"] >= -(-lp.m // rows)
                orc.run(100)
                assert sol.iterate(100) == (P.PDHG_OK, 100)
                assert_iterates_close(sol, orc, 1e-10)
        else:
            out = []
            for bal in (0, 1):
                with P.Solver.from_lp(lp, panel_balance=bal, **eng) as s:
                    assert s.info()["panels"] >= -(-lp.m // rows)
                    assert s.iterate(640) == (P.PDHG_OK, 640)
                    out.append(s.solution()[0])
            assert rel_err(out[0], out[1]) <= 1e-4
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(lp, primal_panels=1, panel_balance=2)


def test_option_checks(tiny_lp):
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(tiny_lp, primal_panels=1, panel_rows=28161)
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(tiny_lp, primal_panels=2)
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(tiny_lp, primal_panels=1, persistent=1)
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny_lp, tiny_lp], primal_panels=1)


def test_halpern_fp64_with_panels():
    """The reflected Halpern form in FP64 with the panel-tiled step (anchor =
    last restart point in the combine and in the short-column step) against
    the oracle's Halpern variant."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3)
    eng = dict(primal_panels=1, panel_rows=256, long_row_min=32, halpern=1)
    orc, sol = _solvers(lp, eng, halpern=True, **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)
    orc2, sol2 = _solvers(lp, eng, halpern=True)
    orc2.run(1500, 1e-9)
    sol2.iterate(1500, 1e-9)
    assert compare_traces(sol2.trace(), orc2.trace) >= 10


@pytest.mark.parametrize("prec", [P.PDHG_FP64, P.PDHG_FP32, P.PDHG_MIXED])
@pytest.mark.parametrize("halpern", [0, 1])
def test_hot_columns_dual_step_is_bit_identical(prec, halpern):
    """The dual step that stages xbar's first entries (the longest columns) in
    shared memory gathers the same values in the same order as the direct
    step, so whole restarted runs are bit-identical: a staged part smaller
    than, and one larger than, the vector (every column staged), in FP64,
    FP32 and the mixed form (whose FP64 phase stages at most half as many)."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3, fp32_values=True)
    eng = dict(primal_panels=1, panel_rows=256, long_row_min=32, precision=prec, halpern=halpern,
               polish_switch=1e-4)
    with P.Solver.from_lp(lp, **eng) as ref:
        ref.iterate(1500, 1e-7)
        want = ref.solution(), [(r["iteration"], r["kind"], r["omega"]) for r in ref.trace()]
    for hot in (1000, 20000, 56320):  # 1, 2 and 3 resident blocks per SM (FP32; FP64 stages half)
        with P.Solver.from_lp(lp, dual_hot_cols=hot, **eng) as sol:
            sol.iterate(1500, 1e-7)
            got = sol.solution(), [(r["iteration"], r["kind"], r["omega"]) for r in sol.trace()]
        for a, b in zip(got[0], want[0]):
            np.testing.assert_array_equal(a, b)
        assert got[1] == want[1]
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(lp, dual_hot_cols=56321)


@pytest.mark.parametrize("panels", [0, 1])
def test_singleton_order_matches_oracle(panels):
    """Columns with one entry numbered by the row of that entry (option
    singleton_order): a renumbering only, so the iterates agree with the
    oracle at 1e-10 after 100 plain iterations and restarted runs take the
    same decisions; checked with and without the panel-tiled primal step."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3)
    assert int((np.bincount(lp.col_idx, minlength=lp.n) == 1).sum()) > lp.n // 2
    eng = dict(primal_panels=panels, panel_rows=256, long_row_min=32, singleton_order=1)
    orc, sol = _solvers(lp, eng, **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)
    orc2, sol2 = _solvers(lp, eng)
    orc2.run(1500, 1e-9)
    sol2.iterate(1500, 1e-9)
    assert compare_traces(sol2.trace(), orc2.trace) >= 10
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(lp, singleton_order=2)



@pytest.mark.parametrize("pmin", [4, 12])
def test_panel_min_len_matches_oracle(pmin):
    """Shorter columns in the panels (option panel_min_len below long_row_min:
    whole units of short columns go to the panels, the rest to the direct
    step): the same iterates as the oracle at 1e-10."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3)
    eng = dict(primal_panels=1, panel_rows=256, long_row_min=32, panel_min_len=pmin)
    orc, sol = _solvers(lp, eng, **TINY_PLAIN)
    orc.run(100)
    assert sol.iterate(100) == (P.PDHG_OK, 100)
    assert_iterates_close(sol, orc, 1e-10)
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(lp, panel_min_len=-1)


def test_mixed_fp32_phase_uses_the_fp32_layout():
    """PDHG_MIXED keeps an FP32-tuned panel layout for its FP32 phase (shorter
    columns in the panels, twice the rows per panel) beside the FP64 one; it
    is the layout a PDHG_FP32 context builds, so until the switch to FP64 the
    two contexts' iterates are bit-identical. After the switch the FP64 phase
    (on the FP64 layout) still reaches the known optimum."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3, fp32_values=True)
    eng = dict(primal_panels=1, long_row_min=64)
    # the mixed form's FP32 phase runs on corrections to its restart point
    # (refine32, its default); the FP32 context is asked for the same
    with P.Solver.from_lp(lp, precision=P.PDHG_MIXED, polish_switch=1e-30, **eng) as mx, \
            P.Solver.from_lp(lp, precision=P.PDHG_FP32, refine32=1, **eng) as f32:
        mx.iterate(640)
        f32.iterate(640)
        assert mx.info()["precision_now"] == P.PDHG_FP32
        for a, b in zip(mx.solution(), f32.solution()):
            np.testing.assert_array_equal(a, b)
    with P.Solver.from_lp(lp, precision=P.PDHG_MIXED, polish_switch=1e-5, **eng) as mx:
        st, _ = mx.iterate(100_000, 1e-8)
        assert st == P.PDHG_OK and mx.info()["polish_started_at"] > 0
        assert mx.kkt()["primal_obj"] == pytest.approx(lp.f_star, rel=1e-7)


@pytest.mark.parametrize("extra", [dict(), dict(halpern=1, restart_scheme=1), dict(precision=P.PDHG_FP32),
                                   dict(precision=P.PDHG_MIXED, polish_switch=1e-4),
                                   dict(halpern=1, kernel_timing=1)])
def test_overlapped_short_step_is_bit_identical(extra):
    """panel_overlap (the default for FP32 steps): the short-column step starts as the panel
    pass's blocks finish and only its combine blocks wait for the partial sums.
    Every sum keeps its order, so restarted runs (graph-replayed, or direct
    launches with kernel timing) equal the sequential launches' bit for bit."""
    lp = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                        support=0.3, fp32_values=True)
    eng = dict(primal_panels=1, panel_rows=256, long_row_min=32, **extra)
    out = []
    for overlap in (0, 1):
        with P.Solver.from_lp(lp, panel_overlap=overlap, **eng) as s:
            s.iterate(1280, 1e-12)
            out.append((s.solution(), [(r["iteration"], r["kind"], r["omega"]) for r in s.trace()]))
    for a, b in zip(out[0][0], out[1][0]):
        np.testing.assert_array_equal(a, b)
    assert out[0][1] == out[1][1]
