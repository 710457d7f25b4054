"""Option refine32: FP32 phases on FP32 corrections to an FP64 restart point.

A restart moves the FP64 reference to the new point and recomputes, in FP64,
the FP32 iteration's costs (chat - Ahat^T y_r, bhat - Ahat x_r) and the lower
bounds -x_r of the primal corrections. Checked here:
- without restarts the reference stays the zero start point, the costs are
  chat and bhat rounded and the bounds 0, so every iterate equals the plain
  FP32 form's bit for bit;
- with restarts, the FP32 and mixed forms (PDLP style, reflected Halpern,
  cuPDLP+) reach rel. KKT 1e-8 and the objective of the generator's known
  optimum within 1e-7 (relative to 1 + |f*|), where the plain FP32 iteration
  stalls above that, and the primal solution approaches the unique x*;
- the last restart point is held in FP64 and the iterates keep x >= 0;
- the option's checks."""
import numpy as np
import pytest

from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import TINY_PLAIN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.fixture(scope="module")
def zipf_lp():
    return lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                          support=0.3, fp32_values=True)


FORMS = {"pdlp": {}, "halpern": dict(halpern=1), "cupdlp_plus": dict(halpern=1, restart_scheme=1)}


@pytest.mark.parametrize("panels", [0, 1])
def test_without_restarts_equals_plain_fp32(zipf_lp, panels):
    plain = dict(TINY_PLAIN, precision=P.PDHG_FP32, primal_panels=panels, panel_rows=256, long_row_min=32)
    out = []
    for refine in (0, 1):
        with P.Solver.from_lp(zipf_lp, refine32=refine, **plain) as s:
            assert s.iterate(300) == (P.PDHG_OK, 300)
            assert s.info()["refine32"] == refine
            out.append(s.solution())
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("form", sorted(FORMS))
@pytest.mark.parametrize("prec", [P.PDHG_FP32, P.PDHG_MIXED])
def test_reaches_1e8(zipf_lp, form, prec):
    """polish_switch = 0: the mixed form switches to FP64 only on a stall, so
    both precisions run the refined FP32 iteration to the tolerance."""
    opts = dict(FORMS[form], precision=prec, refine32=1, polish_switch=0.0, primal_panels=1, panel_rows=256,
                long_row_min=32)
    with P.Solver.from_lp(zipf_lp, **opts) as s:
        st, done = s.iterate(200_000, 1e-8)
        k = s.kkt()
        info = s.info()
        x, _, _ = s.solution()
    assert st == P.PDHG_OK, (done, k["rel_kkt"])
    assert k["rel_kkt"] <= 1e-8
    assert abs(k["primal_obj"] - zipf_lp.f_star) <= 1e-7 * (1 + abs(zipf_lp.f_star))
    assert abs(k["dual_obj"] - zipf_lp.f_star) <= 1e-7 * (1 + abs(zipf_lp.f_star))
    if form == "pdlp":  # the reflected Halpern iterate itself may leave x >= 0 (by rounding-sized amounts)
        assert np.all(x >= 0.0)
    print(f"{form} precision {prec}: {done} iterations, FP64 from {info['polish_started_at']}")


def test_plain_fp32_stalls_where_refined_does_not(zipf_lp):
    """The same iteration budget: the plain FP32 form does not reach 1e-8 (its
    iterate's rounding floors the residuals), the refined one does."""
    opts = dict(halpern=1, restart_scheme=1, precision=P.PDHG_FP32, primal_panels=1, panel_rows=256,
                long_row_min=32)
    with P.Solver.from_lp(zipf_lp, refine32=1, **opts) as s:
        assert s.iterate(60_000, 1e-8)[0] == P.PDHG_OK
        used = s.info()["iterations"]
    with P.Solver.from_lp(zipf_lp, **opts) as s:
        st, _ = s.iterate(2 * used, 1e-8)
        assert st == P.PDHG_ERR_NOT_CONVERGED and s.kkt()["rel_kkt"] > 1e-8


def test_points_consistent(zipf_lp):
    """Mid-solve (FP32 phase, after restarts): the last restart point is held in
    FP64 (not an FP32 number in general) and is primal feasible in sign (the
    reflected Halpern iterate itself need not be); a scheduled snapshot lands."""
    with P.Solver.from_lp(zipf_lp, precision=P.PDHG_MIXED, refine32=1, polish_switch=0.0, halpern=1,
                          restart_scheme=1, snapshot_every=640) as s:
        s.iterate(1280)
        info = s.info()
        assert info["restarts"] >= 2 and info["precision_now"] == P.PDHG_FP32
        xr, _, _ = s.solution(P.PDHG_LAST_RESTART)
        assert np.any(xr.astype(np.float32).astype(np.float64) != xr)
        assert np.all(xr >= 0.0)  # a restart point is a PDHG step's output: projected
        snap = s.snapshot()
        assert snap["iteration"] == 1280 and np.all(snap["z"] >= 0.0)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_tiny_lp(tiny_lp, form):
    with P.Solver.from_lp(tiny_lp, precision=P.PDHG_MIXED, refine32=1, polish_switch=0.0, **FORMS[form]) as s:
        assert s.iterate(200_000, 1e-8)[0] == P.PDHG_OK
        k = s.kkt()
    assert abs(k["primal_obj"] - tiny_lp.f_star) <= 1e-7 * (1 + abs(tiny_lp.f_star))


def test_option_checks(tiny_lp):
    for opts in (dict(refine32=2), dict(refine32=-2), dict(refine32=1),
                 dict(refine32=1, precision=P.PDHG_FP32, record_for_backward=1, restarts=0, primal_weight=0),
                 dict(precision=P.PDHG_MIXED, polish_switch=-0.5)):
        with pytest.raises(P.PDHGError):
            P.Solver.from_lp(tiny_lp, **opts)
    with pytest.raises(P.PDHGError):
        P.BatchSolver([tiny_lp, tiny_lp], precision=P.PDHG_MIXED, refine32=1)
    # the default: on for PDHG_MIXED, off for PDHG_FP32; with the streamed steps too
    for prec, want in ((P.PDHG_MIXED, 1), (P.PDHG_FP32, 0), (P.PDHG_FP64, 0)):
        with P.Solver.from_lp(tiny_lp, precision=prec) as s:
            assert s.info()["refine32"] == want
    with P.Solver.from_lp(tiny_lp, precision=P.PDHG_FP32, refine32=1, stream_steps=1) as s:
        assert (s.info()["refine32"], s.info()["stream_steps"]) == (1, 1)


@pytest.mark.parametrize("form", sorted(FORMS))
def test_follows_the_fp64_trajectory(zipf_lp, form):
    """The refined FP32 iteration moves like the FP64 one: the same restart
    decisions (iteration, candidate kind) at the first 30 evaluations, primal
    weights within 1e-4 and relative KKT errors within 1e-3 of FP64's."""
    opts = dict(FORMS[form], primal_panels=1, panel_rows=256, long_row_min=32)
    with P.Solver.from_lp(zipf_lp, precision=P.PDHG_FP64, **opts) as s:
        s.iterate(1920, 1e-12)
        ref = s.trace()
    with P.Solver.from_lp(zipf_lp, precision=P.PDHG_MIXED, refine32=1, polish_switch=0.0, **opts) as s:
        s.iterate(1920, 1e-12)
        got = s.trace()
        assert s.info()["precision_now"] == P.PDHG_FP32
    assert len(ref) >= 20 and len(got) == len(ref)
    for a, b in zip(got, ref):
        assert (a["iteration"], a["kind"], a["candidate"]) == (b["iteration"], b["kind"], b["candidate"])
        # the PID weight (cuPDLP+) takes logarithms of the restart moves: 1.3e-5 measured
        assert abs(a["omega"] - b["omega"]) <= 1e-4 * abs(b["omega"])
        # the first evaluations' corrections are as large as the iterate itself
        # (the reference starts at 0): their FP32 rounding moves rel_kkt by up
        # to ~2e-4 relative (measured); later ones are far closer
        assert abs(a["rel_kkt"] - b["rel_kkt"]) <= 1e-3 * b["rel_kkt"] + 1e-12
