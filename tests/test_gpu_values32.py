"""FP64 steps on FP32 copies of A's unscaled values (option values32).

When every value of A is an FP32 number (the mixed-precision workload's
generator rounds A to FP32 so that every precision solves the same LP), the
FP64 steps can stream 4-byte values with no loss: the kernels read A exactly,
multiply in FP64, and apply the scaling per row and column (Ahat xbar =
D_r (A (D_c xbar))). The iterates then differ from the oracle's, which
multiplies by the scaled FP64 matrix, only in the rounding of each product,
so they meet the same 1e-10 bar as the scaled FP64 path over restarted runs
(PDLP-style, reflected Halpern, and the fixed-point residual scheme), with the
panel-tiled and the direct primal step."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, assert_iterates_close, compare_traces

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.fixture(scope="module")
def zipf32():
    """Zipf-shaped columns (some long enough for the panels and the warp-per-row
    units) with values rounded to FP32."""
    return lpgen.generate(3000, 9000, 5, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                          support=0.3, fp32_values=True)


FORMS = {
    "pdlp": ({}, {}),
    "halpern": (dict(halpern=True), dict(halpern=1)),
    "fixed_point": (dict(halpern=True, restart_scheme=1), dict(halpern=1, restart_scheme=1)),
}
ENGINES = {"direct": dict(primal_panels=0), "panels": dict(primal_panels=1, panel_rows=512, long_row_min=32)}


def _pair(lp, form, engine):
    oform, cform = FORMS[form]
    oopt = O.Options(**oform)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, values32=1, **cform, **ENGINES[engine],
                   **copts)
    return orc, sol


@pytest.mark.parametrize("engine", sorted(ENGINES))
@pytest.mark.parametrize("form", sorted(FORMS))
def test_restarted_iterates_match_oracle(zipf32, form, engine):
    """192 iterations (three evaluations with restart decisions and primal
    weight updates): iterates and decisions as the oracle's."""
    orc, sol = _pair(zipf32, form, engine)
    with sol:
        assert sol.info()["values32"] == 1
        orc.run(192)
        assert sol.iterate(192) == (P.PDHG_OK, 192)
        tr = sol.trace()
        assert compare_traces(tr, orc.trace) == len(orc.trace) == 3
        for g, o in zip(tr, orc.trace):
            assert g["omega"] == pytest.approx(o.omega, rel=1e-10)
        assert_iterates_close(sol, orc, 1e-10)
        assert_iterates_close(sol, orc, 1e-10, P.PDHG_LAST_RESTART)
        if form == "pdlp":
            assert_iterates_close(sol, orc, 1e-10, P.PDHG_AVERAGE)


def test_matches_the_scaled_fp64_path(zipf32):
    """Against the scaled FP64 path of this library over 2,000 restarted
    iterations: the same decisions, iterates within 1e-10."""
    lp = zipf32
    kw = dict(primal_panels=1, panel_rows=512, long_row_min=32)
    with P.Solver.from_lp(lp, values32=1, **kw) as u, P.Solver.from_lp(lp, values32=0, **kw) as v:
        assert u.info()["values32"] == 1 and v.info()["values32"] == 0
        u.iterate(2000)
        v.iterate(2000)
        tu, tv = u.trace(), v.trace()
        assert [(r["iteration"], r["kind"], r["candidate"]) for r in tu] == \
            [(r["iteration"], r["kind"], r["candidate"]) for r in tv]
        for a, b in zip(u.solution(), v.solution()):
            assert np.linalg.norm(a - b) <= 1e-10 * max(np.linalg.norm(b), 1.0)


def test_solves_to_the_known_optimum(zipf32):
    lp = zipf32
    for prec in (P.PDHG_FP64, P.PDHG_MIXED):
        with P.Solver.from_lp(lp, precision=prec, values32=1, primal_panels=1, long_row_min=64) as s:
            st, _ = s.iterate(200_000, 1e-8)
            assert st == P.PDHG_OK
            k = s.kkt()
            assert k["rel_kkt"] <= 1e-8
            assert k["primal_obj"] == pytest.approx(lp.f_star, rel=1e-7)
            assert k["dual_obj"] == pytest.approx(lp.f_star, rel=1e-7)


def test_automatic_choice_and_checks(zipf32):
    exact = zipf32
    inexact = lpgen.generate(300, 900, 6, nnz_per_col=4, val_range=(0.1, 10.0), support=0.3)
    assert np.any(inexact.val.astype(np.float32).astype(np.float64) != inexact.val)
    # default (-1): on for the FP64 phase of PDHG_MIXED when A is FP32-exact only
    for lp, prec, want in ((exact, P.PDHG_MIXED, 1), (inexact, P.PDHG_MIXED, 0), (exact, P.PDHG_FP64, 0),
                           (exact, P.PDHG_FP32, 0)):
        with P.Solver.from_lp(lp, precision=prec) as s:
            assert s.info()["values32"] == want, (prec, want)
    with P.Solver.from_lp(exact, values32=0, precision=P.PDHG_MIXED) as s:
        assert s.info()["values32"] == 0
    with pytest.raises(P.PDHGError) as e:
        P.Solver.from_lp(inexact, values32=1)
    assert e.value.status == P.PDHG_ERR_INVALID
    for bad in (dict(values32=2), dict(values32=-2), dict(values32=1, precision=P.PDHG_FP32),
                dict(values32=1, record_for_backward=1, restarts=0, primal_weight=0)):
        with pytest.raises(P.PDHGError):
            P.Solver.from_lp(exact, **bad)


def test_hot_columns_are_not_staged_on_unscaled_values(zipf32):
    """dual_hot_cols is ignored by the FP64 steps on the unscaled values: the
    iterates equal those without it, bit for bit."""
    lp = zipf32
    with P.Solver.from_lp(lp, values32=1, dual_hot_cols=4096) as h, P.Solver.from_lp(lp, values32=1) as d:
        h.iterate(256)
        d.iterate(256)
        for a, b in zip(h.solution(), d.solution()):
            np.testing.assert_array_equal(a, b)
