"""FP32 iteration with FP64 evaluation (PDHG_FP32) and FP32 followed by an
FP64 polishing phase (PDHG_MIXED), against the FP64 oracle and the generator's
known optimum. FP32 results differ from FP64 by rounding of the FP32 matrix,
vectors and accumulation; the errors are printed and held to loose bounds,
while the mixed form must reach the requested relative KKT (evaluated in FP64).
"""
import numpy as np
import pytest

from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import TINY_PLAIN, pair, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def test_fp32_100_iterations_close_to_fp64_oracle(tiny_lp):
    orc, _ = pair(tiny_lp, **TINY_PLAIN)
    orc.run(100)
    with P.Solver.from_lp(tiny_lp, precision=P.PDHG_FP32, pock_chambolle=0, restarts=0, primal_weight=0) as sol:
        assert sol.info()["precision_now"] == P.PDHG_FP32
        sol.iterate(100)
        x, y, z = sol.solution()
    xo, yo, _ = orc.solution()
    ex, ey = rel_err(x, xo), rel_err(y, yo)
    print(f"FP32 vs FP64 oracle after 100 iterations: x {ex:.2e}, y {ey:.2e}")
    assert ex < 1e-4 and ey < 1e-4
    assert ex > 0 or ey > 0  # really computed in FP32


@pytest.mark.parametrize("tol", [1e-6, 1e-8])
def test_mixed_reaches_tolerance_and_optimum(tiny_lp, tol):
    lp = tiny_lp
    orc, _ = pair(lp)
    assert orc.run(200000, tol)
    fo = float(lp.c @ orc.solution()[0])
    with P.Solver.from_lp(lp, precision=P.PDHG_MIXED, polish_switch=1e-5) as sol:
        st, done = sol.iterate(200000, tol)
        info = sol.info()
        k = sol.kkt()
        x, _, _ = sol.solution()
    assert st == P.PDHG_OK and k["rel_kkt"] <= tol
    assert info["precision_now"] == P.PDHG_FP64 and 0 < info["polish_started_at"] <= done
    err_f = abs(k["primal_obj"] - lp.f_star) / (1 + abs(lp.f_star))
    err_o = abs(k["primal_obj"] - fo) / (1 + abs(fo))
    print(f"mixed to {tol:g}: {done} iterations (FP64 from {info['polish_started_at']}), "
          f"objective error vs f* {err_f:.2e}, vs FP64 oracle {err_o:.2e}, oracle iterations {orc.k}")
    assert err_f <= 10 * tol and err_o <= 10 * tol
    assert rel_err(x, lp.x_star) <= 1e3 * tol


def test_fp32_only_reaches_1e_4(tiny_lp):
    lp = tiny_lp
    with P.Solver.from_lp(lp, precision=P.PDHG_FP32) as sol:
        st, done = sol.iterate(200000, 1e-4)
        k = sol.kkt()
        assert sol.info()["precision_now"] == P.PDHG_FP32
    assert st == P.PDHG_OK and k["rel_kkt"] <= 1e-4
    print(f"FP32 to 1e-4: {done} iterations, objective error vs f* "
          f"{abs(k['primal_obj'] - lp.f_star) / (1 + abs(lp.f_star)):.2e}")


def test_mixed_on_ragged_multi_tile_lp():
    lp = lpgen.generate(3001, 7919, 5, nnz_per_col=5, support=0.3)
    with P.Solver.from_lp(lp, precision=P.PDHG_MIXED, polish_switch=1e-5) as sol:
        st, done = sol.iterate(300000, 1e-7)
        k = sol.kkt()
        snap_count, _ = sol.snapshot_poll()
    assert st == P.PDHG_OK and k["rel_kkt"] <= 1e-7
    assert abs(k["primal_obj"] - lp.f_star) <= 1e-6 * (1 + abs(lp.f_star))


def test_mixed_snapshots_follow_algorithm1(tiny_lp):
    with P.Solver.from_lp(tiny_lp, precision=P.PDHG_MIXED, eps_cross=1e-2, eps_factor=0.1) as sol:
        sol.iterate(200000, 1e-7)
        cnt, _ = sol.snapshot_poll()
        snap = sol.snapshot()
    assert cnt >= 4
    assert snap["rel_kkt"] <= 1e-2 * 0.1 ** (cnt - 1)
    assert np.all(snap["z"] >= 0) and np.all(snap["x"] >= 0)
