"""Layout autotuner (pdhg_autotune, pdhg_profile_key).

The profile key and the cache file are host logic and are tested here without
a GPU: a stored choice for the same profile is returned before any device
work. Timing runs (and the use of the tuned options) are GPU tests."""
import numpy as np
import pytest

from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def test_profile_key_is_deterministic_and_shape_sensitive():
    tiny = lpgen.tiny_lp(0)
    k1 = P.pdhg_profile_key([tiny])
    assert k1 == P.pdhg_profile_key([lpgen.tiny_lp(0)])
    assert P.pdhg_profile_key([tiny], P.PDHG_MIXED) != k1
    other = lpgen.generate(200, 500, 0, nnz_per_col=2)
    assert P.pdhg_profile_key([other]) != k1
    assert P.pdhg_profile_key([tiny, tiny]) != k1
    # every column of the tiny LP has 5 entries: one length class [4, 8) for A^T
    assert k1.endswith("/T3:100")


def test_cache_hit_needs_no_device(tmp_path):
    tiny = lpgen.tiny_lp(0)
    key = P.pdhg_profile_key([tiny])
    path = tmp_path / "tune.txt"
    path.write_text(
        "some/other/key 512 1 32 0.1\n"
        f"{key} 999 4 64 0.2\n"      # invalid block size: ignored
        f"{key} 128 2 64 0.3\n"
        "garbage line\n"
        f"{key} 512 1 256 0.25\n"    # the last valid line wins
    )
    base = P.pdhg_default_options(eps_cross=1e-3)
    tuned, hit = P.pdhg_autotune([tiny], base, str(path))
    assert hit
    assert (tuned.step_block, tuned.rows_per_thread, tuned.long_row_min) == (512, 1, 256)
    assert tuned.eps_cross == 1e-3  # the rest of the options are the caller's


def test_invalid_inputs_rejected():
    tiny = lpgen.tiny_lp(0)
    bad = lpgen.generate(10, 20, 3, nnz_per_col=2)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[0] = 99
    with pytest.raises(P.PDHGError) as ei:
        P.pdhg_profile_key([tiny, bad])
    assert ei.value.status == P.PDHG_ERR_INVALID and "instance 1" in str(ei.value)
    with pytest.raises(P.PDHGError):
        P.pdhg_autotune([tiny], P.pdhg_default_options(inputs_on_device=1))


@pytest.mark.gpu
def test_autotune_times_stores_and_reuses(tmp_path):
    tiny = lpgen.tiny_lp(0)
    path = tmp_path / "tune.txt"
    tuned, hit = P.pdhg_autotune([tiny], None, str(path))
    assert not hit
    assert tuned.step_block in (128, 256, 512) and tuned.rows_per_thread in (1, 2, 4)
    assert tuned.long_row_min in (32, 64, 128, 256, 512)
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith(P.pdhg_profile_key([tiny]) + " ")
    again, hit2 = P.pdhg_autotune([tiny], None, str(path))
    assert hit2
    assert (again.step_block, again.rows_per_thread, again.long_row_min) == (
        tuned.step_block, tuned.rows_per_thread, tuned.long_row_min)
    # the tuned layout solves the LP like any other
    with P.Solver.from_lp(tiny, **{k: getattr(tuned, k) for k in ("step_block", "rows_per_thread",
                                                                   "long_row_min")}) as s:
        st, _ = s.iterate(200000, 1e-8)
        assert st == P.PDHG_OK
        assert s.kkt()["primal_obj"] == pytest.approx(tiny.f_star, rel=1e-7)


@pytest.mark.gpu
@pytest.mark.parametrize("step_block", [128, 512])
def test_block_sizes_solve_batches(step_block):
    lps = [lpgen.generate(m, int(2.5 * m), 40 + i, nnz_per_col=5, support=0.3) for i, m in enumerate((300, 50, 900))]
    lps.append(lpgen.tiny_lp(0))
    tol = 1e-7
    with P.BatchSolver(lps, step_block=step_block) as bs:
        st, _ = bs.iterate(100000, tol)
        assert st == P.PDHG_OK
        for i, lp in enumerate(lps):
            x, _, _ = bs.solution(i)
            assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=10 * tol, abs=10 * tol), i


@pytest.mark.gpu
def test_autotune_batch():
    lps = [lpgen.generate(m, int(2.5 * m), 60 + i, nnz_per_col=5, support=0.3) for i, m in enumerate((400, 80, 1500))]
    tuned, hit = P.pdhg_autotune(lps)
    assert not hit and tuned.step_block in (128, 256, 512)
    with P.BatchSolver(lps, step_block=tuned.step_block, rows_per_thread=tuned.rows_per_thread,
                       long_row_min=tuned.long_row_min) as bs:
        st, _ = bs.iterate(100000, 1e-6)
        assert st == P.PDHG_OK
        assert np.all(bs.info()["converged"])
