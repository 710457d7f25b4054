"""Batched solves (pdhg_create_batch): many LPs of uneven sizes share every
launch, with per-instance scaling, step sizes, restarts and termination.
Each instance must behave like the single-LP engine on the same LP."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _batch_lps():
    sizes = [200, 17, 1000, 333, 2500, 50, 1]
    lps = [lpgen.generate(m, max(1, int(round(2.5 * m))), 100 + i, nnz_per_col=min(5, m), support=0.3)
           for i, m in enumerate(sizes)]
    lps.append(lpgen.tiny_lp(0))
    return lps


def test_batch_instances_match_single_lp_engine():
    lps = _batch_lps()
    tol = 1e-6
    with P.BatchSolver(lps) as bs:
        st, done = bs.iterate(100000, tol)
        info = bs.info()
        sols = [bs.solution(i) for i in range(len(lps))]
    assert st == P.PDHG_OK and info["converged"].all()
    assert (info["rel_kkt"] <= tol).all()
    assert done == info["iterations"].max()
    for i, lp in enumerate(lps):
        with P.Solver.from_lp(lp) as s:
            st1, k1 = s.iterate(100000, tol)
            x1, y1, z1 = s.solution()
        assert st1 == P.PDHG_OK
        # same method per instance; reductions group differently, so a
        # rounding-level near-tie may move a restart by an evaluation or two
        assert abs(int(info["iterations"][i]) - k1) <= 2 * 64, (i, info["iterations"][i], k1)
        x, y, z = sols[i]
        f = float(lp.c @ x)
        assert f == pytest.approx(lp.f_star, rel=10 * tol, abs=10 * tol), i
        if info["iterations"][i] == k1:
            assert rel_err(x, x1) <= 1e-8 and rel_err(y, y1) <= 1e-8, i


def test_batch_instance_against_oracle():
    lps = _batch_lps()
    with P.BatchSolver(lps) as bs:
        bs.iterate(200000, 1e-8)
        x, _, _ = bs.solution(len(lps) - 1)  # the tiny LP
    lp = lps[-1]
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options())
    assert orc.run(200000, 1e-8)
    assert float(lp.c @ x) == pytest.approx(float(lp.c @ orc.solution()[0]), rel=1e-7)
    assert float(lp.c @ x) == pytest.approx(lp.f_star, rel=1e-7)


def test_converged_instances_stop():
    lps = _batch_lps()
    with P.BatchSolver(lps) as bs:
        bs.iterate(100000, 1e-4)
        it1 = bs.info()["iterations"].copy()
        x1 = bs.solution(0)[0]
        bs.iterate(640, 1e-4)  # everything already converged: nothing moves
        it2 = bs.info()["iterations"]
        x2 = bs.solution(0)[0]
    np.testing.assert_array_equal(it1, it2)
    np.testing.assert_array_equal(x1, x2)


def test_batch_validation():
    lps = _batch_lps()[:3]
    bad = lpgen.generate(10, 20, 3, nnz_per_col=2)
    bad.col_idx = bad.col_idx.copy()
    bad.col_idx[0] = 99
    with pytest.raises(P.PDHGError) as ei:
        P.BatchSolver(lps + [bad])
    assert ei.value.status == P.PDHG_ERR_INVALID and "instance 3" in str(ei.value)
    with pytest.raises(P.PDHGError):
        P.BatchSolver(lps, precision=P.PDHG_MIXED)


def test_batch_kkt_per_instance():
    """pdhg_batch_kkt of every instance equals the KKT measures of its
    returned solution on its problem as given (oracle's definition)."""
    lps = _batch_lps()
    tol = 1e-6
    with P.BatchSolver(lps) as bs:
        bs.iterate(100000, tol)
        for i, lp in enumerate(lps):
            k = bs.kkt(i)
            x, y, _ = bs.solution(i)
            A = O.csr_matrix(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
            ko = O.kkt(A, lp.b, lp.c, x, y)
            assert k["rel_kkt"] <= tol, i
            # residual norms near convergence are differences of O(1) terms:
            # rounding enters at ~1e-16 of ||A|| ||x|| relative to a ~1e-6 residual
            for key, rel in (("rp_norm2", 1e-6), ("rd_norm2", 1e-6), ("rel_kkt", 1e-6), ("primal_obj", 1e-10),
                             ("dual_obj", 1e-10)):
                assert k[key] == pytest.approx(ko[key], rel=rel, abs=1e-12), (i, key)
        with pytest.raises(P.PDHGError):
            bs.kkt(len(lps))
