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


# ---------------------------------------------------------------------------
# per-instance snapshots (pdhg_snapshot_i): Algorithm 1's hand-off for every LP
# of a batch
# ---------------------------------------------------------------------------

def test_batch_periodic_snapshots_match_oracle():
    """snapshot_every = 128: after 256 iterations every instance that is still
    iterating holds the candidate of its evaluation at 256 (its second
    snapshot); the tiny LP's equals the oracle's snapshot at 1e-8."""
    lps = _batch_lps()
    lp = lps[-1]
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(snapshot_every=128))
    orc.run(256)
    with P.BatchSolver(lps, snapshot_every=128) as bs:
        bs.iterate(256)
        info = bs.info()
        snap = bs.snapshot(len(lps) - 1)
        for i in range(len(lps)):
            si = bs.snapshot(i)
            assert si["count"] == 2 and si["iteration"] == 256, (i, si["count"], si["iteration"])
            assert info["iterations"][i] == 256
    ref = orc.snapshots[-1]
    assert len(orc.snapshots) == 2 and ref["iteration"] == 256
    assert snap["rel_kkt"] == pytest.approx(ref["rel_kkt"], rel=1e-6)
    for key in ("x", "y", "z"):
        scale = max(float(np.max(np.abs(ref[key]))), float(np.linalg.norm(lp.c)) / np.sqrt(lp.n) if key == "z" else 0)
        assert float(np.max(np.abs(snap[key] - ref[key]))) <= 1e-8 * scale, key


def test_batch_algorithm1_thresholds_match_oracle():
    """eps_cross = 1e-2, eps_factor = 0.1: the tiny LP's instance takes a
    snapshot at the first evaluation at or below each threshold, as the oracle
    does; its latest one equals the oracle's."""
    lps = _batch_lps()
    lp = lps[-1]
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, O.Options(eps_cross=1e-2))
    assert orc.run(200000, 1e-7)
    with P.BatchSolver(lps, eps_cross=1e-2, eps_factor=0.1) as bs:
        st, _ = bs.iterate(200000, 1e-7)
        assert st == P.PDHG_OK
        snap = bs.snapshot(len(lps) - 1)
        counts = [bs.snapshot(i)["count"] for i in range(len(lps))]
    ref = orc.snapshots[-1]
    assert snap["count"] == len(orc.snapshots) >= 4
    assert snap["iteration"] == ref["iteration"]
    assert snap["rel_kkt"] == pytest.approx(ref["rel_kkt"], rel=1e-6)
    for key in ("x", "y"):
        assert float(np.max(np.abs(snap[key] - ref[key]))) <= 1e-8 * float(np.max(np.abs(ref[key]))), key
    # every instance went from rel. KKT > 1e-2 to 1e-7 and took at least one
    # snapshot (one per evaluation: an instance that falls past several
    # thresholds between two evaluations, like the 1 x 2 LP, takes fewer)
    assert min(counts) >= 1 and sorted(counts)[len(counts) // 2] >= 4


@pytest.mark.parametrize("halpern", [0, 1])
def test_cooperative_batch_snapshots_bit_identical(halpern):
    """The cooperative launch (persistent = 2) packs the same snapshots as the
    multi-launch batch engine."""
    lps = _batch_lps()
    out = []
    for persistent in (0, 2):
        with P.BatchSolver(lps, eps_cross=1e-2, snapshot_every=200, halpern=halpern, persistent=persistent) as bs:
            bs.iterate(100000, 1e-7)
            out.append([bs.snapshot(i) for i in range(len(lps))])
    for a, b in zip(*out):
        assert (a["count"], a["iteration"], a["rel_kkt"]) == (b["count"], b["iteration"], b["rel_kkt"])
        for key in ("x", "y", "z"):
            np.testing.assert_array_equal(a[key], b[key])


def test_batch_snapshot_errors():
    lps = _batch_lps()
    with P.BatchSolver(lps) as bs:
        bs.iterate(64)
        with pytest.raises(P.PDHGError) as ei:
            bs.snapshot(0)
        assert ei.value.status == P.PDHG_ERR_STATE
        with pytest.raises(P.PDHGError) as ei:
            bs.snapshot(len(lps))
        assert ei.value.status == P.PDHG_ERR_INVALID
    with P.BatchSolver(lps, snapshot_every=1000) as bs:
        bs.iterate(64)
        with pytest.raises(P.PDHGError) as ei:
            bs.snapshot(0)
        assert ei.value.status == P.PDHG_ERR_STATE
    with pytest.raises(P.PDHGError):
        P.BatchSolver(lps[:2], snapshot_every=100, persistent=1)
