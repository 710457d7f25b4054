"""The whole batch in one cooperative launch (persistent = 2): every
instance's iterations, evaluations, restart and primal-weight decisions and
termination test run inside a single kernel launch, the phases separated by
grid-wide barriers, replayed from a CUDA graph.

Each block of the cooperative grid runs, for the batch blocks it takes, the
same per-block code as the multi-launch batch engine (which is tested against
the single-LP engine and the oracle in test_gpu_batch.py), so the two forms
must agree bit for bit: solutions, iteration counts, restart counts and
rel. KKT. The barrier waits are bounded; a budget of one clock cycle makes the
first wait give up, which must end the launch with PDHG_ERR_TIMEOUT and leave
the context answering queries."""
import numpy as np
import pytest

from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P

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


def _run(lps, chunks, tol, **opts):
    with P.BatchSolver(lps, **opts) as bs:
        st = done = None
        total = 0
        for c in chunks:
            st, done = bs.iterate(c, tol)
            total += done
        info = bs.info()
        sols = [bs.solution(i) for i in range(len(lps))]
        eng = bs.engine_info()
    return st, total, info, sols, eng


def _assert_same(a, b):
    assert a[0] == b[0] and a[1] == b[1]
    for key in ("iterations", "converged", "rel_kkt", "restarts"):
        np.testing.assert_array_equal(a[2][key], b[2][key], err_msg=key)
    for sa, sb in zip(a[3], b[3]):
        for u, v in zip(sa, sb):
            np.testing.assert_array_equal(u, v)


@pytest.mark.parametrize("halpern", [0, 1])
@pytest.mark.parametrize("graphs", [1, 0])
def test_cooperative_launch_is_bit_identical_to_the_multi_launch_batch(halpern, graphs):
    lps = _batch_lps()
    ref = _run(lps, [100000], 1e-7, halpern=halpern)
    got = _run(lps, [100000], 1e-7, halpern=halpern, persistent=2, use_graphs=graphs)
    assert ref[0] == P.PDHG_OK and ref[2]["converged"].all()
    _assert_same(got, ref)
    assert got[4]["persistent_grid"] > 0
    # one launch per pdhg_iterate call (the multi-launch engine: thousands)
    assert got[4]["kernel_launches"] == 1 and ref[4]["kernel_launches"] > 100
    if graphs:
        assert got[4]["graph_launches"] == 1


def test_resumed_calls_and_iteration_limit():
    """Calls that stop inside an evaluation period and resume, and a limit
    reached before the tolerance (NOT_CONVERGED), give the same state as the
    multi-launch engine run in the same chunks."""
    lps = _batch_lps()
    chunks = [1, 63, 100, 37, 500]
    ref = _run(lps, chunks, 1e-9)
    got = _run(lps, chunks, 1e-9, persistent=2)
    assert ref[0] == P.PDHG_ERR_NOT_CONVERGED
    _assert_same(got, ref)
    ref = _run(lps, [700, 100000], 1e-7)
    got = _run(lps, [700, 100000], 1e-7, persistent=2)
    _assert_same(got, ref)


def test_large_instances_match_multi_launch_batch():
    """A few instances of the benchmark batch's size range (m up to 1e5), so
    that every instance spans many blocks of the cooperative grid."""
    sizes = [100_000, 3_000, 31_623, 1_000]
    lps = [lpgen.batch_lp(0, i, m) for i, m in enumerate(sizes)]
    ref = _run(lps, [200_000], 1e-6)
    got = _run(lps, [200_000], 1e-6, persistent=2)
    assert ref[0] == P.PDHG_OK
    _assert_same(got, ref)


def test_barrier_wait_that_gives_up_reports_timeout():
    """barrier_cycles = 1: a block that has to wait at the first grid barrier
    gives up at once; the launch ends (every other block leaves at its next
    barrier), pdhg_iterate returns PDHG_ERR_TIMEOUT naming the barrier, and
    the context still answers queries. A new batch on the same GPU then runs
    normally. No wait is unbounded, so nothing hangs."""
    lps = _batch_lps()
    with P.BatchSolver(lps, persistent=2, barrier_cycles=1) as bs:
        with pytest.raises(P.PDHGError) as ei:
            bs.iterate(640, 1e-7)
        assert ei.value.status == P.PDHG_ERR_TIMEOUT
        assert "barrier" in P.pdhg_last_error(bs.ctx)
        info = bs.info()
        assert len(info["iterations"]) == len(lps)
        assert np.isfinite(bs.kkt(0)["rel_kkt"])
    ref = _run(lps, [100000], 1e-7)
    got = _run(lps, [100000], 1e-7, persistent=2)
    _assert_same(got, ref)


def test_option_checks(tiny_lp):
    with pytest.raises(P.PDHGError):
        P.Solver.from_lp(tiny_lp, persistent=2)
    for bad in (dict(persistent=3), dict(persistent=2, kernel_timing=1), dict(persistent=2, barrier_cycles=-1)):
        with pytest.raises(P.PDHGError) as ei:
            P.BatchSolver([tiny_lp, tiny_lp], **bad)
        assert ei.value.status == P.PDHG_ERR_INVALID, bad
