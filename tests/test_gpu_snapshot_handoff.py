"""Algorithm 1's hand-off of snapshots to a concurrent consumer thread
(pdhg_snapshot_wait): while one thread runs pdhg_iterate, another receives the
snapshots as they reach pinned host memory. Received snapshots come in order,
each equal to the oracle's snapshot at the same iteration; the last one is
always received; a wait with nothing new times out on the host."""
import threading
import time

import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import SHARED, max_rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


@pytest.mark.parametrize("persistent", [0, 1])
def test_consumer_thread_receives_algorithm1_snapshots(tiny_lp, persistent):
    lp = tiny_lp
    oopt = O.Options(eps_cross=1e-2, eps_factor=0.1)
    orc = O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, oopt)
    assert orc.run(200000, 1e-8)
    ref = {s["iteration"]: s for s in orc.snapshots}
    copts = {k: (int(v) if isinstance(v, bool) else v) for k, v in ((k, getattr(oopt, k)) for k in SHARED)}
    sol = P.Solver(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c, persistent=persistent, **copts)
    got, done, errors = [], threading.Event(), []

    def consumer():
        last = 0
        try:
            while True:
                try:
                    snap = sol.snapshot_wait(last, timeout_ms=200)
                except P.PDHGError as e:
                    if e.status == P.PDHG_ERR_TIMEOUT and done.is_set():
                        return
                    if e.status != P.PDHG_ERR_TIMEOUT:
                        raise
                    continue
                last = snap["index"]
                got.append(snap)
                time.sleep(0.002)  # a slow consumer: snapshots may be skipped, never torn
        except Exception as e:  # surfaced in the main thread
            errors.append(e)

    t = threading.Thread(target=consumer)
    t.start()
    st, _ = sol.iterate(200000, 1e-8)
    count, _ = sol.snapshot_poll()
    done.set()
    t.join(timeout=30)
    assert not t.is_alive() and not errors, errors
    assert st == P.PDHG_OK and count == len(orc.snapshots) >= 5
    idx = [g["index"] for g in got]
    assert idx == sorted(set(idx)) and idx[-1] == count
    for g in got:
        r = ref[g["iteration"]]
        assert g["rel_kkt"] == pytest.approx(r["rel_kkt"], rel=1e-6)
        for key in ("x", "y", "z"):
            assert max_rel_err(g[key], r[key]) <= 1e-8, (g["iteration"], key)
    sol.close()


def test_wait_times_out_on_the_host(tiny_lp):
    with P.Solver.from_lp(tiny_lp) as sol:
        t0 = time.perf_counter()
        with pytest.raises(P.PDHGError) as ei:
            sol.snapshot_wait(0, timeout_ms=50)
        assert ei.value.status == P.PDHG_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 5.0
        # the context stays usable
        assert sol.iterate(64) == (P.PDHG_OK, 64)
