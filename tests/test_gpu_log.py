"""The per-evaluation JSONL log (environment variable PDHG_LOG, read when a
context is created): one line per evaluation of pdhg_iterate with the
candidate's relative residuals and gap (Section 2's termination test), the
decisions taken, the primal weight and the elapsed time. Checked against the
engine's own decision trace; off when the variable is unset or names a file
that cannot be opened."""
import json
import os

import pytest

from paper_2510_24429_b300 import pdhg as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _solve_logged(lp, path, iters, **opts):
    old = os.environ.get("PDHG_LOG")
    os.environ["PDHG_LOG"] = str(path)
    try:
        s = P.Solver.from_lp(lp, **opts)
    finally:
        if old is None:
            del os.environ["PDHG_LOG"]
        else:
            os.environ["PDHG_LOG"] = old
    with s:
        st, done = s.iterate(iters, 1e-12)
        trace = s.trace()
    return trace


@pytest.mark.parametrize("opts", [dict(), dict(precision=P.PDHG_MIXED, halpern=1, restart_scheme=1)])
def test_one_line_per_evaluation(tiny_lp, tmp_path, opts):
    path = tmp_path / "pdhg.jsonl"
    trace = _solve_logged(tiny_lp, path, 640, **opts)
    recs = [json.loads(line) for line in path.read_text().splitlines()]
    assert [r["iteration"] for r in recs] == [64 * (i + 1) for i in range(10)]
    assert len(trace) == len(recs)
    for r, t in zip(recs, trace):
        assert r["iteration"] == t["iteration"]
        assert r["omega"] == t["omega"]
        assert r["rel_kkt"] == pytest.approx(max(r["rel_p"], r["rel_d"], r["rel_gap"]), rel=1e-12)
        assert r["rel_kkt"] == pytest.approx(t["rel_kkt"], rel=1e-12)
        assert r["candidate"] in ("current", "average")
        assert r["restart"] in ("none", "restart_current", "restart_average", "take_average", "restart_step")
        assert r["precision"] == ("fp32" if opts.get("precision") == P.PDHG_MIXED else "fp64")
        assert r["elapsed_s"] >= 0.0
    assert recs[-1]["restarts"] >= 1
    assert all(a["elapsed_s"] <= b["elapsed_s"] for a, b in zip(recs, recs[1:]))


def test_appends_and_off_by_default(tiny_lp, tmp_path):
    path = tmp_path / "log.jsonl"
    _solve_logged(tiny_lp, path, 128)
    _solve_logged(tiny_lp, path, 128)
    assert len(path.read_text().splitlines()) == 4  # two contexts, two evaluations each
    assert "PDHG_LOG" not in os.environ or os.environ["PDHG_LOG"] != str(path)
    with P.Solver.from_lp(tiny_lp) as s:  # unset: nothing written anywhere
        s.iterate(128, 1e-12)
    assert len(path.read_text().splitlines()) == 4
    # a path that cannot be opened (a directory) leaves the log off; the solve runs
    _solve_logged(tiny_lp, tmp_path, 128)
