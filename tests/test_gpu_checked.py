"""The range-checked build (libpdhg_checked.so, compiled with PDHG_CHECKED):
every matrix unit's entry range and rows and every gathered column index are
checked before use; an index out of range sets a device error word, the access
is skipped (nothing traps), and the call returns PDHG_ERR_INVALID.

It stands in for a memory checker on this GPU pool. The checked library is
loaded in a child process (the binding keeps one library per process) that
runs small cases of every engine form and expects no check to fire and the
same parity with the oracle as the normal build; then it passes the
allocation-free KKT entry point a CSR with one column index out of range and
expects PDHG_ERR_INVALID from the check, and a correct call after it."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import sys
import numpy as np
import scipy.sparse as sp
import torch
sys.path.insert(0, ROOT)
from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import build, lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import TINY_PLAIN, assert_iterates_close, pair

P.load(build.build(checked=True))
torch.cuda.set_device(0)
tiny = lpgen.tiny_lp(0)
zipf = lpgen.generate(3000, 9000, 2, nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0),
                      support=0.3, fp32_values=True)
# every engine form on small cases: no check may fire, parity as usual
orc, sol = pair(tiny, **TINY_PLAIN)
orc.run(100); sol.iterate(100)
assert_iterates_close(sol, orc, 1e-10)
orc, sol = pair(tiny)
orc.run(640, 1e-9); st, _ = sol.iterate(640, 1e-9)
for eng in (dict(primal_panels=1, panel_rows=256, long_row_min=32), dict(primal_panels=0)):
    o = O.Oracle(zipf.m, zipf.n, zipf.row_ptr, zipf.col_idx, zipf.val, zipf.b, zipf.c,
                 O.Options(pock_chambolle=False, restarts=False, primal_weight=False))
    o.run(100)
    with P.Solver.from_lp(zipf, pock_chambolle=0, restarts=0, primal_weight=0, **eng) as s:
        s.iterate(100)
        assert_iterates_close(s, o, 1e-10)
for extra in (dict(precision=P.PDHG_FP32), dict(precision=P.PDHG_MIXED), dict(halpern=1), dict(dual_hot_cols=5000),
              dict(feas_polish=1, gap_tol=1e-4)):
    with P.Solver.from_lp(zipf, primal_panels=1, panel_rows=256, long_row_min=32, **extra) as s:
        st, _ = s.iterate(3000, 1e-6)
        assert st in (P.PDHG_OK, P.PDHG_ERR_NOT_CONVERGED), extra
with P.Solver.from_lp(tiny, restarts=0, primal_weight=0, record_for_backward=1) as s:
    s.iterate(60)
    s.backward(np.ones(tiny.n))
lps = [lpgen.generate(m, int(2.5 * m), 7 + m, nnz_per_col=5, support=0.3) for m in (40, 300, 90)]
for persistent in (0, 1, 2):
    with P.BatchSolver(lps, persistent=persistent) as bs:
        st, _ = bs.iterate(20000, 1e-6)
        assert st == P.PDHG_OK, persistent
# the allocation-free entry point: a column index out of range is caught
A = sp.csr_matrix((zipf.val, zipf.col_idx, zipf.row_ptr), shape=(zipf.m, zipf.n))
At = sp.csr_matrix(A.T)
dev = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a)).to(dtype=dt, device="cuda")
mats = [dev(A.indptr, torch.int64), dev(A.indices, torch.int32), dev(A.data, torch.float64),
        dev(At.indptr, torch.int64), dev(At.indices, torch.int32), dev(At.data, torch.float64),
        dev(zipf.b, torch.float64), dev(zipf.c, torch.float64)]
x, y = dev(np.full(zipf.n, 0.5), torch.float64), dev(np.full(zipf.m, 0.25), torch.float64)
good = P.pdhg_kkt_noalloc(zipf.m, zipf.n, *mats, x, y)
bad = mats[1].clone()
bad[5] = zipf.n + 7
try:
    P.pdhg_kkt_noalloc(zipf.m, zipf.n, mats[0], bad, *mats[2:], x, y)
    raise SystemExit("no error for an out-of-range column index")
except P.PDHGError as e:
    assert e.status == P.PDHG_ERR_INVALID and "checked build" in str(e), e
again = P.pdhg_kkt_noalloc(zipf.m, zipf.n, *mats, x, y)
assert again == good
print("checked build ok")
'''


def test_checked_build_runs_clean_and_catches_a_bad_index():
    from paper_2510_24429_b300 import build

    build.build(checked=True)
    res = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], cwd=ROOT, capture_output=True,
                         text=True, timeout=900)
    assert res.returncode == 0, res.stdout[-3000:] + res.stderr[-3000:]
    assert "checked build ok" in res.stdout
