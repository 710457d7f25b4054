"""Inputs through the device-side setup: CSRs handed over in device memory
(validated on the device, then built in place) give the same engine as host
inputs; malformed device CSRs are rejected with the same statuses as host
ones; an LP without stored entries goes through every zero-size path of the
layout build."""
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


def _dev(lp, **over):
    import torch

    arrs = dict(row_ptr=lp.row_ptr, col_idx=lp.col_idx, val=lp.val, b=lp.b, c=lp.c)
    arrs.update(over)
    return {k: torch.as_tensor(np.asarray(v)).cuda() for k, v in arrs.items()}


def test_device_inputs_match_host_inputs(tiny_lp):
    d = _dev(tiny_lp)
    with P.Solver(tiny_lp.m, tiny_lp.n, d["row_ptr"], d["col_idx"], d["val"], d["b"], d["c"]) as sd, \
            P.Solver.from_lp(tiny_lp) as sh:
        assert sd.iterate(200) == sh.iterate(200)
        for a, b in zip(sd.solution(), sh.solution()):
            np.testing.assert_array_equal(a, b)


def _malformed(tiny_lp):
    lp = tiny_lp
    ci = np.asarray(lp.col_idx).copy()
    ci_oob = ci.copy()
    ci_oob[7] = lp.n + 3
    r = int(np.argmax(np.diff(lp.row_ptr) >= 2))  # a row with two entries
    ci_uns = ci.copy()
    a = int(lp.row_ptr[r])
    ci_uns[a], ci_uns[a + 1] = ci_uns[a + 1], ci_uns[a]
    rp_dec = np.asarray(lp.row_ptr).copy()
    rp_dec[5] = rp_dec[7]  # row 5 ends before it starts... row 4 grows, row 5 shrinks
    rp_end = np.asarray(lp.row_ptr).copy()
    rp_end[-1] -= 1
    v_nan = np.asarray(lp.val).copy()
    v_nan[3] = np.nan
    b_inf = np.asarray(lp.b).copy()
    b_inf[0] = np.inf
    return [("col out of range", dict(col_idx=ci_oob), P.PDHG_ERR_INVALID),
            ("unsorted columns", dict(col_idx=ci_uns), P.PDHG_ERR_INVALID),
            ("row_ptr not monotone", dict(row_ptr=rp_dec), P.PDHG_ERR_INVALID),
            ("row_ptr[m] != nnz", dict(row_ptr=rp_end), P.PDHG_ERR_INVALID),
            ("NaN value", dict(val=v_nan), P.PDHG_ERR_NUMERIC),
            ("Inf in b", dict(b=b_inf), P.PDHG_ERR_NUMERIC)]


def test_malformed_device_inputs_rejected(tiny_lp):
    for name, over, status in _malformed(tiny_lp):
        d = _dev(tiny_lp, **over)
        with pytest.raises(P.PDHGError) as ei:
            P.Solver(tiny_lp.m, tiny_lp.n, d["row_ptr"], d["col_idx"], d["val"], d["b"], d["c"])
        assert ei.value.status == status, name
        # the same input from the host gets the same status
        h = dict(row_ptr=tiny_lp.row_ptr, col_idx=tiny_lp.col_idx, val=tiny_lp.val, b=tiny_lp.b, c=tiny_lp.c)
        h.update(over)
        with pytest.raises(P.PDHGError) as eh:
            P.Solver(tiny_lp.m, tiny_lp.n, h["row_ptr"], h["col_idx"], h["val"], h["b"], h["c"])
        assert eh.value.status == status, name


@pytest.mark.parametrize("panels", [0, 1])
def test_lp_without_entries(panels):
    """A = 0, b = 0, c > 0: the optimum is x = 0 with objective 0."""
    m, n = 3, 5
    rp = np.zeros(m + 1, np.int64)
    ci = np.zeros(0, np.int32)
    v = np.zeros(0)
    c = np.linspace(0.5, 2.0, n)
    with P.Solver(m, n, rp, ci, v, np.zeros(m), c, primal_panels=panels, panel_rows=2) as s:
        st, _ = s.iterate(6400, 1e-9)
        x, y, z = s.solution()
        k = s.kkt()
    assert st == P.PDHG_OK and k["rel_kkt"] <= 1e-9
    assert np.all(x == 0.0) and np.allclose(z, c)
