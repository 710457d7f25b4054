"""The generator's torch form (for LPs too large for host memory) against the
numpy form on the CPU: the same matrix, x* and z* bit for bit, y*, b and c to
rounding; and the literal capped Zipf counts of the large workload's stress
variant."""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2510_24429_b300 import lpgen

torch = pytest.importorskip("torch")


def _column_counts(lp):
    return np.diff(sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).tocsc().indptr)


@pytest.mark.parametrize("m,n,seed,kw", [
    (200, 500, 0, dict(nnz_per_col=5, val_range=(0.1, 1.0), support=150)),
    (3000, 9000, 2, dict(nnz_per_col=None, zipf=(1.5, 10000, 90000), val_range=(0.1, 10.0), support=0.3)),
    (50, 400, 7, dict(nnz_per_col=40, val_range=(0.1, 1.0), support=0.3)),  # many redraws of equal rows
])
def test_torch_form_matches_numpy_form(m, n, seed, kw):
    lp = lpgen.generate(m, n, seed, **kw)
    t = lpgen.generate_t(m, n, seed, _column_counts(lp), val_range=kw["val_range"], support=kw["support"],
                         device="cpu")
    assert t.nnz == lp.nnz
    for a, b in ((t.row_ptr, lp.row_ptr), (t.col_idx, lp.col_idx), (t.val, lp.val), (t.x_star, lp.x_star),
                 (t.z_star, lp.z_star)):
        assert np.array_equal(a.numpy(), b)
    np.testing.assert_allclose(t.y_star.numpy(), lp.y_star, rtol=0, atol=4 * np.finfo(float).eps * 8)
    for a, b in ((t.b, lp.b), (t.c, lp.c)):
        np.testing.assert_allclose(a.numpy(), b, rtol=0, atol=1e-13 * (1 + np.abs(b).max()))
    assert t.f_star == pytest.approx(lp.f_star, rel=1e-12)


def test_zipf_exact_counts():
    n, s, cap = 200_000, 1.5, 10_000
    z = lpgen.zipf_draws(0, n, s, cap)
    k = lpgen.zipf_exact_counts(0, n, s, cap, m=1_000_000)
    assert np.array_equal(k, np.minimum(z, cap).astype(np.int64))
    assert k.min() >= 1 and k.max() <= cap
    assert np.array_equal(lpgen.zipf_exact_counts(0, n, s, cap, m=50), np.minimum(k, 50))
    # the mean of min(Z, cap) is sum_{k <= cap} P(Z >= k) (153 here); heavy tail, so
    # a loose band: the sample standard deviation is ~500 per column
    mean = lpgen.zipf_tail(s, cap).sum()
    assert abs(k.mean() - mean) < 6 * k.std() / np.sqrt(n)
    # the rescaled counts of the large workload come from the same draws
    kr = lpgen.zipf_column_counts(0, n, s, cap, int(n * 10), 1_000_000)
    assert np.all(np.diff(kr[np.argsort(z, kind="stable")]) >= 0)
