"""The seeded input generator against the recipe it states.

* Its random numbers are SplitMix64 draws (the published finaliser, checked on
  the sequential generator's first outputs), uniform in [0, 1) and standard
  normal in distribution.
* The large workload's recipe, here at a tenth of its size (m = 1e5,
  n = 3e5, nnz = 3e6): column counts k_j = rint(alpha min(Z_j, cap)) with
  Z_j ~ Zipf(1.5), cap 1e4, checked against the Zipf tail
  P(Z >= k) = zeta(1.5, k) / zeta(1.5) computed here from its definition;
  rows drawn uniformly (row counts with mean and variance nnz / m); values
  +-U[0.1, 10] with a fair sign; well-formed CSR.
* The seeded optimum: b = A x*, c = A^T y* + z*, x*, z* >= 0 and x*_j z*_j = 0
  on every column, with x* positive on 30% of the columns, so that
  f* = c^T x* = b^T y* is the LP's optimal value (Section 2's optimality
  conditions).
* Batch sizes log-uniform in [1e3, 1e5]; generation is a pure function of the
  seed."""
import json
import math
import pathlib

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.special import zeta

from paper_2510_24429_b300 import lpgen

GOLDEN = pathlib.Path(__file__).parent / "golden"


def test_mix64_is_splitmix64():
    g = json.loads((GOLDEN / "splitmix64_seed0.json").read_text())
    # the sequential generator seeded with 0 outputs mix64(i * GAMMA), i = 1, 2, ...
    with np.errstate(over="ignore"):
        out = lpgen._mix64(np.arange(1, 5, dtype=np.uint64) * lpgen.GAMMA)
    assert [f"{int(v):016x}" for v in out] == g["outputs_hex"]


def test_uniform_and_normal_draws():
    N = 1 << 20
    idx = np.arange(N, dtype=np.uint64)
    u = lpgen.rand_uniform(0, lpgen.S_MAG, idx)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / N)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt((1 / 80 - 1 / 144) / N)
    z = lpgen.rand_normal(0, lpgen.S_YS, idx)
    assert abs(z.mean()) < 5 / math.sqrt(N) and abs(z.var() - 1.0) < 5 * math.sqrt(2 / N)
    assert abs(float(np.mean(z ** 3))) < 5 * math.sqrt(15 / N)  # symmetric
    assert abs(float(np.mean(z ** 4)) - 3.0) < 5 * math.sqrt(96 / N)  # normal kurtosis
    # streams and seeds are uncorrelated
    v = lpgen.rand_uniform(0, lpgen.S_XS, idx)
    w = lpgen.rand_uniform(1, lpgen.S_MAG, idx)
    assert abs(np.corrcoef(u, v)[0, 1]) < 5 / math.sqrt(N)
    assert abs(np.corrcoef(u, w)[0, 1]) < 5 / math.sqrt(N)


M, N, NNZ, CAP = 100_000, 300_000, 3_000_000, 10_000


@pytest.fixture(scope="module")
def zipf_lp():
    return lpgen.large_lp(0, m=M, n=N, nnz=NNZ)


def test_zipf_workload_is_well_formed_csr(zipf_lp):
    lp = zipf_lp
    rp, ci = lp.row_ptr, lp.col_idx
    assert lp.m == M and lp.n == N and rp[0] == 0 and rp[-1] == ci.size == lp.val.size
    assert np.all(np.diff(rp) >= 0)
    assert ci.min() >= 0 and ci.max() < N
    row_of = np.repeat(np.arange(M), np.diff(rp))
    same_row = row_of[1:] == row_of[:-1]
    assert np.all(np.diff(ci.astype(np.int64))[same_row] > 0)  # strictly increasing: no duplicates


def test_zipf_column_counts_follow_the_zipf_tail(zipf_lp):
    counts = np.bincount(zipf_lp.col_idx, minlength=N)
    assert abs(int(counts.sum()) - NNZ) <= NNZ // 1000
    assert counts.min() == 1
    # counts = rint(alpha min(Z, cap)): the largest count fixes alpha to 1e-4 relative
    alpha = counts.max() / CAP
    tail = lambda k: zeta(1.5, k) / zeta(1.5, 1)  # noqa: E731  P(Z >= k), Z ~ Zipf(1.5)
    for K in (20, 100, 400, int(counts.max())):
        expected = tail(math.ceil((K - 0.5) / alpha))  # rint(alpha Z) >= K  <=>  Z >= (K - 1/2) / alpha
        observed = float(np.mean(counts >= K))
        sd = math.sqrt(expected * (1 - expected) / N)
        assert abs(observed - expected) < 5 * sd, (K, observed, expected)
    # the heavy tail: the CCDF falls as k^(-1/2) between the body and the cap
    r = np.mean(counts >= 200) / np.mean(counts >= 100)
    assert abs(r - 2 ** -0.5) < 0.03, r


def test_zipf_rows_values_and_signs(zipf_lp):
    lp = zipf_lp
    per_row = np.diff(lp.row_ptr)
    mean = NNZ / M
    assert per_row.mean() == pytest.approx(mean, rel=1e-3)
    assert per_row.var() == pytest.approx(mean, rel=0.05)  # uniform rows: multinomial, var ~ mean
    a = np.abs(lp.val)
    assert a.min() >= 0.1 and a.max() <= 10.0
    assert abs(a.mean() - 5.05) < 5 * (9.9 / math.sqrt(12)) / math.sqrt(a.size)
    neg = float(np.mean(lp.val < 0))
    assert abs(neg - 0.5) < 5 * 0.5 / math.sqrt(a.size)


@pytest.mark.parametrize("which", ["zipf", "tiny", "batch", "adjoint"])
def test_seeded_optimum_is_complementary(which, zipf_lp):
    lp = {"zipf": lambda: zipf_lp, "tiny": lambda: lpgen.tiny_lp(0),
          "batch": lambda: lpgen.batch_lp(0, 3, 2000),
          "adjoint": lambda: lpgen.adjoint_lp(0, m=20_000, n=60_000)}[which]()
    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n))
    xs, ys, zs = lp.x_star, lp.y_star, lp.z_star
    assert np.all(xs >= 0) and np.all(zs >= 0) and np.all(xs * zs == 0)
    on = xs > 0
    assert np.all((xs[on] >= 0.5) & (xs[on] <= 2.0)) and np.all((zs[~on] >= 0.5) & (zs[~on] <= 2.0))
    n_sup = 150 if which == "tiny" else int(round(0.3 * lp.n))
    assert int(on.sum()) == n_sup
    scale_b = 1 + np.abs(A) @ xs
    scale_c = 1 + np.abs(A.T) @ np.abs(ys) + zs
    assert np.max(np.abs(A @ xs - lp.b) / scale_b) < 1e-14
    assert np.max(np.abs(A.T @ ys + zs - lp.c) / scale_c) < 1e-14
    f1, f2 = float(lp.c @ xs), float(lp.b @ ys)
    assert abs(f1 - f2) <= 1e-12 * (1 + np.abs(lp.c) @ xs + np.abs(lp.b) @ np.abs(ys))


def test_adjoint_lp_values_are_fp32_exact():
    lp = lpgen.adjoint_lp(0, m=20_000, n=60_000)
    assert np.array_equal(lp.val.astype(np.float32).astype(np.float64), lp.val)
    assert np.all(np.bincount(lp.col_idx, minlength=lp.n) == 6)


def test_batch_sizes_are_log_uniform():
    sizes = np.array(lpgen.batch_sizes(0, 256))
    assert sizes.min() >= 1000 and sizes.max() <= 100_000
    logs = np.log(sizes)
    lo, hi = math.log(1e3), math.log(1e5)
    assert abs(logs.mean() - (lo + hi) / 2) < 5 * (hi - lo) / math.sqrt(12 * 256)
    lp = lpgen.batch_lp(0, 7, int(sizes[7]))
    assert lp.n == round(2.5 * lp.m) and np.all(np.bincount(lp.col_idx, minlength=lp.n) == 5)


def test_generation_is_a_function_of_the_seed():
    a, b, c = lpgen.tiny_lp(0), lpgen.tiny_lp(0), lpgen.tiny_lp(1)
    for f in ("row_ptr", "col_idx", "val", "b", "c", "x_star", "y_star", "z_star"):
        assert np.array_equal(getattr(a, f), getattr(b, f)), f
    assert not np.array_equal(a.val, c.val) and not np.array_equal(a.b, c.b)
