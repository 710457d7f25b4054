"""Seeded synthetic standard-form LP generator (input data only).

Builds ``min c^T x  s.t.  A x = b, x >= 0`` together with a known complementary
primal-dual optimum ``(x*, y*, z*)``: ``b = A x*`` and ``c = A^T y* + z*`` with
``x*_j z*_j = 0`` for every column, so ``x*`` and ``(y*, z*)`` satisfy the
optimality conditions of the LP pair in Section 2 of the paper (zero residuals,
``x, z >= 0`` and ``x^T z = 0``), and ``f* = c^T x* = b^T y*``.

The paper measures on the Mittelmann LP set and on a proprietary set; neither
is available here, so these generators stand in for them with the sizes and
structure of the workloads this package is measured on.

This module is shared by the tests, the benchmark and the oracle-driving code.
It contains no step of the PDHG method: only random numbers, sparsity
patterns and the two products that define ``b`` and ``c``.

Random numbers come from a counter-based SplitMix64 stream: draw ``i`` of
stream ``s`` under seed ``seed`` is ``mix64(key(seed, s) + (i + 1) * GAMMA)``,
with ``mix64`` the SplitMix64 finaliser (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014). Every random
quantity is indexed by what it belongs to (column, slot, row), so the LP does
not depend on the order in which it is built.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream ids
S_ROWS, S_SIGN, S_MAG, S_SUPPORT, S_XS, S_ZS, S_YS, S_ZIPF, S_SIZES, S_TARGET = range(1, 11)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _key(seed: int, stream: int) -> np.uint64:
    s = np.array([(int(seed) * 0x100000001B3 + int(stream) * 0x1F123BB5) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _mix64(s)[0]


def rand_bits(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """64 random bits for each counter in ``idx`` (uint64)."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(_key(seed, stream) + (idx + np.uint64(1)) * GAMMA)


def rand_uniform(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits."""
    return (rand_bits(seed, stream, idx) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def rand_normal(seed: int, stream: int, idx: np.ndarray) -> np.ndarray:
    """Standard normals by Box-Muller from draws 2i and 2i+1 of the stream."""
    idx = np.asarray(idx, dtype=np.uint64)
    u1 = rand_uniform(seed, stream, 2 * idx)
    u2 = rand_uniform(seed, stream, 2 * idx + np.uint64(1))
    return np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class LP:
    """A standard-form LP in CSR form (rows = constraints) plus its seeded optimum."""

    m: int
    n: int
    row_ptr: np.ndarray  # int64 [m+1]
    col_idx: np.ndarray  # int32 [nnz], sorted within each row, no duplicates
    val: np.ndarray  # float64 [nnz]
    b: np.ndarray  # float64 [m]
    c: np.ndarray  # float64 [n]
    x_star: np.ndarray
    y_star: np.ndarray
    z_star: np.ndarray
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def f_star(self) -> float:
        return float(self.c @ self.x_star)

    def dense(self) -> np.ndarray:
        A = np.zeros((self.m, self.n))
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        A[rows, self.col_idx] = self.val
        return A


def _distinct_rows(seed: int, m: int, col_of_slot: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """Rows for every slot, distinct within a column (redraw duplicates)."""
    nnz = col_of_slot.size
    if np.any(counts > m):
        raise ValueError("column count exceeds m")
    slots = np.arange(nnz, dtype=np.uint64)
    rows = np.floor(rand_uniform(seed, S_ROWS, slots) * m).astype(np.int64)
    attempt = 0
    while True:
        key = col_of_slot.astype(np.int64) * m + rows
        order = np.lexsort((np.arange(nnz), key))
        ks = key[order]
        dup = np.nonzero(ks[1:] == ks[:-1])[0] + 1
        if dup.size == 0:
            return rows
        attempt += 1
        redo = order[dup]
        ctr = redo.astype(np.uint64) + np.uint64(attempt) * np.uint64(nnz)
        rows[redo] = np.floor(rand_uniform(seed, S_ROWS, ctr) * m).astype(np.int64)
        if attempt > 10000:  # pragma: no cover - impossible for counts << m
            raise RuntimeError("row draw did not terminate")


def zipf_tail(s: float, cap: int) -> np.ndarray:
    """P(Z >= k) for k = 1..cap, Z ~ Zipf(s) on {1, 2, ...}."""
    from scipy.special import zeta

    k = np.arange(1, cap + 1, dtype=np.float64)
    return zeta(s, k) / zeta(s, 1.0)


def zipf_draws(seed: int, n: int, s: float, cap: int) -> np.ndarray:
    """min(Z_j, cap) for j < n, Z_j ~ Zipf(s) by inversion of the tail (float64)."""
    tail = zipf_tail(s, cap)
    u = 1.0 - rand_uniform(seed, S_ZIPF, np.arange(n, dtype=np.uint64))  # (0, 1]
    # Z = largest k with tail[k] >= u; tail is decreasing, so search the reversed array.
    rev = tail[::-1]
    pos = np.searchsorted(rev, u, side="left")  # rev[pos-1] < u <= rev[pos]
    Z = cap - pos  # index into tail
    return np.clip(Z, 1, cap).astype(np.float64)


def zipf_exact_counts(seed: int, n: int, s: float, cap: int, m: int) -> np.ndarray:
    """The literal capped Zipf law: k_j = min(Z_j, cap, m), the draws of
    ``zipf_column_counts`` without its rescaling (mean count
    sum_{k <= cap} P(Z >= k), about 153 for s = 1.5 and cap = 1e4)."""
    return np.minimum(zipf_draws(seed, n, s, cap), m).astype(np.int64)


def zipf_column_counts(seed: int, n: int, s: float, cap: int, nnz_target: int, m: int) -> np.ndarray:
    """Per-column counts k_j = max(1, rint(alpha * min(Z_j, cap))), Z_j ~ Zipf(s),
    with alpha chosen by bisection so that sum_j k_j is as close as possible to
    ``nnz_target``. The shape of the tail is the Zipf law; alpha only rescales it
    so that the mean count matches the requested nnz."""
    Z = zipf_draws(seed, n, s, cap)

    zu, zn = np.unique(Z, return_counts=True)

    def counts(alpha, z):
        return np.minimum(np.maximum(1, np.rint(alpha * z)), m).astype(np.int64)

    def total(alpha):
        return int((counts(alpha, zu) * zn).sum())

    lo, hi = 0.0, float(m)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) < nnz_target:
            lo = mid
        else:
            hi = mid
    a = hi if abs(total(hi) - nnz_target) <= abs(total(lo) - nnz_target) else lo
    return counts(a, Z)


def generate(
    m: int,
    n: int,
    seed: int,
    *,
    nnz_per_col: int | None = 5,
    zipf: tuple[float, int, int] | None = None,
    val_range: tuple[float, float] = (0.1, 1.0),
    support: int | float = 0.3,
    star_range: tuple[float, float] = (0.5, 2.0),
    fp32_values: bool = False,
    name: str = "",
) -> LP:
    """Generate an LP.

    nnz_per_col: fixed number of distinct rows per column (uniform rows).
    zipf:        (s, cap, nnz_target) for power-law column counts instead.
    val_range:   entries are +-U[lo, hi] with a fair random sign.
    support:     number (int) or fraction (float) of columns with x*_j > 0.
    fp32_values: round A's values to FP32 (kept in float64) so that FP32 and
                 FP64 engines solve the same LP.
    """
    if zipf is not None:
        counts = zipf_column_counts(seed, n, zipf[0], zipf[1], zipf[2], m)
    else:
        counts = np.full(n, int(nnz_per_col), dtype=np.int64)
    nnz = int(counts.sum())
    col_of_slot = np.repeat(np.arange(n, dtype=np.int64), counts)
    rows = _distinct_rows(seed, m, col_of_slot, counts)
    slots = np.arange(nnz, dtype=np.uint64)
    lo, hi = val_range
    mag = lo + (hi - lo) * rand_uniform(seed, S_MAG, slots)
    sign = np.where((rand_bits(seed, S_SIGN, slots) >> np.uint64(63)) == np.uint64(1), -1.0, 1.0)
    vals = sign * mag
    if fp32_values:
        vals = vals.astype(np.float32).astype(np.float64)

    # CSR by (row, col)
    order = np.argsort(rows * n + col_of_slot, kind="stable")
    r_sorted = rows[order]
    col_idx = col_of_slot[order].astype(np.int32)
    val = vals[order]
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(r_sorted, minlength=m), out=row_ptr[1:])

    # seeded optimum
    n_sup = int(support) if isinstance(support, (int, np.integer)) else int(round(float(support) * n))
    keys = rand_bits(seed, S_SUPPORT, np.arange(n, dtype=np.uint64))
    sup = np.argsort(keys, kind="stable")[:n_sup]
    on = np.zeros(n, dtype=bool)
    on[sup] = True
    jj = np.arange(n, dtype=np.uint64)
    slo, shi = star_range
    x_star = np.where(on, slo + (shi - slo) * rand_uniform(seed, S_XS, jj), 0.0)
    z_star = np.where(on, 0.0, slo + (shi - slo) * rand_uniform(seed, S_ZS, jj))
    y_star = rand_normal(seed, S_YS, np.arange(m, dtype=np.uint64))

    b = np.bincount(r_sorted, weights=val * x_star[col_idx], minlength=m).astype(np.float64)
    c = np.bincount(col_idx, weights=val * y_star[r_sorted], minlength=n).astype(np.float64) + z_star
    return LP(m, n, row_ptr, col_idx, val, b, c, x_star, y_star, z_star, name=name)


# ---------------------------------------------------------------------------
# The workloads (sizes and structure of the configurations this package is
# measured on).
# ---------------------------------------------------------------------------

def tiny_lp(seed: int = 0) -> LP:
    """m=200, n=500, 5 distinct uniform rows per column, values +-U[0.1,1],
    x* on 150 columns U[0.5,2], z* U[0.5,2] on the other 350, y* ~ N(0,1)."""
    return generate(200, 500, seed, nnz_per_col=5, val_range=(0.1, 1.0), support=150, name=f"tiny-200x500-s{seed}")


def large_lp(seed: int = 0, m: int = 1_000_000, n: int = 3_000_000, nnz: int = 30_000_000,
             fp32_values: bool = False) -> LP:
    """m=1e6, n=3e6, nnz~3e7, Zipf(s=1.5, cap 1e4)-shaped column counts rescaled to
    the nnz target, uniform rows, values +-U[0.1,10], 30% of x* positive."""
    return generate(m, n, seed, nnz_per_col=None, zipf=(1.5, 10_000, nnz), val_range=(0.1, 10.0),
                    support=0.3, fp32_values=fp32_values, name=f"zipf-{m}x{n}-nnz{nnz}-s{seed}")


def batch_sizes(seed: int, count: int = 256, m_lo: float = 1e3, m_hi: float = 1e5) -> list[int]:
    """Row counts log-uniform in [m_lo, m_hi] for a batch of LPs."""
    u = rand_uniform(seed, S_SIZES, np.arange(count, dtype=np.uint64))
    return [int(round(math.exp(math.log(m_lo) + (math.log(m_hi) - math.log(m_lo)) * ui))) for ui in u]


def batch_lp(seed: int, i: int, m: int) -> LP:
    """Instance i of a batch: n = 2.5 m, 5 nnz per column, tiny-LP value ranges,
    30% support."""
    n = int(round(2.5 * m))
    return generate(m, n, seed * 1000 + i, nnz_per_col=5, val_range=(0.1, 1.0), support=0.3,
                    name=f"batch-{seed}-{i}-{m}x{n}")


def adjoint_lp(seed: int = 0, m: int = 100_000, n: int = 300_000, nnz_per_col: int = 6) -> LP:
    """m=1e5, n=3e5, 6 nnz per column, tiny-LP value ranges, 30% support; values
    rounded to FP32 so an FP32 forward pass sees exactly this LP."""
    return generate(m, n, seed, nnz_per_col=nnz_per_col, val_range=(0.1, 1.0), support=0.3,
                    fp32_values=True, name=f"adjoint-{m}x{n}-s{seed}")


def x_target(lp: LP, seed: int, scale: float = 0.01) -> np.ndarray:
    """x* + N(0, scale^2) noise for the unrolled-PDHG loss."""
    return lp.x_star + scale * rand_normal(seed, S_TARGET, np.arange(lp.n, dtype=np.uint64))


# ---------------------------------------------------------------------------
# The same recipe as torch tensor operations on any torch device, for LPs too
# large to build in host memory (the literal capped-Zipf variant of the large
# workload has ~4.6e8 entries; the numpy build above would need ~40 GB of host
# memory). Same counters and streams: the matrix, x* and z* equal generate()'s
# bit for bit; y*, b and c agree to rounding (torch's log1p and cos, and its
# summation order). 64-bit draws are held as int64 bit patterns; products wrap
# modulo 2^64 like the uint64 arithmetic above, and right shifts are logical.
# ---------------------------------------------------------------------------

def _s64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


_GAMMA_S, _M1_S, _M2_S = _s64(int(GAMMA)), _s64(int(_M1)), _s64(int(_M2))


def _shr(z, k: int):
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64_t(z):
    z = (z ^ _shr(z, 30)) * _M1_S
    z = (z ^ _shr(z, 27)) * _M2_S
    return z ^ _shr(z, 31)


def rand_bits_t(seed: int, stream: int, idx):
    """``rand_bits`` for an int64 tensor of counters (bit patterns in int64)."""
    return _mix64_t(_s64(int(_key(seed, stream))) + (idx + 1) * _GAMMA_S)


def rand_uniform_t(seed: int, stream: int, idx):
    import torch

    return _shr(rand_bits_t(seed, stream, idx), 11).to(torch.float64) * (2.0 ** -53)


def rand_normal_t(seed: int, stream: int, idx):
    import torch

    u1 = rand_uniform_t(seed, stream, 2 * idx)
    u2 = rand_uniform_t(seed, stream, 2 * idx + 1)
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)


@dataclasses.dataclass
class TorchLP:
    """An LP of the generator as torch tensors on one device (CSR by rows)."""

    m: int
    n: int
    row_ptr: "object"  # int64 [m+1]
    col_idx: "object"  # int32 [nnz]
    val: "object"  # float64 [nnz]
    b: "object"
    c: "object"
    x_star: "object"
    y_star: "object"
    z_star: "object"
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    @property
    def f_star(self) -> float:
        return float((self.c * self.x_star).sum())


def generate_t(m: int, n: int, seed: int, counts: np.ndarray, *, val_range=(0.1, 1.0), support=0.3,
               star_range=(0.5, 2.0), device="cuda", name: str = "") -> TorchLP:
    """``generate`` with the given per-column counts, as torch operations on
    ``device``."""
    import torch

    counts = np.asarray(counts, dtype=np.int64)
    if np.any(counts > m):
        raise ValueError("column count exceeds m")
    nnz = int(counts.sum())
    ct = torch.as_tensor(counts, device=device)
    col = torch.repeat_interleave(torch.arange(n, device=device, dtype=torch.int64), ct)
    slots = torch.arange(nnz, device=device, dtype=torch.int64)
    rows = torch.floor(rand_uniform_t(seed, S_ROWS, slots) * m).to(torch.int64)
    # rows distinct within a column: of equal (column, row) pairs the later
    # slots are drawn again, from counters past the earlier attempts'
    attempt = 0
    while True:
        ks, order = torch.sort(col * m + rows, stable=True)
        dup = torch.nonzero(ks[1:] == ks[:-1]).squeeze(1) + 1
        del ks
        if dup.numel() == 0:
            break
        attempt += 1
        redo = order[dup]
        rows[redo] = torch.floor(rand_uniform_t(seed, S_ROWS, redo + attempt * nnz) * m).to(torch.int64)
        if attempt > 10000:  # pragma: no cover - impossible for counts << m
            raise RuntimeError("row draw did not terminate")
    del order
    lo, hi = val_range
    vals = lo + (hi - lo) * rand_uniform_t(seed, S_MAG, slots)
    vals = torch.where(_shr(rand_bits_t(seed, S_SIGN, slots), 63) == 1, -vals, vals)
    del slots
    # the optimum
    n_sup = int(support) if isinstance(support, (int, np.integer)) else int(round(float(support) * n))
    jj = torch.arange(n, device=device, dtype=torch.int64)
    # unsigned order of the 64-bit keys: flip the sign bit, then sort as int64
    keys = rand_bits_t(seed, S_SUPPORT, jj) ^ _s64(1 << 63)
    on = torch.zeros(n, dtype=torch.bool, device=device)
    on[torch.sort(keys, stable=True).indices[:n_sup]] = True
    slo, shi = star_range
    x_star = torch.where(on, slo + (shi - slo) * rand_uniform_t(seed, S_XS, jj), torch.zeros((), dtype=torch.float64,
                                                                                          device=device))
    z_star = torch.where(on, torch.zeros((), dtype=torch.float64, device=device),
                         slo + (shi - slo) * rand_uniform_t(seed, S_ZS, jj))
    y_star = rand_normal_t(seed, S_YS, torch.arange(m, device=device, dtype=torch.int64))
    # c = A^T y* + z*, summed column by column in slot order
    coff = torch.zeros(n + 1, dtype=torch.int64, device=device)
    coff[1:] = torch.cumsum(ct, 0)
    c = torch.segment_reduce(vals * y_star[rows], "sum", offsets=coff) + z_star
    # CSR by (row, col); b = A x*, summed row by row
    order = torch.sort(rows * n + col, stable=True).indices
    r_sorted = rows[order]
    col_idx = col[order].to(torch.int32)
    val = vals[order]
    del rows, col, vals, order
    row_ptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    row_ptr[1:] = torch.cumsum(torch.bincount(r_sorted, minlength=m), 0)
    del r_sorted
    b = torch.segment_reduce(val * x_star[col_idx.to(torch.int64)], "sum", offsets=row_ptr)
    return TorchLP(m, n, row_ptr, col_idx, val, b, c, x_star, y_star, z_star, name=name)


def zipf_exact_lp_t(seed: int = 0, m: int = 1_000_000, n: int = 3_000_000, device="cuda") -> TorchLP:
    """The large workload with the literal capped Zipf law for the column
    counts (s = 1.5, cap 1e4: nnz ~4.6e8 at n = 3e6), uniform rows, values
    +-U[0.1,10], 30% of x* positive, built on ``device``."""
    counts = zipf_exact_counts(seed, n, 1.5, 10_000, m)
    return generate_t(m, n, seed, counts, val_range=(0.1, 10.0), support=0.3, device=device,
                      name=f"zipf-exact-{m}x{n}-nnz{int(counts.sum())}-s{seed}")
