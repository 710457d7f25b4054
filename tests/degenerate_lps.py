"""Small LPs where the method's degenerate cases show: primal infeasible (no x
with Ax = b, x >= 0), dual infeasible (cost unbounded below), a pure
feasibility problem (c = 0) and a zero right-hand side (b = 0). Shared by the
oracle pins and the GPU tests."""
import numpy as np

from paper_2510_24429_b300 import lpgen


class Small:
    def __init__(self, dense, b, c, name):
        A = np.asarray(dense, dtype=np.float64)
        self.m, self.n = A.shape
        rows, cols = np.nonzero(A)
        self.row_ptr = np.zeros(self.m + 1, dtype=np.int64)
        np.cumsum(np.bincount(rows, minlength=self.m), out=self.row_ptr[1:])
        self.col_idx = cols.astype(np.int32)
        self.val = A[rows, cols]
        self.b = np.asarray(b, dtype=np.float64)
        self.c = np.asarray(c, dtype=np.float64)
        self.dense = A
        self.name = name


def infeasible_2x2():
    """x1 + x2 = 1 and x1 + x2 = 2: Farkas certificate y = (-1, 1)/sqrt(2)
    (A^T y = 0, b^T y > 0), the only one up to scale."""
    return Small([[1, 1], [1, 1]], [1, 2], [0, 0], "infeasible-2x2")


def unbounded_1x2():
    """min -x1 s.t. x1 - x2 = 0, x >= 0: ray d = (1, 1)/sqrt(2) (A d = 0,
    d >= 0, c^T d < 0), the only one up to scale."""
    return Small([[1, -1]], [0], [-1, 0], "unbounded-1x2")


def infeasible_tiny(seed=0):
    """The tiny generator LP with its first nonempty row repeated with right-hand
    side b_i + 1: infeasible; y = e_new - e_i is a Farkas certificate."""
    lp = lpgen.tiny_lp(seed)
    import scipy.sparse as sp

    A = sp.csr_matrix((lp.val, lp.col_idx, lp.row_ptr), shape=(lp.m, lp.n)).toarray()
    i = int(np.flatnonzero(np.abs(A).sum(axis=1) > 0)[0])
    A2 = np.vstack([A, A[i]])
    b2 = np.concatenate([lp.b, [lp.b[i] + 1.0]])
    return Small(A2, b2, lp.c, "infeasible-tiny")


def zero_objective_tiny(seed=0):
    """The tiny generator LP with c = 0: every feasible x is optimal (x* is one)."""
    lp = lpgen.tiny_lp(seed)
    s = Small(np.zeros((1, 1)), [0], [0], "zero-objective-tiny")
    s.m, s.n, s.row_ptr, s.col_idx, s.val = lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val
    s.b, s.c = lp.b.copy(), np.zeros(lp.n)
    return s


def zero_rhs_tiny(seed=0):
    """The tiny generator LP with b = 0 and c = |c| + 0.1 > 0: the optimum is x = 0."""
    lp = lpgen.tiny_lp(seed)
    s = Small(np.zeros((1, 1)), [0], [0], "zero-rhs-tiny")
    s.m, s.n, s.row_ptr, s.col_idx, s.val = lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val
    s.b, s.c = np.zeros(lp.m), np.abs(lp.c) + 0.1
    return s
