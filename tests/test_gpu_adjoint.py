"""Adjoint of K unrolled PDHG iterations (pdhg_backward), against the oracle's
own reverse pass, which is pinned by central finite differences of the
oracle's forward pass. FP64 gradients must agree to 1e-9 relative; the FP32
adjoint's error against the FP64 reverse pass is printed and held to 1e-2."""
import numpy as np
import pytest

from oracle import pdhg_oracle as O
from paper_2510_24429_b300 import lpgen
from paper_2510_24429_b300 import pdhg as P
from tests.gpu_helpers import rel_err

pytestmark = pytest.mark.gpu

OPTS = dict(restarts=0, primal_weight=0, record_for_backward=1)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2510_24429_b300 import build

    build.build()
    P.load()


def _oracle(lp, pc=True):
    return O.Oracle(lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val, lp.b, lp.c,
                    O.Options(restarts=False, primal_weight=False, pock_chambolle=pc))


def _seed(lp, s=11):
    rng = np.random.default_rng(s)
    return rng.standard_normal(lp.n), rng.standard_normal(lp.m)


@pytest.mark.parametrize("K,C", [(120, 50), (50, 50), (7, 3), (1, 50)])
def test_fp64_adjoint_matches_oracle_reverse_pass(tiny_lp, K, C):
    lp = tiny_lp
    wx, wy = _seed(lp)
    gc_o, gb_o = O.unrolled_adjoint(_oracle(lp), K, wx, wy)
    with P.Solver.from_lp(lp, checkpoint_every=C, **OPTS) as sol:
        sol.iterate(K)
        gc, gb = sol.backward(wx, wy)
        # a second reverse pass over the same recording gives the same result
        gc2, gb2 = sol.backward(wx, wy)
    assert rel_err(gc, gc_o) <= 1e-9 and rel_err(gb, gb_o) <= 1e-9
    np.testing.assert_array_equal(gc, gc2)
    np.testing.assert_array_equal(gb, gb2)


def test_fp64_adjoint_on_ragged_lp():
    lp = lpgen.generate(3001, 7919, 5, nnz_per_col=5, support=0.3)
    wx, _ = _seed(lp, 4)
    gc_o, gb_o = O.unrolled_adjoint(_oracle(lp), 75, wx)
    with P.Solver.from_lp(lp, checkpoint_every=50, **OPTS) as sol:
        sol.iterate(75)
        gc, gb = sol.backward(wx)
    assert rel_err(gc, gc_o) <= 1e-9 and rel_err(gb, gb_o) <= 1e-9


def test_fp64_adjoint_against_oracle_finite_differences(tiny_lp):
    lp = tiny_lp
    K, h = 60, 1e-6
    orc = _oracle(lp)
    xt = lpgen.x_target(lp, 7)
    with P.Solver.from_lp(lp, checkpoint_every=25, **OPTS) as sol:
        sol.iterate(K)
        x, _, _ = sol.solution()
        gc, gb = sol.backward(x - xt)
    rng = np.random.default_rng(9)
    checked = 0
    for _ in range(20):
        dc, db = rng.standard_normal(lp.n), rng.standard_normal(lp.m)
        xp, _ = O.unrolled_forward(orc, K, c=lp.c + h * dc, b=lp.b + h * db)
        xm, _ = O.unrolled_forward(orc, K, c=lp.c - h * dc, b=lp.b - h * db)
        if any(np.any((a > 0) != (b_ > 0)) for a, b_ in zip(xp, xm)):
            continue  # the perturbation crosses a kink of max(u, 0)
        fd = (O.unrolled_loss(orc, K, xt, c=lp.c + h * dc, b=lp.b + h * db)
              - O.unrolled_loss(orc, K, xt, c=lp.c - h * dc, b=lp.b - h * db)) / (2 * h)
        assert gc @ dc + gb @ db == pytest.approx(fd, rel=1e-5, abs=1e-9)
        checked += 1
    assert checked >= 15


def test_fp32_adjoint_error_vs_fp64_reverse_pass(tiny_lp):
    lp = lpgen.generate(200, 500, 0, nnz_per_col=5, support=150, fp32_values=True)
    wx, _ = _seed(lp, 2)
    gc_o, gb_o = O.unrolled_adjoint(_oracle(lp), 100, wx)
    with P.Solver.from_lp(lp, precision=P.PDHG_FP32, checkpoint_every=50, **OPTS) as sol:
        sol.iterate(100)
        gc, gb = sol.backward(wx)
    ec, eb = rel_err(gc, gc_o), rel_err(gb, gb_o)
    print(f"FP32 adjoint vs FP64 reverse pass: dL/dc {ec:.2e}, dL/db {eb:.2e}")
    assert ec <= 1e-2 and eb <= 1e-2


def test_autograd_function(tiny_lp):
    import torch

    lp = tiny_lp
    csr = (lp.m, lp.n, lp.row_ptr, lp.col_idx, lp.val)
    xt = torch.tensor(lpgen.x_target(lp, 7), device="cuda")
    for dev in ("cpu", "cuda"):
        c = torch.tensor(lp.c, device=dev, requires_grad=True)
        b = torch.tensor(lp.b, device=dev, requires_grad=True)
        x = P.pdhg_unroll(c, b, csr, 80, checkpoint_every=30)
        loss = 0.5 * ((x.to("cuda") - xt) ** 2).sum()
        loss.backward()
        orc = _oracle(lp)
        xs, _ = O.unrolled_forward(orc, 80)
        gc_o, gb_o = O.unrolled_adjoint(orc, 80, orc.d_c * xs[-1] - xt.cpu().numpy())
        assert rel_err(c.grad.cpu().numpy(), gc_o) <= 1e-8
        assert rel_err(b.grad.cpu().numpy(), gb_o) <= 1e-8


def test_backward_needs_recording(tiny_lp):
    with P.Solver.from_lp(tiny_lp, restarts=0, primal_weight=0) as sol:
        sol.iterate(5)
        with pytest.raises(P.PDHGError) as ei:
            sol.backward(np.zeros(tiny_lp.n))
        assert ei.value.status == P.PDHG_ERR_STATE
    with pytest.raises(P.PDHGError) as ei:
        P.Solver.from_lp(tiny_lp, record_for_backward=1)  # restarts on by default
    assert ei.value.status == P.PDHG_ERR_INVALID
