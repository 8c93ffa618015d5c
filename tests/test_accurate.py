"""The accurate apply epilogue (DCD_PREC_TF32X3A) against the FP64 oracle.

It serves the gradient recomputed under DCD_FLAG_REFRESH, where the result
g = K w / lambda + m alpha - y is a small difference of large terms: the
coefficients w = alpha / lambda of a converged K-RR solve have mixed signs
and sum_j |K_ij w_j| is hundreds of times |sum_j K_ij w_j|.  The accurate
epilogue forms the exponent and the kernel value in double-single
arithmetic and contracts in double-single with FP64 coefficients, leaving
the split-tf32 dot products (FP32-accumulated in the tensor cores) as the
main error.
"""
import numpy as np
import pytest

import oracle
from paper_2406_18001_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def B():
    from paper_2406_18001_gb300 import binding
    return binding


def dev(x, dtype=None):
    t = torch.as_tensor(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


KERNELS = [("rbf", dict(gamma=0.35)), ("poly", dict(coef0=1.0, degree=3)), ("linear", {})]


@pytest.mark.parametrize("kind,kw", KERNELS)
@pytest.mark.parametrize("m,ncols,n", [(333, 45, 45), (3000, 600, 96), (1100, 300, 300)])
def test_accurate_apply_matches_oracle(kind, kw, m, ncols, n):
    """g += rs * K(A, A_cols) w against the oracle's kernel of the FP32 data
    (not of a rounded operand): ragged row tiles, N-chunks and k-blocks."""
    g = np.random.default_rng(m + ncols)
    A = (g.standard_normal((m, n)) * (0.25 if kind != "rbf" else 1.0 / np.sqrt(n))).astype(np.float32)
    cols = g.integers(0, m, size=ncols)
    w = g.standard_normal(ncols)
    rs = np.where(g.random(m) < 0.5, -1.0, 1.0)
    g0 = g.standard_normal(m)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    gd = dev(g0)
    B().kernel_block_apply(dev(A), kb, "tf32x3a", dev(cols, torch.int32), dev(w), gd, rowscale=dev(rs))
    Kb = oracle.kernel_block(ko, A.astype(np.float64), cols)
    want = g0 + rs * (Kb @ w)
    scale = np.max(np.abs(Kb)) * np.sum(np.abs(w))
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= 1e-6 * scale
