"""The accurate apply epilogue (DCD_PREC_REFRESH) against the FP64 oracle.

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
@pytest.mark.parametrize("m,ncols,n", [(333, 45, 45), (3000, 600, 96), (1100, 300, 300), (500, 100, 1100)])
def test_accurate_apply_matches_oracle(kind, kw, m, ncols, n):
    """g += rs * K(A, A_cols) w against the oracle's kernel of the FP32 data
    (not of a rounded operand): ragged row tiles, N-chunks and k-blocks;
    n = 1100 takes the split-tf32 products (beyond the exact slice sums)."""
    g = np.random.default_rng(m + ncols)
    A = (g.standard_normal((m, n)) * (0.25 if kind != "rbf" else 1.0 / np.sqrt(n))).astype(np.float32)
    cols = g.integers(0, m, size=ncols)
    w = g.standard_normal(ncols)
    rs = np.where(g.random(m) < 0.5, -1.0, 1.0)
    g0 = g.standard_normal(m)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    gd = dev(g0)
    B().kernel_block_apply(dev(A), kb, "refresh", dev(cols, torch.int32), dev(w), gd, rowscale=dev(rs))
    Kb = oracle.kernel_block(ko, A.astype(np.float64), cols)
    want = g0 + rs * (Kb @ w)
    scale = np.max(np.abs(Kb)) * np.sum(np.abs(w))
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= 1e-6 * scale


def cancellation_case(m=3000, n=128, lam=1e-3, seed=41):
    p = inputs.krr_dense(m=m, n=n, seed=seed, dtype=np.float32)
    ko = oracle.kernel("rbf", gamma=0.5)
    K = oracle.kernel_block(ko, p.A.astype(np.float64), np.arange(m))
    star = np.linalg.solve(K / lam + m * np.eye(m), p.y)
    return p, K, star / lam


@pytest.fixture(scope="module")
def cancel():
    return cancellation_case()


@pytest.mark.parametrize("prec,tol", [("refresh", 5e-7), ("tf32x3", 1e-5)])
def test_apply_under_cancellation(cancel, prec, tol):
    """K w with w = alpha*/lambda of the closed form (sum_j |K_ij w_j| is
    hundreds of times the result): relative 2-norm error of K w.  The
    recomputed-gradient arithmetic leaves the FP32 rounding of the kernel
    values; the split-tf32 products carry the tensor cores' FP32 accumulation
    error of the dot products, ~1.7e-7 per entry, which the cancellation
    multiplies."""
    p, K, w = cancel
    m = K.shape[0]
    want = K @ w
    gd = torch.zeros(m, dtype=torch.float64, device="cuda")
    B().kernel_block_apply(dev(p.A), B().kernel("rbf", gamma=0.5), prec,
                           torch.arange(m, dtype=torch.int32, device="cuda"), dev(w), gd)
    err = np.linalg.norm(gd.cpu().numpy() - want) / np.linalg.norm(want)
    print(prec, "relative error of K w under cancellation", err)
    assert err <= tol


@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_refreshed_solve_meets_tolerance_in_fp64(prec):
    """A mixed solve with DCD_FLAG_REFRESH (the bench's time-to-tolerance
    setting, scaled down: m = 4000, n = 256, sigma = 1, lambda = 1e-4, b = 16,
    s = 64) must meet relative residual 1e-6 on the oracle's FP64 gradient
    of the alpha it returns, and report that gradient's metric.  Plain bf16
    steps converge too: every recomputation restarts the cached gradient from
    the exact one (iterative refinement)."""
    p = inputs.krr_dense(m=4000, n=256, seed=43, dtype=np.float32)
    lam, tol = 1e-4, 1e-6
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        al, gr, st, rc = B().krr_solve(dev(p.A), dev(p.y), kb, lam, 16, 64, 2000000, seed=3, prec=prec, tol=tol,
                                       check_every=4, flags=B().FLAG_REFRESH, stream=side.cuda_stream)
        side.synchronize()
    assert rc == B().OK and st["converged"] == 1 and st["refreshes"] >= 1
    a = al.cpu().numpy()
    gw = oracle.krr_gradient(p.A.astype(np.float64), p.y, ko, lam, a)
    true = np.linalg.norm(gw) / np.linalg.norm(p.y)
    print(prec, "converged after", st["iters_done"], "block updates, refreshes", st["refreshes"],
          "reported", st["final_metric"], "FP64", true)
    assert true <= tol
    assert abs(true - st["final_metric"]) <= 0.1 * tol
