"""The literal-order step (DCD_FLAG_LITERAL) against the FP64 oracle.

In the literal order (Algorithms 2 and 4 as printed) each outer step stores
the m x sb block U_k / Q_k, forms U_j^T alpha_sk from it, reads the Gram as
G_k = V_k^T U_k and keeps no gradient between steps.  The fused step instead
contracts the block in the tensor-core epilogue into a cached gradient; both
compute the same iterates in exact arithmetic.
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


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x)).cuda()


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("b,s", [(4, 1), (8, 5), (16, 16), (32, 3)])
def test_literal_bdcd_fp64_matches_algorithm4(b, s):
    p = inputs.krr_dense(m=400, n=21, seed=51, dtype=np.float64)
    kb, ko = B().kernel("rbf", gamma=0.6), oracle.kernel("rbf", gamma=0.6)
    H = 7 * s + (s - 1)  # a shorter last outer step when s > 1
    al, gr, st, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 1e-2, b, s, H, seed=5, prec="fp64",
                                  flags=B().FLAG_LITERAL)
    want = oracle.sstep_bdcd_krr(p.A, p.y, ko, 1e-2, b, s, H, seed=5)
    assert st["iters_done"] == H
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.krr_gradient(p.A, p.y, ko, 1e-2, al.cpu().numpy())
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.linalg.norm(p.y)


@pytest.mark.parametrize("loss,s", [(1, 1), (1, 16), (2, 7)])
def test_literal_dcd_fp64_matches_algorithm2(loss, s):
    p = inputs.blobs(m=300, n=12, seed=52)
    kb, ko = B().kernel("rbf", gamma=0.2), oracle.kernel("rbf", gamma=0.2)
    H = 9 * s + 1
    al, gr, st, _ = B().svm_solve(dev(p.A), dev(p.y), kb, loss, 0.8, s, H, seed=6, prec="fp64",
                                  flags=B().FLAG_LITERAL)
    want = oracle.sstep_dcd_svm(p.A, p.y, ko, loss, 0.8, s, H, seed=6)
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.svm_gradient(p.A, p.y, ko, loss, 0.8, al.cpu().numpy())
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.sqrt(len(gw))


def test_literal_repeated_indices_small_m():
    """m = 12 with b = 4, s = 16: blocks of one outer step overlap and repeat
    (the V^T V terms), read from the stored block's rows."""
    p = inputs.krr_dense(m=12, n=3, seed=6, dtype=np.float64)
    kb, ko = B().kernel("rbf", gamma=0.7), oracle.kernel("rbf", gamma=0.7)
    al, _, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.1, 4, 16, 37, seed=4, prec="fp64", start_iter=3,
                                flags=B().FLAG_LITERAL)
    want = oracle.sstep_bdcd_krr(p.A, p.y, ko, 0.1, 4, 16, 37, seed=4, first_block=3)
    assert rel(al.cpu().numpy(), want) < 1e-10


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_literal_mixed_matches_oracle(prec):
    """Tensor-core block stored in FP32 (the store form), U^T alpha in FP64:
    the mixed-precision targets (alpha 1e-4, dual objective 1e-6)."""
    p = inputs.krr_dense(m=1000, n=64, seed=12, dtype=np.float32)
    A64 = p.A.astype(np.float64)
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    al, _, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 1e-2, 16, 16, 640, seed=3, prec=prec,
                                flags=B().FLAG_LITERAL)
    want = oracle.bdcd_krr(A64, p.y, ko, 1e-2, 16, 640, seed=3)
    a = al.cpu().numpy()
    assert rel(a, want) < 1e-4
    f, fw = oracle.krr_objective(A64, p.y, ko, 1e-2, a), oracle.krr_objective(A64, p.y, ko, 1e-2, want)
    assert abs(f - fw) <= 1e-6 * abs(fw)


def test_literal_rejects_a_tolerance():
    p = inputs.krr_dense(m=50, n=3, seed=1, dtype=np.float64)
    with pytest.raises(B().DcdError) as e:
        B().krr_solve(dev(p.A), dev(p.y), B().kernel("rbf", gamma=1.0), 0.1, 4, 2, 10, prec="fp64", tol=1e-6,
                      check_every=1, flags=B().FLAG_LITERAL)
    assert e.value.status == B().EINVAL
