"""CSR data matrices: the CUDA-core SpMM kernel block and the solves on it,
against the FP64 oracle on the same matrix in dense form."""
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
    t = torch.from_numpy(np.ascontiguousarray(x))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def ragged_csr(m, n, seed, max_nnz=9, empty_every=7, dtype=np.float64):
    """Rows of 0..max_nnz distinct sorted columns (every empty_every-th row
    empty), values N(0, 0.3)."""
    g = np.random.default_rng(seed)
    rp, ci, va = [0], [], []
    for i in range(m):
        k = 0 if i % empty_every == 3 else int(g.integers(1, max_nnz + 1))
        cols = np.sort(g.choice(n, size=k, replace=False))
        ci.extend(cols.tolist())
        va.extend((g.standard_normal(k) * 0.3).tolist())
        rp.append(len(ci))
    return inputs.CsrProblem(np.array(rp, np.int64), np.array(ci, np.int32), np.array(va, dtype), n,
                             np.where(g.random(m) < 0.5, -1.0, 1.0))


def to_lib(p, dtype=np.float64, host=False):
    v = p.values.astype(dtype)
    if host:
        return B().Csr(p.row_ptr.copy(), p.col_idx.copy(), v, p.n)
    return B().Csr(dev(p.row_ptr), dev(p.col_idx), dev(v), p.n)


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


KERNELS = [("rbf", dict(gamma=0.7)), ("poly", dict(coef0=1.0, degree=3)), ("linear", {})]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 2e-6)])
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_csr_kernel_block_matches_dense_oracle(prec, tol, kind, kw):
    p = ragged_csr(157, 90, seed=1)
    A = p.to_dense()
    g = np.random.default_rng(2)
    cols = g.integers(0, p.m, size=45)  # repeats allowed
    rows = g.integers(0, p.m, size=70)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    Acsr = to_lib(p, np.float64 if prec == "fp64" else np.float32)
    got = B().kernel_block(Acsr, kb, prec, dev(cols, torch.int32), rows=dev(rows, torch.int32)).cpu().numpy()
    Ar = A if prec == "fp64" else A.astype(np.float32).astype(np.float64)
    want = oracle.kernel_block(ko, Ar, cols, rows=rows)
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 2e-6)])
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_csr_kernel_block_apply(prec, tol, kind, kw):
    p = ragged_csr(301, 64, seed=3, max_nnz=20)
    A = p.to_dense()
    g = np.random.default_rng(4)
    cols = g.integers(0, p.m, size=70)  # more than one column pass of 32
    w = g.standard_normal(70)
    rs = np.where(g.random(p.m) < 0.5, -1.0, 1.0)
    g0 = g.standard_normal(p.m)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    gd = dev(g0)
    B().kernel_block_apply(to_lib(p, np.float64 if prec == "fp64" else np.float32), kb, prec,
                           dev(cols, torch.int32), dev(w), gd, rowscale=dev(rs))
    Ar = A if prec == "fp64" else A.astype(np.float32).astype(np.float64)
    Kb = oracle.kernel_block(ko, Ar, cols)
    want = g0 + rs * (Kb @ w)
    scale = np.max(np.abs(Kb)) * np.sum(np.abs(w))
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= tol * scale


def test_csr_long_rows_overflow_the_hit_list():
    # rows denser than the per-warp hit list: the list is flushed mid-tile
    p = ragged_csr(70, 40, seed=5, max_nnz=40, empty_every=1000)
    A = p.to_dense()
    cols = np.arange(0, 70, 3)
    kb, ko = B().kernel("poly", coef0=1.0, degree=2), oracle.kernel("poly", coef0=1.0, degree=2)
    got = B().kernel_block(to_lib(p), kb, "fp64", dev(cols, torch.int32)).cpu().numpy()
    want = oracle.kernel_block(ko, A, cols)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("s", [1, 16, 32])
def test_csr_dcd_svm_l2_fp64_iterates_match_oracle(s):
    """Config-3 shape in miniature: squared hinge, poly (a.b+1)^3, C = 0.5."""
    p = inputs.sparse_csr(m=400, n=300, nnz_per_row=12, seed=6)
    A = p.to_dense()
    kb, ko = B().kernel("poly", coef0=1.0, degree=3), oracle.kernel("poly", coef0=1.0, degree=3)
    al, gr, st, _ = B().svm_solve(to_lib(p, np.float64), dev(p.y), kb, 2, 0.5, s, 1500, seed=4, prec="fp64")
    want = oracle.sstep_dcd_svm(A, p.y, ko, 2, 0.5, s, 1500, seed=4)
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.svm_gradient(A, p.y, ko, 2, 0.5, want)
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.sqrt(len(gw))


def test_csr_dcd_svm_fp32_block_matches_oracle():
    p = inputs.sparse_csr(m=500, n=400, nnz_per_row=10, seed=7)
    A = p.to_dense().astype(np.float32).astype(np.float64)
    kb, ko = B().kernel("poly", coef0=1.0, degree=3), oracle.kernel("poly", coef0=1.0, degree=3)
    al, _, _, _ = B().svm_solve(to_lib(p, np.float32), dev(p.y), kb, 2, 0.5, 16, 2000, seed=1, prec="bf16x3")
    want = oracle.sstep_dcd_svm(A, p.y, ko, 2, 0.5, 16, 2000, seed=1)
    a = al.cpu().numpy()
    assert rel(a, want) < 1e-5
    f = oracle.svm_objectives(A, p.y, ko, 2, 0.5, a)
    fw = oracle.svm_objectives(A, p.y, ko, 2, 0.5, want)
    assert abs(f["dual"] - fw["dual"]) <= 1e-7 * abs(fw["dual"])


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_csr_bdcd_krr_matches_oracle(prec, tol):
    p = ragged_csr(300, 50, seed=8, max_nnz=15)
    A = p.to_dense()
    y = np.random.default_rng(9).standard_normal(p.m)
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    al, _, _, _ = B().krr_solve(to_lib(p, np.float64 if prec == "fp64" else np.float32), dev(y), kb, 0.05, 4, 8,
                                200, seed=2, prec=prec)
    Ar = A if prec == "fp64" else A.astype(np.float32).astype(np.float64)
    want = oracle.bdcd_krr(Ar, y, ko, 0.05, 4, 200, seed=2)
    assert rel(al.cpu().numpy(), want) < tol


def test_csr_host_io_matches_device():
    p = ragged_csr(200, 60, seed=10)
    y = np.random.default_rng(11).standard_normal(p.m)
    kb = B().kernel("rbf", gamma=0.3)
    ad, gd, _, _ = B().krr_solve(to_lib(p), dev(y), kb, 0.05, 4, 4, 80, seed=1, prec="fp64")
    ah, gh, _, _ = B().krr_solve(to_lib(p, host=True), y.copy(), kb, 0.05, 4, 4, 80, seed=1, prec="fp64",
                                 flags=B().FLAG_HOST_IO)
    assert np.array_equal(ad.cpu().numpy(), ah) and np.array_equal(gd.cpu().numpy(), gh)


@pytest.mark.parametrize("what", ["column", "offsets"])
def test_csr_invalid_arrays_are_rejected(what):
    p = ragged_csr(50, 30, seed=12)
    ci, rp = p.col_idx.copy(), p.row_ptr.copy()
    if what == "column":
        ci[5] = 30  # == n
    else:
        rp[10], rp[11] = rp[11], rp[10] - 1  # a decreasing pair
    A = B().Csr(dev(rp), dev(ci), dev(p.values), p.n)
    with pytest.raises(B().DcdError) as e:
        B().krr_solve(A, dev(np.ones(p.m)), B().kernel("linear"), 0.1, 2, 2, 10, prec="fp64")
    assert e.value.status == B().EINVAL
