"""FP8 per-row-scaled storage and the kind::f8f6f4 kernel block: the device
quantiser must give the oracle's codes and scales bit for bit, and the FP8
block and solves must match the FP64 oracle run on the dequantised matrix."""
import numpy as np
import pytest

import oracle

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


def spread_rows(m, n, seed):
    """Rows N(0,1) times a per-row magnitude over 12 decades, one zero row,
    one row with a single nonzero, and a few entries in the e4m3 subnormal
    range of their row."""
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n)) * np.exp(g.uniform(-14, 14, (m, 1)))
    A[min(3, m - 1)] = 0.0
    if m > 7:
        A[7] = 0.0
        A[7, n // 2] = -3.0
    A[:, 0] *= 1e-3
    return A


def fp8_storage(A):
    q, s = oracle.quantize_e4m3_rows(A)
    return q, s, oracle.dequantize_e4m3_rows(q, s)


@pytest.mark.parametrize("dtype", ["f64", "f32", "bf16"])
@pytest.mark.parametrize("m,n", [(1, 1), (300, 77), (129, 256), (40, 1000)])
def test_quantizer_is_bit_exact(dtype, m, n):
    A = spread_rows(m, n, seed=m + n)
    if dtype == "bf16":
        At = dev(A.astype(np.float32), torch.bfloat16)
        Ah = At.float().cpu().numpy()
    else:
        At = dev(A.astype(np.float64 if dtype == "f64" else np.float32))
        Ah = At.cpu().numpy()
    F = B().quantize_e4m3(At)
    q, s = oracle.quantize_e4m3_rows(Ah)
    assert np.array_equal(F.scale.cpu().numpy(), s)
    assert np.array_equal(F.codes.cpu().numpy(), q)


def test_quantizer_rejects_non_finite():
    A = np.ones((10, 20), np.float32)
    A[4, 7] = np.inf
    with pytest.raises(B().DcdError) as e:
        B().quantize_e4m3(dev(A))
    assert e.value.status == B().EINVAL


KERNELS = [("rbf", dict(gamma=0.02)), ("poly", dict(coef0=1.0, degree=3)), ("linear", {})]


def unit_rows(m, n, seed, scale_spread=2.0):
    g = np.random.default_rng(seed)
    A = g.standard_normal((m, n)) / np.sqrt(n)
    return A * np.exp(g.uniform(-scale_spread, scale_spread, (m, 1)))


@pytest.mark.parametrize("kind,kw", KERNELS)
def test_fp8_kernel_block_matches_oracle_on_dequantised_rows(kind, kw):
    A = unit_rows(333, 300, seed=1) * 4.0  # 3 k-blocks of 128 codes, the last ragged
    q, s, D = fp8_storage(A)
    g = np.random.default_rng(2)
    cols = g.integers(0, 333, size=290)  # two N-chunks, repeats allowed
    rows = g.integers(0, 333, size=200)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    F = B().Fp8(dev(q), dev(s))
    got = B().kernel_block(F, kb, "fp8", dev(cols, torch.int32), rows=dev(rows, torch.int32)).cpu().numpy()
    want = oracle.kernel_block(ko, D, cols, rows=rows)
    # exact code products, FP32 accumulation and epilogue
    assert np.max(np.abs(got - want)) <= 2e-5 * np.max(np.abs(want))
    # quantising inside the call gives the same block
    got2 = B().kernel_block(dev(A.astype(np.float32)), kb, "fp8", dev(cols, torch.int32),
                            rows=dev(rows, torch.int32)).cpu().numpy()
    assert np.array_equal(got, got2)


def test_fp8_rbf_diagonal_is_one():
    A = unit_rows(200, 512, seed=3) * 8.0
    q, s, D = fp8_storage(A)
    idx = np.arange(200)
    got = B().kernel_block(B().Fp8(dev(q), dev(s)), B().kernel("rbf", gamma=1 / 128), "fp8",
                           dev(idx, torch.int32)).cpu().numpy()
    # d^2(i, i) = 2 gamma ||a_i||^2 - 2 gamma s_i^2 (q_i.q_i) cancels to rounding: the FP32 norms and
    # scale products (a few ulp u each) plus an FP32 dot of n exact products (~sqrt(n) u)
    u, n = 2.0 ** -24, A.shape[1]
    bound = (4 + np.sqrt(n)) * u * 2 * (1 / 128) * np.sum(D * D, axis=1)
    assert np.all(np.abs(np.diag(got) - 1.0) <= bound)


@pytest.mark.parametrize("kind,kw", KERNELS)
def test_fp8_kernel_block_apply(kind, kw):
    A = unit_rows(517, 130, seed=4) * 3.0
    q, s, D = fp8_storage(A)
    g = np.random.default_rng(5)
    cols = g.integers(0, 517, size=70)
    w = g.standard_normal(70)
    rs = np.where(g.random(517) < 0.5, -1.0, 1.0)
    g0 = g.standard_normal(517)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    gd = dev(g0)
    B().kernel_block_apply(B().Fp8(dev(q), dev(s)), kb, "fp8", dev(cols, torch.int32), dev(w), gd, rowscale=dev(rs))
    Kb = oracle.kernel_block(ko, D, cols)
    want = g0 + rs * (Kb @ w)
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= 2e-5 * np.max(np.abs(Kb)) * np.sum(np.abs(w))


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - b) / np.linalg.norm(b)


@pytest.mark.parametrize("s", [1, 8, 32])
def test_fp8_bdcd_krr_matches_oracle(s):
    """Config-5 shape in miniature: ill-conditioned features, RBF sigma = 8,
    b = 32, FP8 storage; the FP64 oracle runs on the dequantised matrix."""
    from paper_2406_18001_gb300 import inputs
    A = inputs.ill_conditioned(800, 256, seed=6).astype(np.float64)
    q, sc, D = fp8_storage(A)
    y = np.random.default_rng(7).standard_normal(800)
    gam, lam = 1.0 / 128, 1e-3
    kb, ko = B().kernel("rbf", gamma=gam), oracle.kernel("rbf", gamma=gam)
    al, gr, st, _ = B().krr_solve(B().Fp8(dev(q), dev(sc)), dev(y), kb, lam, 32, s, 320, seed=3, prec="fp8")
    want = oracle.bdcd_krr(D, y, ko, lam, 32, 320, seed=3)
    a = al.cpu().numpy()
    assert rel(a, want) < 1e-4
    fo = oracle.krr_objective(D, y, ko, lam, want)
    assert abs(oracle.krr_objective(D, y, ko, lam, a) - fo) <= 1e-6 * abs(fo)
    gw = oracle.krr_gradient(D, y, ko, lam, a)
    assert np.linalg.norm(gr.cpu().numpy() - gw) <= 1e-4 * np.linalg.norm(gw) + 1e-6 * np.linalg.norm(y)


def test_fp8_storage_in_fp64_mode_is_exact_dequantisation():
    A = unit_rows(300, 100, seed=8)
    q, sc, D = fp8_storage(A)
    y = np.random.default_rng(9).standard_normal(300)
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    al, _, _, _ = B().krr_solve(B().Fp8(dev(q), dev(sc)), dev(y), kb, 0.05, 4, 8, 200, seed=2, prec="fp64")
    want = oracle.bdcd_krr(D, y, ko, 0.05, 4, 200, seed=2)
    assert rel(al.cpu().numpy(), want) < 1e-10


@pytest.mark.parametrize("loss", [1, 2])
def test_fp8_dcd_svm_matches_oracle(loss):
    from paper_2406_18001_gb300 import inputs
    p = inputs.blobs(m=500, n=64, seed=10)
    q, sc, D = fp8_storage(p.A)
    kb, ko = B().kernel("rbf", gamma=1 / 128), oracle.kernel("rbf", gamma=1 / 128)
    al, _, _, _ = B().svm_solve(B().Fp8(dev(q), dev(sc)), dev(p.y), kb, loss, 1.0, 16, 3000, seed=1, prec="fp8")
    want = oracle.sstep_dcd_svm(D, p.y, ko, loss, 1.0, 16, 3000, seed=1)
    a = al.cpu().numpy()
    assert rel(a, want) < 1e-4
    f = oracle.svm_objectives(D, p.y, ko, loss, 1.0, a)
    fw = oracle.svm_objectives(D, p.y, ko, loss, 1.0, want)
    assert abs(f["dual"] - fw["dual"]) <= 1e-6 * abs(fw["dual"])


def test_fp8_host_io_matches_device():
    A = unit_rows(200, 140, seed=11)
    q, sc, _ = fp8_storage(A)
    y = np.random.default_rng(12).standard_normal(200)
    kb = B().kernel("rbf", gamma=0.3)
    ad, gd, _, _ = B().krr_solve(B().Fp8(dev(q), dev(sc)), dev(y), kb, 0.05, 4, 4, 80, seed=1, prec="fp8")
    ah, gh, _, _ = B().krr_solve(B().Fp8(q.copy(), sc.copy()), y.copy(), kb, 0.05, 4, 4, 80, seed=1, prec="fp8",
                                 flags=B().FLAG_HOST_IO)
    assert np.array_equal(ad.cpu().numpy(), ah) and np.array_equal(gd.cpu().numpy(), gh)


@pytest.mark.parametrize("what", ["nan_code", "negative_scale"])
def test_fp8_invalid_storage_is_rejected(what):
    q, sc, _ = fp8_storage(unit_rows(50, 30, seed=13))
    if what == "nan_code":
        q[17, 4] = 0x7F
    else:
        sc[9] = -1.0
    with pytest.raises(B().DcdError) as e:
        B().krr_solve(B().Fp8(dev(q), dev(sc)), dev(np.ones(50)), B().kernel("linear"), 0.1, 2, 2, 10, prec="fp8")
    assert e.value.status == B().EINVAL
