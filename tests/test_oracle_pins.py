"""Pins for the FP64 oracle: each check ties it to something other than
itself -- a published test vector, scipy/numpy library routines, closed
forms, brute force on tiny inputs, or an invariant the paper states.

A plausible slip in the oracle (a dropped correction term, a sign, a swapped
index, the wrong omega or nu) fails at least one of these.
"""
import itertools
import os

import numpy as np
import pytest
from scipy import optimize, stats
from scipy.spatial.distance import cdist

import oracle
from paper_2406_18001_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300)


# ----------------------------------------------------------------- RNG ----
def test_splitmix64_published_vector():
    want = [int(x) for x in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"))
            if x.strip() and not x.startswith("#")]
    got = [oracle.splitmix64(1234567, k) for k in range(1, 6)]
    assert got == want


def test_draw_is_splitmix_composition():
    for seed, stream, ctr in [(0, 0, 0), (7, 3, 11), (2**63 + 5, 2**40, 123456789)]:
        start = oracle.splitmix64(seed, 2 * stream + 1)
        assert oracle.draw(seed, stream, ctr) == oracle.splitmix64(start, ctr + 1)


def test_dcd_indices_uniform_and_in_range():
    m = 10
    idx = oracle.sample_dcd(seed=3, m=m, first=0, count=200000)
    assert idx.min() >= 0 and idx.max() < m
    counts = np.bincount(idx, minlength=m)
    assert stats.chisquare(counts).pvalue > 1e-4
    # the stream depends only on (seed, iteration): a suffix equals a later start
    assert np.array_equal(oracle.sample_dcd(3, m, 1000, 50), idx[1000:1050])
    # exact multiply-shift mapping of the raw draws
    for t in (0, 1, 17):
        u = oracle.draw(3, 0, t)
        assert idx[t] == (u * m) >> 64


def test_bdcd_blocks_distinct_and_uniform_subsets():
    m, b, nb = 5, 2, 40000
    blocks = oracle.sample_bdcd(seed=11, m=m, b=b, first_block=0, nblocks=nb)
    assert blocks.min() >= 0 and blocks.max() < m
    assert all(len(set(r)) == b for r in blocks[:2000])
    keys = {c: i for i, c in enumerate(itertools.combinations(range(m), b))}
    counts = np.zeros(len(keys))
    for r in blocks:
        counts[keys[tuple(sorted(r))]] += 1
    assert stats.chisquare(counts).pvalue > 1e-4
    big = oracle.sample_bdcd(seed=1, m=1000, b=32, first_block=5, nblocks=300)
    assert all(len(set(r)) == 32 for r in big)
    assert np.array_equal(oracle.sample_bdcd(1, 1000, 32, 6, 1)[0], big[1])


def test_bdcd_block_of_full_size_is_a_permutation():
    blk = oracle.sample_bdcd(seed=2, m=17, b=17, first_block=3, nblocks=1)[0]
    assert sorted(blk) == list(range(17))


# ------------------------------------------------------------- kernels ----
def test_rbf_matches_scipy_and_unit_diagonal():
    g = np.random.default_rng(0)
    A = g.standard_normal((40, 7))
    cols = np.array([3, 0, 39, 3, 17])
    k = oracle.kernel("rbf", gamma=0.37)
    got = oracle.kernel_block(k, A, cols)
    want = np.exp(-0.37 * cdist(A, A[cols], "sqeuclidean"))
    assert np.max(np.abs(got - want)) < 1e-14
    assert got[3, 0] == 1.0 and got[39, 2] == 1.0


def test_linear_matches_numpy():
    g = np.random.default_rng(1)
    A = g.standard_normal((30, 11))
    cols = np.arange(0, 30, 3)
    got = oracle.kernel_block(oracle.kernel("linear"), A, cols, rows=np.arange(5, 25))
    assert np.max(np.abs(got - A[5:25] @ A[cols].T)) < 1e-13


def test_poly_exact_on_integer_data():
    g = np.random.default_rng(2)
    Ai = g.integers(-3, 4, size=(12, 5))
    k = oracle.kernel("poly", coef0=2.0, degree=3)
    got = oracle.kernel_block(k, Ai.astype(float), np.arange(12))
    for i in range(12):
        for j in range(12):
            assert got[i, j] == float((2 + int(Ai[i] @ Ai[j])) ** 3)


# ------------------------------------------------------------- helpers ----
def full_Q(A, y, kind, **kw):
    if kind == "rbf":
        K = np.exp(-kw["gamma"] * cdist(A, A, "sqeuclidean"))
    elif kind == "poly":
        K = (kw["coef0"] + A @ A.T) ** kw["degree"]
    else:
        K = A @ A.T
    return K, (y[:, None] * y[None, :]) * K


def svm_dual_min(Q, alpha, loss, C):
    f = 0.5 * alpha @ Q @ alpha - alpha.sum()
    if loss == 2:
        f += alpha @ alpha / (4 * C)
    return f


def brute_force_svm(Q, loss, C):
    """Exact optimum of the box QP by enumerating active sets."""
    m = Q.shape[0]
    Qe = Q + (np.eye(m) / (2 * C) if loss == 2 else 0)
    states = (0, 1, 2) if loss == 1 else (0, 2)  # 0: at zero, 1: at C, 2: free
    best, best_a = np.inf, None
    for pat in itertools.product(states, repeat=m):
        pat = np.array(pat)
        F, U = pat == 2, pat == 1
        a = np.zeros(m)
        a[U] = C
        if F.any():
            rhs = 1.0 - Qe[np.ix_(F, U)] @ a[U]
            try:
                a[F] = np.linalg.solve(Qe[np.ix_(F, F)], rhs)
            except np.linalg.LinAlgError:
                continue
            if np.any(a[F] < -1e-12) or (loss == 1 and np.any(a[F] > C + 1e-12)):
                continue
        f = 0.5 * a @ Qe @ a - a.sum()
        if f < best:
            best, best_a = f, a
    return best, best_a


# ---------------------------------------------------------- Algorithm 1 ---
@pytest.mark.parametrize("loss", [1, 2])
def test_dcd_single_step_is_exact_1d_minimiser(loss):
    p = inputs.blobs(m=25, n=4, seed=5)
    A, y = p.A, p.y
    C = 0.7
    kw = dict(gamma=0.3)
    k = oracle.kernel("rbf", **kw)
    _, Q = full_Q(A, y, "rbf", **kw)
    g = np.random.default_rng(3)
    for trial in range(6):
        a0 = g.uniform(0, C, size=25)
        first = 100 + trial
        i = int(oracle.sample_dcd(9, 25, first, 1)[0])
        a1 = oracle.dcd_svm(A, y, k, loss, C, H=1, seed=9, first=first, alpha0=a0)
        assert np.all(np.delete(a1 - a0, i) == 0)
        hi = C - a0[i] if loss == 1 else 50.0

        def f(t):
            a = a0.copy()
            a[i] += t
            return svm_dual_min(Q, a, loss, C)

        r = optimize.minimize_scalar(f, bounds=(-a0[i], hi), method="bounded",
                                     options={"xatol": 1e-12, "maxiter": 500})
        assert abs((a1[i] - a0[i]) - r.x) < 1e-6
        assert f(a1[i] - a0[i]) <= r.fun + 1e-12


@pytest.mark.parametrize("loss,kind,kw", [
    (1, "rbf", dict(gamma=0.5)),
    (2, "rbf", dict(gamma=0.5)),
    (1, "poly", dict(coef0=1.0, degree=2)),
])
def test_dcd_converges_to_brute_force_optimum(loss, kind, kw):
    p = inputs.blobs(m=7, n=3, seed=2)
    A, y = p.A, p.y
    C = 0.9
    _, Q = full_Q(A, y, kind, **kw)
    best, best_a = brute_force_svm(Q, loss, C)
    k = oracle.kernel(kind, **kw)
    a = oracle.dcd_svm(A, y, k, loss, C, H=6000, seed=1)
    assert svm_dual_min(Q, a, loss, C) - best < 1e-10
    assert np.max(np.abs(a - best_a)) < 1e-6
    ob = oracle.svm_objectives(A, y, k, loss, C, a)
    assert abs(ob["gap"]) < 1e-8 * max(1.0, abs(ob["primal"]))
    assert ob["kkt"] < 1e-6


@pytest.mark.parametrize("loss", [1, 2])
def test_duality_gap_and_kkt_vanish(loss):
    p = inputs.blobs(m=60, n=5, seed=4)
    k = oracle.kernel("rbf", gamma=0.2)
    a = oracle.dcd_svm(p.A, p.y, k, loss, 1.0, H=40000, seed=3)
    ob = oracle.svm_objectives(p.A, p.y, k, loss, 1.0, a)
    assert ob["gap"] >= -1e-9
    assert ob["gap"] < 1e-8 * abs(ob["primal"])
    # the gap was large at the start
    ob0 = oracle.svm_objectives(p.A, p.y, k, loss, 1.0, np.zeros(60))
    assert ob0["gap"] > 1.0


# ---------------------------------------------------------- Algorithm 2 ---
@pytest.mark.parametrize("loss,kind,kw", [
    (1, "rbf", dict(gamma=0.4)),
    (2, "poly", dict(coef0=1.0, degree=3)),
    (1, "linear", {}),
])
@pytest.mark.parametrize("s", [1, 2, 3, 8, 16])
def test_sstep_dcd_equals_dcd(loss, kind, kw, s):
    """Section 3.2: s-step DCD computes the same iterates as DCD."""
    p = inputs.blobs(m=9, n=4, seed=6)  # m = 9 makes repeated indices within an s-block common
    k = oracle.kernel(kind, **kw)
    H = 203
    a1 = oracle.dcd_svm(p.A, p.y, k, loss, 0.8, H, seed=5, first=7)
    a2 = oracle.sstep_dcd_svm(p.A, p.y, k, loss, 0.8, s, H, seed=5, first=7)
    assert rel(a2, a1) < 1e-12


def test_sstep_dcd_block_has_duplicates():
    idx = oracle.sample_dcd(5, 9, 7, 16)
    assert len(set(idx)) < 16


# ---------------------------------------------------------- Algorithm 3 ---
def krr_closed(A, y, gamma, lam):
    K = np.exp(-gamma * cdist(A, A, "sqeuclidean"))
    m = A.shape[0]
    return np.linalg.solve(K / lam + m * np.eye(m), y), K


def test_bdcd_converges_to_dense_solve():
    p = inputs.krr_dense(m=48, n=6, seed=1, dtype=np.float64)
    lam = 0.05
    want, _ = krr_closed(p.A, p.y, 0.5, lam)
    k = oracle.kernel("rbf", gamma=0.5)
    a = oracle.bdcd_krr(p.A, p.y, k, lam, b=8, H=3000, seed=2)
    assert rel(a, want) < 1e-8
    assert rel(oracle.krr_closed_form(p.A, p.y, k, lam), want) < 1e-12


def test_bdcd_full_block_is_exact_in_one_step():
    p = inputs.krr_dense(m=20, n=3, seed=3, dtype=np.float64)
    want, _ = krr_closed(p.A, p.y, 1.3, 0.2)
    a = oracle.bdcd_krr(p.A, p.y, oracle.kernel("rbf", gamma=1.3), 0.2, b=20, H=1, seed=0)
    assert rel(a, want) < 1e-12


def test_bdcd_identity_kernel_closed_form():
    p = inputs.krr_dense(m=30, n=4, seed=4, dtype=np.float64)
    lam = 0.3
    blocks = oracle.sample_bdcd(8, 30, 5, 0, 200)
    assert len(set(blocks.ravel())) == 30
    a = oracle.bdcd_krr(p.A * 100, p.y, oracle.kernel("rbf", gamma=1e6), lam, b=5, H=200, seed=8)
    assert rel(a, p.y / (1 / lam + 30)) < 1e-14


def test_krr_textbook_mapping():
    """alpha_paper = lam (K + m lam I)^-1 y (the textbook kernel-ridge form)."""
    p = inputs.krr_dense(m=25, n=3, seed=5, dtype=np.float64)
    lam = 0.01
    K = np.exp(-0.5 * cdist(p.A, p.A, "sqeuclidean"))
    tb = lam * np.linalg.solve(K + 25 * lam * np.eye(25), p.y)
    assert rel(oracle.krr_closed_form(p.A, p.y, oracle.kernel("rbf", gamma=0.5), lam), tb) < 1e-12


# ---------------------------------------------------------- Algorithm 4 ---
@pytest.mark.parametrize("kind,kw", [("rbf", dict(gamma=0.7)), ("poly", dict(coef0=0.5, degree=2)),
                                     ("linear", {})])
@pytest.mark.parametrize("s", [1, 2, 5, 16])
def test_sstep_bdcd_equals_bdcd(kind, kw, s):
    """Section 3.4: s-step BDCD computes the same iterates as BDCD; m = 12
    with b = 4 makes blocks of one outer step overlap (the V^T V term)."""
    p = inputs.krr_dense(m=12, n=3, seed=6, dtype=np.float64)
    k = oracle.kernel(kind, **kw)
    H = 37
    a1 = oracle.bdcd_krr(p.A, p.y, k, 0.1, 4, H, seed=4, first_block=3)
    a2 = oracle.sstep_bdcd_krr(p.A, p.y, k, 0.1, 4, s, H, seed=4, first_block=3)
    assert rel(a2, a1) < 1e-12


def test_sstep_bdcd_converges_like_bdcd():
    p = inputs.krr_dense(m=64, n=5, seed=7, dtype=np.float64)
    want, _ = krr_closed(p.A, p.y, 0.5, 0.02)
    a = oracle.sstep_bdcd_krr(p.A, p.y, oracle.kernel("rbf", gamma=0.5), 0.02, 8, 16, 4000, seed=1)
    assert rel(a, want) < 1e-8


# ---------------------------------------------- objectives / gradients ----
@pytest.mark.parametrize("loss", [1, 2])
def test_svm_objectives_linear_kernel_primal(loss):
    p = inputs.blobs(m=30, n=6, seed=8)
    C = 0.6
    a = np.random.default_rng(5).uniform(0, C, size=30)
    w = p.A.T @ (p.y * a)
    margin = p.y * (p.A @ w)
    xi = np.maximum(0.0, 1.0 - margin)
    P = 0.5 * w @ w + C * np.sum(xi if loss == 1 else xi ** 2)
    D = a.sum() - 0.5 * w @ w - (a @ a / (4 * C) if loss == 2 else 0.0)
    ob = oracle.svm_objectives(p.A, p.y, oracle.kernel("linear"), loss, C, a)
    assert abs(ob["primal"] - P) < 1e-11 * abs(P)
    assert abs(ob["dual"] - D) < 1e-11 * abs(D)
    omega = 0.0 if loss == 1 else 1 / (2 * C)
    g = oracle.svm_gradient(p.A, p.y, oracle.kernel("linear"), loss, C, a)
    assert rel(g, margin - 1 + omega * a) < 1e-13


def test_krr_gradient_and_objective():
    p = inputs.krr_dense(m=40, n=4, seed=9, dtype=np.float64)
    lam = 0.07
    K = np.exp(-0.9 * cdist(p.A, p.A, "sqeuclidean"))
    a = np.random.default_rng(6).standard_normal(40)
    M = K / lam + 40 * np.eye(40)
    k = oracle.kernel("rbf", gamma=0.9)
    assert rel(oracle.krr_gradient(p.A, p.y, k, lam, a), M @ a - p.y) < 1e-13
    f = 0.5 * a @ M @ a - p.y @ a
    assert abs(oracle.krr_objective(p.A, p.y, k, lam, a) - f) < 1e-12 * abs(f)


def test_thread_count_does_not_change_any_result():
    """The parallel row loops write separate outputs, each formed as with one
    thread: every routine gives the same bits at 1 and at 4 threads."""
    p = inputs.krr_dense(m=90, n=7, seed=12, dtype=np.float64)
    q = inputs.blobs(m=80, n=5, seed=13)
    k = oracle.kernel("rbf", gamma=0.6)
    a = np.random.default_rng(7).standard_normal(90)
    res = []
    for t in (1, 4):
        oracle.set_threads(t)
        res.append([oracle.sstep_bdcd_krr(p.A, p.y, k, 0.05, 4, 8, 60, seed=2),
                    oracle.bdcd_krr(p.A, p.y, k, 0.05, 4, 20, seed=2),
                    oracle.sstep_dcd_svm(q.A, q.y, k, 1, 1.0, 8, 300, seed=3),
                    oracle.dcd_svm(q.A, q.y, k, 2, 1.0, 100, seed=3),
                    oracle.kernel_block(k, p.A, np.arange(30)),
                    oracle.krr_gradient(p.A, p.y, k, 0.05, a),
                    np.array([oracle.krr_objective(p.A, p.y, k, 0.05, a)]),
                    oracle.svm_gradient(q.A, q.y, k, 2, 1.0, np.abs(a[:80])),
                    oracle.krr_closed_form(p.A, p.y, k, 0.05)])
    oracle.set_threads(os.cpu_count() or 1)
    for x1, x4 in zip(*res):
        assert np.array_equal(x1, x4)


# ------------------------------------------------- FP8 e4m3 row storage ---
def test_e4m3_values_of_the_format():
    v = oracle.e4m3_value(np.arange(256, dtype=np.uint8))
    assert v[0x7E] == 448.0 and v[0x01] == 2.0 ** -9 and v[0x08] == 2.0 ** -6 and v[0x38] == 1.0
    assert v[0x07] == 7 * 2.0 ** -9 and v[0x0F] == 1.875 * 2.0 ** -6  # largest subnormal / normal of binade -6
    assert np.isnan(v[0x7F]) and np.isnan(v[0xFF]) and np.all(v[0x80:0xFF] == -v[0:0x7F])
    finite = v[:0x7F]
    assert np.all(np.diff(finite) > 0)  # codes 0..0x7e are increasing magnitudes
    c = np.arange(256, dtype=np.uint8)[~np.isnan(v)]
    assert np.array_equal(oracle.e4m3_encode(oracle.e4m3_value(c)), c)


def test_e4m3_rounding_special_cases():
    x = np.array([17.0, 19.0, 2.0 ** -10, 3 * 2.0 ** -10, 464.0, 1e30, -1e30, -2.0 ** -11, 0.0, 240.0 + 8.0])
    want = [16.0, 20.0, 0.0, 2 * 2.0 ** -9, 448.0, 448.0, -448.0, -0.0, 0.0, 256.0]
    got = oracle.e4m3_value(oracle.e4m3_encode(x))
    assert np.array_equal(got, want) and np.signbit(got[7])


def test_e4m3_encode_matches_torch_float8():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    g = np.random.default_rng(0)
    v = oracle.e4m3_value(np.arange(127, dtype=np.uint8))
    x = np.concatenate([g.uniform(-448, 448, 20000), g.uniform(-0.03, 0.03, 20000), g.standard_normal(20000),
                        (v[1:126] + v[2:127]) / 2, -(v[1:126] + v[:125]) / 2]).astype(np.float32)
    t = torch.from_numpy(x).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(t, oracle.e4m3_encode(x.astype(np.float64)))


def test_quantize_rows_scale_range_and_error_bound():
    g = np.random.default_rng(1)
    A = g.standard_normal((64, 45)) * np.exp(g.uniform(-8, 8, (64, 1)))
    A[5] = 0.0
    A[9, :] = 0.0
    A[9, 3] = -2.5
    q, s = oracle.quantize_e4m3_rows(A)
    assert q.dtype == np.uint8 and s.dtype == np.float32
    A32 = A.astype(np.float32).astype(np.float64)
    amax = np.max(np.abs(A32), axis=1)
    from fractions import Fraction
    for si, ai in zip(s, amax):  # s_i is amax_i / 448 correctly rounded to FP32
        half_ulp = Fraction(float(np.spacing(si))) / 2
        assert abs(Fraction(float(si)) - Fraction(float(ai)) / 448) <= half_ulp
    assert s[5] == 0 and np.all(q[5] == 0)
    qv = oracle.e4m3_value(q)
    nz = amax > 0
    assert np.all(np.max(np.abs(qv[nz]), axis=1) == 448.0)  # each row's largest entry maps to +-448
    assert q[9, 3] == 0xFE and np.all(q[9, np.arange(45) != 3] == 0)
    D = oracle.dequantize_e4m3_rows(q, s)
    x = np.abs(A32 / np.where(s > 0, s, 1)[:, None])
    # half a unit in the last place: 2^-4 relative for normals, 2^-10 absolute (in units of s) below 2^-6
    bound = np.where(x >= 2.0 ** -6, 2.0 ** -4 * np.abs(A32), 2.0 ** -10 * s[:, None].astype(np.float64))
    assert np.all(np.abs(D - A32) <= bound * (1 + 1e-6))
