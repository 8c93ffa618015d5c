"""The CSR kernel block applied through the transposed (CSC) copy of A: only
the nonzeros in columns some sampled row holds are visited, sorted back into
each row's element order, so the result must equal the full pass over every
nonzero bit for bit; and, at the K-SVM sparse configuration's full shape,
the oracle's kernel values on a sample of rows."""
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


def lib_csr(p, dtype):
    return B().Csr(dev(p.row_ptr), dev(p.col_idx), dev(p.values.astype(dtype)), p.n)


def on_stream(fn, *args, **kw):
    """Runs a solve on a stream of its own (steps are then replayed from a
    CUDA graph, whose kernel count the stats report)."""
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        out = fn(*args, stream=st.cuda_stream, **kw)
    torch.cuda.synchronize()
    return out


def with_dense_rows(p, rows, k, seed):
    """p with rows `rows` replaced by k distinct random columns each (values
    U(0,1), unit norm): a tile of such rows collects more incidences than the
    apply sorts in shared memory and takes the full pass."""
    g = np.random.default_rng(seed)
    rp, ci, va = [0], [], []
    rows = set(int(r) for r in rows)
    for i in range(p.m):
        a, b = p.row_ptr[i], p.row_ptr[i + 1]
        if i in rows:
            c = np.sort(g.choice(p.n, size=k, replace=False)).astype(np.int32)
            v = g.random(k).astype(np.float32)
            v /= np.linalg.norm(v)
        else:
            c, v = p.col_idx[a:b], p.values[a:b]
        ci.append(c)
        va.append(v)
        rp.append(rp[-1] + len(c))
    return inputs.CsrProblem(np.array(rp, np.int64), np.concatenate(ci).astype(np.int32),
                             np.concatenate(va).astype(np.float32), p.n, p.y)


KERNELS = [("poly", dict(coef0=1.0, degree=3)), ("rbf", dict(gamma=0.7)), ("linear", {})]


@pytest.fixture(scope="module")
def sparse():
    # 40000 rows of 20 nonzeros in 50000 columns: a sampled row's columns reach
    # ~320 rows, so the transposed apply is chosen
    return inputs.sparse_csr(m=40000, n=50000, nnz_per_row=20, seed=3)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_svm_solve_through_csc_equals_full_pass_bit_for_bit(sparse, prec, kind, kw):
    p = sparse
    A = lib_csr(p, np.float64 if prec == "fp64" else np.float32)
    kb = B().kernel(kind, **kw)
    res = {}
    for name, flags in (("csc", 0), ("full", B().FLAG_CSR_FULL_PASS)):
        al, gr, st, _ = on_stream(B().svm_solve, A, dev(p.y), kb, 2, 0.5, 32, 32 * 12, seed=5, prec=prec,
                                  flags=flags)
        res[name] = (al.cpu().numpy(), gr.cpu().numpy(), st["gpu_launches_per_step"])
    assert np.array_equal(res["csc"][0], res["full"][0])
    assert np.array_equal(res["csc"][1], res["full"][1])
    assert res["csc"][2] == res["full"][2] + 1  # the scatter beside the apply: the transposed path ran


@pytest.mark.parametrize("prec", ["fp64", "bf16x3"])
def test_krr_solve_through_csc_equals_full_pass_over_several_column_chunks(sparse, prec):
    p = sparse
    A = lib_csr(p, np.float64 if prec == "fp64" else np.float32)
    y = np.random.default_rng(1).standard_normal(p.m)
    kb = B().kernel("rbf", gamma=0.5)
    res = {}
    for name, flags in (("csc", 0), ("full", B().FLAG_CSR_FULL_PASS)):
        # s * b = 72 sampled rows per step: three column chunks of at most 32
        al, gr, st, _ = on_stream(B().krr_solve, A, dev(y), kb, 1e-3, 8, 9, 9 * 6, seed=2, prec=prec, flags=flags)
        res[name] = (al.cpu().numpy(), gr.cpu().numpy(), st["gpu_launches_per_step"])
    assert np.array_equal(res["csc"][0], res["full"][0])
    assert np.array_equal(res["csc"][1], res["full"][1])
    assert res["csc"][2] == res["full"][2] + 3


@pytest.mark.parametrize("prec,flags", [("fp64", 0), ("bf16x3", 0), ("bf16x3", "full")])
def test_svm_lookahead_on_csr_matches_one_stream_steps(sparse, prec, flags):
    """The K-SVM look-ahead on CSR data with in-order steps (the next step's
    column map, pair table and Gram in the other buffer set on a second
    stream, this step's scatter beside its recurrence) gives the one-stream
    steps' iterates bit for bit, with gap checks, recomputations and a short
    last step; through the transposed copy and with the full pass.  The
    default deferred step (the recurrence one step ahead, beside the block)
    gives them up to the association of the sums: 1e-10 relative in FP64,
    1e-5 with the FP32 block (its s x s cross product rounds each kernel value
    in FP32 as the block does, its sum over the step runs in FP64)."""
    p = sparse
    A = lib_csr(p, np.float64 if prec == "fp64" else np.float32)
    kb = B().kernel("poly", coef0=1.0, degree=3)
    f = B().FLAG_CSR_FULL_PASS if flags == "full" else 0
    side = torch.cuda.Stream()
    res = []
    with torch.cuda.stream(side):
        for extra in (B().FLAG_NO_GRAPH, B().FLAG_NO_DEFER, 0):
            al, gr, st, _ = B().svm_solve(A, dev(p.y), kb, 2, 0.5, 32, 32 * 11 + 7, seed=9, prec=prec, tol=1e-3,
                                          check_every=3, flags=f | extra | B().FLAG_REFRESH,
                                          stream=side.cuda_stream)
            res.append((al.cpu().numpy(), gr.cpu().numpy(), st))
        side.synchronize()
    assert res[0][2]["iters_done"] == res[1][2]["iters_done"] == res[2][2]["iters_done"]
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[2][2]["gpu_launches_per_step"] == res[1][2]["gpu_launches_per_step"] + 3
    tol = 1e-10 if prec == "fp64" else 1e-5
    a0, a2 = res[0][0], res[2][0]
    assert np.linalg.norm(a2 - a0) <= tol * np.linalg.norm(a0)
    assert np.max(np.abs(res[2][1] - res[0][1])) <= tol * max(1.0, np.max(np.abs(res[0][1])))


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 1e-5)])
def test_svm_deferred_step_on_csr_matches_oracle(prec, tol):
    """The deferred K-SVM step on CSR data (squared hinge, s = 32, through the
    transposed copy) against the oracle's DCD on the same index sequence,
    dense rows of the matrix (m = 3000: rows recur within and across steps)."""
    p = inputs.sparse_csr(m=3000, n=2000, nnz_per_row=12, seed=6)
    A = lib_csr(p, np.float64 if prec == "fp64" else np.float32)
    kb, ko = B().kernel("poly", coef0=1.0, degree=3), oracle.kernel("poly", coef0=1.0, degree=3)
    side = torch.cuda.Stream()
    H = 32 * 20 + 11
    with torch.cuda.stream(side):
        al, _, st, rc = B().svm_solve(A, dev(p.y), kb, 2, 0.5, 32, H, seed=4, prec=prec, stream=side.cuda_stream)
        side.synchronize()
    assert rc == B().OK and st["iters_done"] == H
    want = oracle.dcd_svm(p.to_dense(), p.y, ko, 2, 0.5, H, seed=4)  # float32 values, exact in FP64
    got = al.cpu().numpy()
    assert np.linalg.norm(got - want) <= tol * np.linalg.norm(want)


def test_krr_lookahead_on_csr_matches_one_stream_steps(sparse):
    """K-RR BDCD on CSR data with the look-ahead (the next step's column map,
    pair table and Gram beside this step): the one-stream steps' bits."""
    p = sparse
    A = lib_csr(p, np.float32)
    y = np.random.default_rng(4).standard_normal(p.m)
    kb = B().kernel("rbf", gamma=0.5)
    side = torch.cuda.Stream()
    res = []
    with torch.cuda.stream(side):
        for extra in (B().FLAG_NO_GRAPH, 0):
            al, gr, st, _ = B().krr_solve(A, dev(y), kb, 1e-3, 8, 9, 9 * 7 + 2, seed=2, prec="bf16x3",
                                          flags=extra, stream=side.cuda_stream)
            res.append((al.cpu().numpy(), gr.cpu().numpy(), st))
        side.synchronize()
    assert res[0][2]["iters_done"] == res[1][2]["iters_done"]
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])


def test_tiles_beyond_the_shared_buffer_take_the_full_pass(sparse):
    # 64 rows of 3000 nonzeros (two whole 32-row tiles and parts of two more)
    p = with_dense_rows(sparse, range(1000, 1064), 3000, seed=8)
    A = lib_csr(p, np.float32)
    kb = B().kernel("poly", coef0=1.0, degree=3)
    res = {}
    for name, flags in (("csc", 0), ("full", B().FLAG_CSR_FULL_PASS)):
        al, gr, st, _ = on_stream(B().svm_solve, A, dev(p.y), kb, 2, 0.5, 32, 32 * 8, seed=6, prec="bf16x3",
                                  flags=flags)
        res[name] = (al.cpu().numpy(), gr.cpu().numpy(), st["gpu_launches_per_step"])
    assert res["csc"][2] == res["full"][2] + 1
    assert np.array_equal(res["csc"][0], res["full"][0]) and np.array_equal(res["csc"][1], res["full"][1])


def test_dense_columns_keep_the_full_pass():
    # 2000 rows of 40 nonzeros in 400 columns: a sampled row reaches most rows,
    # so the transposed copy would read more than the full pass and is not used
    p = inputs.sparse_csr(m=2000, n=400, nnz_per_row=40, seed=4)
    A = lib_csr(p, np.float32)
    kb = B().kernel("poly", coef0=1.0, degree=3)
    _, _, st0, _ = on_stream(B().svm_solve, A, dev(p.y), kb, 2, 0.5, 16, 64, seed=1, prec="bf16x3")
    _, _, st1, _ = on_stream(B().svm_solve, A, dev(p.y), kb, 2, 0.5, 16, 64, seed=1, prec="bf16x3",
                             flags=B().FLAG_CSR_FULL_PASS)
    assert st0["gpu_launches_per_step"] == st1["gpu_launches_per_step"]


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("bf16x3", 3e-6)])
def test_apply_at_full_sparse_shape_matches_oracle_on_sampled_rows(prec, tol):
    """dcd_kernel_block_apply on the 200000 x 50000 CSR matrix (50 nonzeros per
    row, polynomial (a.b + 1)^3, 32 sampled columns: the transposed apply),
    checked row by row against the oracle on 96 random rows and the 32
    sampled rows themselves."""
    p = inputs.sparse_csr(m=200000, n=50000, nnz_per_row=50, seed=0)
    g = np.random.default_rng(12)
    cols = g.integers(0, p.m, size=32)
    w = g.standard_normal(32)
    rs = p.y
    g0 = g.standard_normal(p.m)
    kb, ko = B().kernel("poly", coef0=1.0, degree=3), oracle.kernel("poly", coef0=1.0, degree=3)
    gd = dev(g0)
    B().kernel_block_apply(lib_csr(p, np.float64 if prec == "fp64" else np.float32), kb, prec,
                           dev(cols, torch.int32), dev(w), gd, rowscale=dev(rs))
    got = gd.cpu().numpy()
    check = np.concatenate([g.integers(0, p.m, size=96), cols])

    def dense(rows):
        out = np.zeros((len(rows), p.n))
        for t, r in enumerate(rows):
            a, b = p.row_ptr[r], p.row_ptr[r + 1]
            out[t, p.col_idx[a:b]] = p.values[a:b]  # float32 values, exact in FP64
        return out

    both = np.vstack([dense(check), dense(cols)])
    Kb = oracle.kernel_block(ko, both, np.arange(len(check), len(check) + len(cols)),
                             rows=np.arange(len(check)))
    want = g0[check] + rs[check] * (Kb @ w)
    scale = np.max(np.abs(Kb)) * np.sum(np.abs(w))
    assert np.max(np.abs(got[check] - want)) <= tol * scale
