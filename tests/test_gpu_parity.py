"""CUDA path (through the C ABI) against the FP64 oracle, element by element.

Sizes span several row tiles (64-row FP64 tiles, 128-row tensor-core tiles)
with ragged tails in rows, features (k-blocks of 64 / 32) and sampled
columns (32-column epilogue groups).

Tolerances:
  FP64 form          iterates within 1e-10 relative 2-norm (the FP64 target);
                     kernel entries within 1e-12 relative.
  mixed (bf16/tf32)  kernel entries against the oracle evaluated on the same
                     rounded inputs: FP32 accumulation over n <= 128 products
                     plus ex2.approx give |err| <= 3e-5 * max|K|; iterates:
                     final dual objective within 1e-6 relative and alpha within
                     1e-4 relative 2-norm of the FP64 oracle on the same index
                     stream (the mixed-precision target).
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


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def round_bf16(A):
    return inputs.bf16_bits_to_f32(inputs.to_bf16_bits(A.astype(np.float32))).astype(np.float64)


def round_split(A):
    """hi + lo of the split-bf16 operand (hi = bf16(a), lo = bf16(a - hi))."""
    a = np.ascontiguousarray(A, dtype=np.float32)
    hi = inputs.bf16_bits_to_f32(inputs.to_bf16_bits(a))
    lo = inputs.bf16_bits_to_f32(inputs.to_bf16_bits((a - hi).astype(np.float32)))
    return hi.astype(np.float64) + lo.astype(np.float64)


def round_fp16(A):
    """The fp16 operand: the FP32 values scaled by 2^(e - 15), with the
    matrix's largest magnitude in [2^(e-1), 2^e), rounded to fp16 (nearest
    even) and scaled back."""
    a = np.ascontiguousarray(A, dtype=np.float32).astype(np.float64)
    mx = np.max(np.abs(a))
    e = max(int(np.frexp(mx)[1]) if mx > 0 else 0, -110)
    sc = np.ldexp(1.0, e - 15)
    return (a / sc).astype(np.float16).astype(np.float64) * sc


ROUND = {"bf16": round_bf16, "bf16x3": round_split, "fp16": round_fp16}


def round_tf32(A):
    u = np.ascontiguousarray(A, dtype=np.float32).view(np.uint32).astype(np.uint64)
    # nearest, ties away from zero, to 10 explicit mantissa bits
    r = ((u + 0x1000) & 0xFFFFE000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def round_split_tf32(A):
    """hi + lo of the split-tf32 operand (hi = tf32(a), lo = tf32(a - hi))."""
    a = np.ascontiguousarray(A, dtype=np.float32)
    hi = round_tf32(a)
    lo = round_tf32((a.astype(np.float64) - hi).astype(np.float32))
    return hi + lo


ROUND["tf32x3"] = round_split_tf32
# max |K - K_ref| / max |K_ref| against the FP64 kernel of the rounded operand;
# split tf32 is bounded by the FP32 epilogue (expanded distance, exp2), about
# 3.5e-6 measured on GB300, rather than by its operands
TC_TOL = {"bf16": 3e-5, "tf32": 3e-5, "bf16x3": 3e-5, "tf32x3": 1e-5, "fp16": 3e-5}

KERNELS = [("rbf", dict(gamma=0.35)), ("poly", dict(coef0=1.0, degree=3)), ("linear", {})]


# ------------------------------------------------------------ sampling ----
@pytest.mark.parametrize("m,first,count", [(1, 0, 5), (97, 0, 1000), (50000, 123456789, 4096)])
def test_dcd_sampler_bit_exact(m, first, count):
    got = B().sample_indices(0, 42, m, 1, first, count).cpu().numpy()
    assert np.array_equal(got, oracle.sample_dcd(42, m, first, count))


@pytest.mark.parametrize("m,b,first,nblk", [(16, 16, 0, 3), (100, 7, 5, 40), (50000, 16, 2**40, 64),
                                            (400, 128, 9, 8)])
def test_bdcd_sampler_bit_exact(m, b, first, nblk):
    got = B().sample_indices(1, 7, m, b, first, nblk).cpu().numpy().reshape(nblk, b)
    assert np.array_equal(got, oracle.sample_bdcd(7, m, b, first, nblk))


# ------------------------------------------------------- kernel blocks ----
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_kernel_block_fp64(kind, kw):
    g = np.random.default_rng(1)
    A = g.standard_normal((300, 37)) * 0.3
    cols = g.integers(0, 300, size=70)
    rows = g.integers(0, 300, size=133)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    got = B().kernel_block(dev(A), kb, "fp64", dev(cols, torch.int32), rows=dev(rows, torch.int32)).cpu().numpy()
    want = oracle.kernel_block(ko, A, cols, rows=rows)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3", "tf32x3", "fp16"])
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_kernel_block_tensor_core(prec, kind, kw):
    g = np.random.default_rng(2)
    A = (g.standard_normal((300, 77)) * 0.2).astype(np.float32)
    cols = g.integers(0, 300, size=70)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    got = B().kernel_block(dev(A), kb, prec, dev(cols, torch.int32)).cpu().numpy()
    Ar = ROUND.get(prec, round_tf32)(A)
    want = oracle.kernel_block(ko, Ar, cols)
    err = np.max(np.abs(got - want))
    assert err <= TC_TOL[prec] * np.max(np.abs(want)), err
    if prec == "tf32x3":  # ~22 significant bits: close to the unrounded FP64 kernel too
        exact = oracle.kernel_block(ko, A.astype(np.float64), cols)
        assert np.max(np.abs(got - exact)) <= 1e-5 * np.max(np.abs(exact))


@pytest.mark.parametrize("prec", ["fp64", "bf16", "tf32", "bf16x3", "tf32x3", "fp16"])
@pytest.mark.parametrize("kind,kw", KERNELS)
def test_kernel_block_apply(prec, kind, kw):
    """g += rs * K(A, A_cols) w for every row, block never stored."""
    g = np.random.default_rng(3)
    m, n = 333, 45
    A = g.standard_normal((m, n)) * 0.25
    cols = g.integers(0, m, size=45)
    w = g.standard_normal(45)
    rs = np.where(g.random(m) < 0.5, -1.0, 1.0)
    g0 = g.standard_normal(m)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    gd = dev(g0)
    B().kernel_block_apply(dev(A if prec == "fp64" else A.astype(np.float32)), kb, prec, dev(cols, torch.int32),
                           dev(w), gd, rowscale=dev(rs))
    Ar = A if prec == "fp64" else ROUND.get(prec, round_tf32)(A)
    want = g0 + rs * (oracle.kernel_block(ko, Ar, cols) @ w)
    got = gd.cpu().numpy()
    scale = np.max(np.abs(oracle.kernel_block(ko, Ar, cols))) * np.sum(np.abs(w))
    tol = 1e-12 if prec == "fp64" else TC_TOL[prec]
    assert np.max(np.abs(got - want)) <= tol * scale


@pytest.mark.parametrize("prec", ["bf16", "tf32", "bf16x3", "tf32x3", "fp8", "fp16"])
@pytest.mark.parametrize("m,ncols,n", [(1100, 600, 300), (257, 33, 16), (3000, 1024, 64), (129, 300, 200)])
def test_kernel_block_apply_pair_tiles(prec, m, ncols, n):
    """The apply form runs on CTA pairs over 256-row tiles: ragged pair tiles
    (a pair whose second CTA has no rows), several N-chunks with a ragged last
    one, odd halves of an N-chunk, k-blocks with a ragged tail."""
    g = np.random.default_rng(m + ncols)
    A = g.standard_normal((m, n)) / np.sqrt(n)
    cols = g.integers(0, m, size=ncols)
    w = g.standard_normal(ncols)
    g0 = g.standard_normal(m)
    kb, ko = B().kernel("rbf", gamma=0.7), oracle.kernel("rbf", gamma=0.7)
    gd = dev(g0)
    if prec == "fp8":
        q, sc = oracle.quantize_e4m3_rows(A)
        Ar = oracle.dequantize_e4m3_rows(q, sc)
        Ad, tol = B().Fp8(dev(q), dev(sc)), 2e-5
    else:
        Ar = ROUND.get(prec, round_tf32)(A)
        Ad, tol = dev(A.astype(np.float32)), TC_TOL[prec]
    B().kernel_block_apply(Ad, kb, prec, dev(cols, torch.int32), dev(w), gd)
    Kb = oracle.kernel_block(ko, Ar, cols)
    want = g0 + Kb @ w
    assert np.max(np.abs(gd.cpu().numpy() - want)) <= tol * np.max(np.abs(Kb)) * np.sum(np.abs(w))


@pytest.mark.parametrize("prec", ["bf16x3", "fp8", "tf32"])
@pytest.mark.parametrize("m,ncols,n", [(40000, 1000, 64), (20001, 300, 96), (50000, 1024, 512)])
def test_kernel_block_apply_shared_tiles(prec, m, ncols, n):
    """More 256-row tiles than CTA pairs: the pairs split the (tile, N-chunk)
    units into equal ranges, so some tiles are shared by two pairs.  Parity
    with the oracle on every row, and each shared tile's rows bit-identical
    to the same rows computed as the only tile of a small apply."""
    g = np.random.default_rng(m + 7 * ncols)
    A = g.standard_normal((m, n)) / np.sqrt(n)
    cols = g.integers(0, m, size=ncols)
    w = g.standard_normal(ncols)
    g0 = g.standard_normal(m)
    kb, ko = B().kernel("rbf", gamma=0.7), oracle.kernel("rbf", gamma=0.7)

    def run(Ah, c, gi):
        gd = dev(gi)
        if prec == "fp8":
            q, sc = oracle.quantize_e4m3_rows(Ah)
            Ad = B().Fp8(dev(q), dev(sc))
        else:
            Ad = dev(Ah.astype(np.float32))
        B().kernel_block_apply(Ad, kb, prec, dev(c, torch.int32), dev(w), gd)
        return gd.cpu().numpy()

    got = run(A, cols, g0)
    if prec == "fp8":
        q, sc = oracle.quantize_e4m3_rows(A)
        Ar, tol = oracle.dequantize_e4m3_rows(q, sc), 2e-5
    else:
        Ar, tol = ROUND.get(prec, round_tf32)(A), TC_TOL[prec]
    Kb = oracle.kernel_block(ko, Ar, cols)
    want = g0 + Kb @ w
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(Kb)) * np.sum(np.abs(w))
    # the tiles holding a boundary between two pairs' unit ranges
    tiles, nch = (m + 255) // 256, (ncols + 255) // 256 if ncols > 256 else 1
    pairs = min(tiles, torch.cuda.get_device_properties(0).multi_processor_count // 2)
    U = tiles * nch
    shared = sorted({(p * U // pairs) // nch for p in range(1, pairs) if (p * U // pairs) % nch})
    assert shared
    for t in shared[:3]:
        r0, r1 = 256 * t, min(256 * t + 256, m)
        A2 = np.concatenate([A[r0:r1], A[cols]])
        # a column that is one of the tile's own rows names that row again (the RBF takes d^2 = 0
        # on a row's own sample), the others their copies past the tile
        c2 = np.where((cols >= r0) & (cols < r1), cols - r0, (r1 - r0) + np.arange(ncols))
        g2 = np.concatenate([g0[r0:r1], np.zeros(ncols)])
        got2 = run(A2, c2, g2)
        assert np.array_equal(got2[: r1 - r0], got[r0:r1]), t


def test_kernel_block_bad_index_is_an_error_not_a_fault():
    A = dev(np.ones((10, 4)))
    with pytest.raises(B().DcdError) as e:
        B().kernel_block(A, B().kernel("linear"), "fp64", dev(np.array([1, 10]), torch.int32))
    assert e.value.status == B().EINVAL
    with pytest.raises(B().DcdError):
        B().kernel_block(A.float(), B().kernel("linear"), "bf16", dev(np.array([-1, 2]), torch.int32))


# ---------------------------------------------------- FP64 form solves ----
SVM_CASES = [
    (1, "rbf", dict(gamma=0.4), 1, 1.0),
    (1, "rbf", dict(gamma=0.4), 8, 1.0),
    (2, "poly", dict(coef0=1.0, degree=3), 5, 0.5),
    (1, "linear", {}, 16, 0.7),
    (2, "rbf", dict(gamma=0.1), 32, 2.0),
]


@pytest.mark.parametrize("loss,kind,kw,s,C", SVM_CASES)
def test_dcd_fp64_iterates_match_oracle(loss, kind, kw, s, C):
    p = inputs.blobs(m=400, n=19, seed=3)
    A = p.A * 0.5
    H = 1203  # not a multiple of s: the last outer step is shorter
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    al, gr, st, rc = B().svm_solve(dev(A), dev(p.y), kb, loss, C, s, H, seed=11, prec="fp64")
    want = oracle.dcd_svm(A, p.y, ko, loss, C, H, seed=11)
    assert st["iters_done"] == H and st["outer_steps"] == -(-H // s)
    assert rel(al.cpu().numpy(), want) < 1e-10
    # the cached gradient equals the gradient of the returned alpha
    gw = oracle.svm_gradient(A, p.y, ko, loss, C, al.cpu().numpy())
    # g = Q alpha - 1 + omega alpha, on the scale of the constant term
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.sqrt(len(gw))


def test_dcd_fp64_repeated_indices_within_a_step():
    p = inputs.blobs(m=7, n=5, seed=4)
    assert len(set(oracle.sample_dcd(2, 7, 0, 16))) < 16
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    for loss in (1, 2):
        al, _, _, _ = B().svm_solve(dev(p.A), dev(p.y), kb, loss, 0.8, 16, 160, seed=2, prec="fp64")
        want = oracle.sstep_dcd_svm(p.A, p.y, ko, loss, 0.8, 16, 160, seed=2)
        assert rel(al.cpu().numpy(), want) < 1e-10


KRR_CASES = [
    ("rbf", dict(gamma=0.5), 4, 1, 1e-2),
    ("rbf", dict(gamma=0.5), 16, 8, 1e-3),
    ("poly", dict(coef0=0.5, degree=2), 8, 3, 1e-1),
    ("linear", {}, 1, 32, 1e-2),
    ("rbf", dict(gamma=2.0), 64, 2, 1e-4),
]


@pytest.mark.parametrize("kind,kw,b,s,lam", KRR_CASES)
def test_bdcd_fp64_iterates_match_oracle(kind, kw, b, s, lam):
    p = inputs.krr_dense(m=350, n=23, seed=5, dtype=np.float64)
    H = 301
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    al, gr, st, rc = B().krr_solve(dev(p.A), dev(p.y), kb, lam, b, s, H, seed=9, prec="fp64")
    want = oracle.bdcd_krr(p.A, p.y, ko, lam, b, H, seed=9)
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.krr_gradient(p.A, p.y, ko, lam, al.cpu().numpy())
    # g = M alpha - y vanishes at convergence: measure it on the scale of y
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.linalg.norm(p.y)


def test_bdcd_fp64_overlapping_blocks_small_m():
    p = inputs.krr_dense(m=12, n=3, seed=6, dtype=np.float64)
    kb, ko = B().kernel("rbf", gamma=0.7), oracle.kernel("rbf", gamma=0.7)
    al, _, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.1, 4, 16, 37, seed=4, prec="fp64", start_iter=3)
    want = oracle.sstep_bdcd_krr(p.A, p.y, ko, 0.1, 4, 16, 37, seed=4, first_block=3)
    assert rel(al.cpu().numpy(), want) < 1e-10


def test_bdcd_fp64_full_block_reaches_closed_form():
    p = inputs.krr_dense(m=64, n=5, seed=7, dtype=np.float64)
    kb, ko = B().kernel("rbf", gamma=1.0), oracle.kernel("rbf", gamma=1.0)
    al, _, st, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.05, 64, 1, 1, seed=0, prec="fp64")
    assert rel(al.cpu().numpy(), oracle.krr_closed_form(p.A, p.y, ko, 0.05)) < 1e-12


def test_bdcd_fp64_converges_with_tolerance():
    p = inputs.krr_dense(m=500, n=8, seed=8, dtype=np.float64)
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    al, gr, st, rc = B().krr_solve(dev(p.A), dev(p.y), kb, 0.01, 16, 8, 200000, seed=1, prec="fp64", tol=1e-9,
                                   check_every=4)
    assert rc == B().OK and st["converged"] == 1 and st["final_metric"] <= 1e-9
    star = oracle.krr_closed_form(p.A, p.y, ko, 0.01)
    assert rel(al.cpu().numpy(), star) < 1e-7


@pytest.mark.parametrize("problem", ["krr", "svm"])
def test_refresh_confirms_tolerance_on_a_recomputed_gradient(problem):
    # With DCD_FLAG_REFRESH a solve that meets tol on its cached gradient
    # recomputes the gradient from alpha before accepting; the metric it
    # reports is that of the recomputed gradient, which the FP64 oracle
    # reproduces for the same alpha up to the kernel block's own rounding.
    if problem == "krr":
        p = inputs.krr_dense(m=700, n=24, seed=31, dtype=np.float32)
        kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
        lam, tol = 0.01, 1e-5
        al, gr, st, rc = B().krr_solve(dev(p.A), dev(p.y), kb, lam, 16, 8, 400000, seed=2, prec="bf16x3", tol=tol,
                                       check_every=2, flags=B().FLAG_REFRESH)
        a = al.cpu().numpy()
        gw = oracle.krr_gradient(p.A, p.y, ko, lam, a)
        true = np.linalg.norm(gw) / np.linalg.norm(p.y)
        scale = np.linalg.norm(p.y)
    else:
        p = inputs.blobs(m=600, n=16, seed=32)
        kb, ko = B().kernel("rbf", gamma=1 / 32), oracle.kernel("rbf", gamma=1 / 32)
        C_, tol = 1.0, 1e-4
        al, gr, st, rc = B().svm_solve(dev(p.A.astype(np.float32)), dev(p.y), kb, 2, C_, 32, 2000000, seed=2,
                                       prec="bf16x3", tol=tol, check_every=4, flags=B().FLAG_REFRESH)
        a = al.cpu().numpy()
        ob = oracle.svm_objectives(p.A.astype(np.float32), p.y, ko, 2, C_, a)
        true = (ob["primal"] - ob["dual"]) / abs(ob["primal"])
        gw = oracle.svm_gradient(p.A.astype(np.float32), p.y, ko, 2, C_, a)
        scale = np.sqrt(len(gw))
    assert rc == B().OK and st["converged"] == 1 and st["refreshes"] >= 1 and st["final_metric"] <= tol
    assert abs(true - st["final_metric"]) <= 0.1 * tol
    assert np.linalg.norm(gr.cpu().numpy() - gw) <= 0.1 * tol * scale


def test_resume_split_run_is_bit_identical():
    p = inputs.krr_dense(m=300, n=11, seed=9, dtype=np.float64)
    kb = B().kernel("rbf", gamma=0.5)
    a1, g1, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.02, 8, 4, 100, seed=5, prec="fp64")
    a2, g2, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.02, 8, 4, 40, seed=5, prec="fp64")
    a2, g2, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.02, 8, 4, 60, seed=5, prec="fp64", alpha=a2, grad=g2,
                                 start_iter=40, flags=B().FLAG_GRAD_VALID)
    assert torch.equal(a1, a2) and torch.equal(g1, g2)


@pytest.mark.parametrize("problem,prec", [(1, "fp64"), (1, "bf16x3"), (0, "bf16")])
def test_graph_replay_and_enqueue_match_direct_launches(problem, prec):
    # Full outer steps replay a captured CUDA graph on a non-default stream;
    # the replayed iterates must be bit-identical to direct launches, across
    # enqueue/run pieces and a final short step (H not a multiple of s).
    if problem == 1:
        p, param, b, s = inputs.krr_dense(m=700, n=40, seed=21, dtype=np.float64), 0.01, 8, 8
    else:
        p, param, b, s = inputs.blobs(m=700, n=40, seed=21), 1.0, 1, 16
    H = 10 * s + 3
    kb = B().kernel("rbf", gamma=0.2)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A, y = dev(p.A), dev(p.y)
        ref = B().Plan(problem, A, y, kb, param, b, s, H, seed=4, prec=prec, flags=B().FLAG_NO_GRAPH)
        ref.run(-1)
        # (the look-ahead with the in-order gradient: the deferred one differs by rounding)
        pl = B().Plan(problem, A, y, kb, param, b, s, H, seed=4, prec=prec, flags=B().FLAG_NO_DEFER)
        assert pl.enqueue(3) == 3
        st, _ = pl.run(2)
        assert st["outer_steps"] == 5 and st["gpu_launches_per_step"] > 0
        assert pl.enqueue(100) == 6  # 5 full steps and the short one
        st, _ = pl.run(0)
        assert st["iters_done"] == H
        side.synchronize()
        assert torch.equal(ref.alpha, pl.alpha) and torch.equal(ref.grad, pl.grad)
        ref.close()
        pl.close()


@pytest.mark.parametrize("prec,fp8", [("bf16x3", False), ("fp8", True), ("tf32x3", False), ("fp16", False)])
def test_lookahead_matches_one_stream_steps(prec, fp8):
    """The look-ahead with the in-order gradient (next step's sample, Gram and
    prep on a second stream, rotating step buffers, step graphs) must give the
    iterates of the one-stream steps bit for bit, also with convergence checks
    and gradient recomputations between steps (which use the idle buffer
    set).  The default look-ahead (the recurrence one step ahead, beside the
    block) gives the same iterates up to rounding: within 1e-5 of them (see
    DEFER_TOL), the same number of steps and recomputations."""
    p = inputs.krr_dense(m=2000, n=48, seed=31, dtype=np.float32)
    kb = B().kernel("rbf", gamma=0.5)
    b, s, H = 16, 64, 23 * 64 + 16 * 5
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        if fp8:
            q, sc = oracle.quantize_e4m3_rows(p.A)
            A = B().Fp8(dev(q), dev(sc))
        else:
            A = dev(p.A)
        y = dev(p.y)
        runs = []
        # one stream (direct) / look-ahead, in-order gradient / look-ahead, deferred gradient
        for flags in (B().FLAG_NO_GRAPH, B().FLAG_NO_DEFER, 0):
            al, gr, st, rc = B().krr_solve(A, y, kb, 1e-3, b, s, H, seed=7, prec=prec, tol=5e-3, check_every=2,
                                           flags=flags | B().FLAG_REFRESH, stream=side.cuda_stream)
            runs.append((al, gr, st))
        side.synchronize()
    (a0, g0, s0), (a1, g1, s1), (a2, g2, s2) = runs
    assert s0["iters_done"] == s1["iters_done"] and s0["refreshes"] == s1["refreshes"] >= 1
    assert torch.equal(a0, a1) and torch.equal(g0, g1)
    assert s2["iters_done"] == s0["iters_done"] and s2["refreshes"] == s0["refreshes"]
    assert rel(a2.cpu().numpy(), a0.cpu().numpy()) < DEFER_TOL
    # the gradient (the residual) is small against its terms: its error is on the scale of ||y||
    assert np.linalg.norm(g2.cpu().numpy() - g0.cpu().numpy()) <= DEFER_TOL * np.linalg.norm(p.y)


@pytest.mark.parametrize("prec", ["fp64", "bf16x3", "fp16", "bf16"])
@pytest.mark.parametrize("loss", [1, 2])
def test_svm_lookahead_matches_one_stream_steps(prec, loss):
    """The K-SVM look-ahead with in-order steps (the next step's sample and
    Gram on a second stream, two buffer sets, step graphs) gives the iterates
    of the one-stream steps bit for bit, with duality-gap checks and gradient
    recomputations between steps and a short last step.  The default is the
    deferred step (the recurrence one step ahead, beside the block, on a
    snapshot of alpha and g plus the previous step's part): the same iterates
    up to the association of the sums (FP64: 1e-10 relative; the tensor-core
    forms, whose s x s cross product rounds its kernel values in FP32 apart
    from the block's epilogue: DEFER_TOL), with the snapshot, the cross
    product and the pending parts as three more kernels per step."""
    p = inputs.blobs(m=1500, n=48, seed=17)
    A = p.A.astype(np.float32)
    kb = B().kernel("rbf", gamma=1 / 64)
    s, H = 16, 16 * 37 + 5
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        Ad, yd = dev(A), dev(p.y)
        runs = []
        for flags in (B().FLAG_NO_GRAPH, B().FLAG_NO_DEFER, 0):
            al, gr, st, rc = B().svm_solve(Ad, yd, kb, loss, 1.0, s, H, seed=3, prec=prec, tol=1e-3, check_every=3,
                                           flags=flags | B().FLAG_REFRESH, stream=side.cuda_stream)
            runs.append((al, gr, st))
        side.synchronize()
    (a0, g0, s0), (a1, g1, s1), (a2, g2, s2) = runs
    assert s0["iters_done"] == s1["iters_done"] == s2["iters_done"]
    assert s0["refreshes"] == s1["refreshes"] == s2["refreshes"]
    assert s1["gpu_launches_per_step"] > 0
    assert torch.equal(a0, a1) and torch.equal(g0, g1)
    assert s2["gpu_launches_per_step"] == s1["gpu_launches_per_step"] + 3
    tol = 1e-10 if prec == "fp64" else DEFER_TOL
    assert rel(a2.cpu().numpy(), a0.cpu().numpy()) < tol
    assert np.max(np.abs(g2.cpu().numpy() - g0.cpu().numpy())) <= tol * max(1.0, float(g0.abs().max()))


@pytest.mark.parametrize("loss", [1, 2])
@pytest.mark.parametrize("m,s,H", [(200, 64, 64 * 9 + 17), (1200, 8, 8 * 40), (700, 128, 128 * 4 + 1)])
def test_svm_deferred_step_matches_oracle(loss, m, s, H):
    """The deferred K-SVM step in FP64 against the oracle's DCD (Algorithm 1,
    the same index sequence): rows sampled several times within a step and
    across consecutive steps (m = 200 with s = 64) exercise the pending
    alpha and the diagonal term of the squared hinge; the longest step the
    one-block recurrence takes (s = 128); a short last step."""
    p = inputs.blobs(m=m, n=24, seed=41)
    kb, ko = B().kernel("rbf", gamma=0.1), oracle.kernel("rbf", gamma=0.1)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        al, gr, st, rc = B().svm_solve(dev(p.A), dev(p.y), kb, loss, 0.9, s, H, seed=13, prec="fp64",
                                       stream=side.cuda_stream)
        side.synchronize()
    assert rc == B().OK and st["iters_done"] == H
    want = oracle.dcd_svm(p.A, p.y, ko, loss, 0.9, H, seed=13)
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.svm_gradient(p.A, p.y, ko, loss, 0.9, want)
    assert np.max(np.abs(gr.cpu().numpy() - gw)) < 1e-10 * max(1.0, np.max(np.abs(gw)))


@pytest.mark.parametrize("csr", [False, True])
def test_svm_deferred_step_with_host_buffers_matches_device_buffers(csr):
    """The end-to-end form the bench times: a solve through the C ABI with the
    data, labels and alpha in host memory (copies in and out on the caller's
    stream, the deferred K-SVM steps between them) gives the bits of the same
    solve on device buffers on that stream."""
    kb = B().kernel("poly", coef0=1.0, degree=3) if csr else B().kernel("rbf", gamma=0.05)
    if csr:
        p = inputs.sparse_csr(m=2500, n=3000, nnz_per_row=10, seed=12)
        Ad = B().Csr(dev(p.row_ptr), dev(p.col_idx), dev(p.values), p.n)
        Ah = B().Csr(p.row_ptr, p.col_idx, p.values, p.n)
        prec, loss, C_ = "bf16x3", 2, 0.5
    else:
        p = inputs.blobs(m=1200, n=40, seed=12)
        Ad, Ah = dev(p.A), np.ascontiguousarray(p.A)
        prec, loss, C_ = "fp64", 1, 1.0
    s, H = 16, 16 * 9 + 3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        ad, gd, sd, _ = B().svm_solve(Ad, dev(p.y), kb, loss, C_, s, H, seed=6, prec=prec,
                                      stream=side.cuda_stream)
        ah, gh, sh, _ = B().svm_solve(Ah, p.y.copy(), kb, loss, C_, s, H, seed=6, prec=prec,
                                      flags=B().FLAG_HOST_IO, stream=side.cuda_stream)
        side.synchronize()
    assert sd["iters_done"] == sh["iters_done"] == H
    assert sd["gpu_launches_per_step"] == sh["gpu_launches_per_step"] > 0
    assert np.array_equal(ad.cpu().numpy(), ah) and np.array_equal(gd.cpu().numpy(), gh)


@pytest.mark.parametrize("kind,kw", [("poly", dict(coef0=1.0, degree=3)), ("linear", {})])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x3", 1e-4)])
def test_svm_deferred_step_other_kernels_match_oracle(kind, kw, prec, tol):
    """The deferred K-SVM step with the polynomial and linear kernels (the
    s x s cross product and the block in the same kernel family), squared
    hinge, s = 32 with rows recurring across steps (m = 300), against the
    oracle's DCD on the same index sequence."""
    p = inputs.blobs(m=300, n=20, seed=44)
    A = p.A / np.sqrt(20.0)
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    side = torch.cuda.Stream()
    H = 32 * 12 + 5
    with torch.cuda.stream(side):
        Ad = dev(A if prec == "fp64" else A.astype(np.float32))
        al, _, st, rc = B().svm_solve(Ad, dev(p.y), kb, 2, 0.7, 32, H, seed=21, prec=prec, stream=side.cuda_stream)
        side.synchronize()
    assert rc == B().OK and st["iters_done"] == H
    Ar = A if prec == "fp64" else A.astype(np.float32).astype(np.float64)
    want = oracle.dcd_svm(Ar, p.y, ko, 2, 0.7, H, seed=21)
    assert rel(al.cpu().numpy(), want) < tol


def test_svm_deferred_steps_split_over_calls_match_one_call():
    """The deferred K-SVM step keeps the recurrence and the pending parts
    computed ahead across dcd_plan_enqueue / dcd_plan_run calls: a solve in
    pieces (with a short last step) gives the bits of the solve in one call."""
    p = inputs.blobs(m=900, n=32, seed=5)
    kb = B().kernel("rbf", gamma=0.05)
    s, H = 16, 16 * 13 + 9
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A, y = dev(p.A), dev(p.y)
        ref = B().Plan(0, A, y, kb, 1.0, 1, s, H, seed=8, prec="fp64", loss=2)
        ref.run(-1)
        pl = B().Plan(0, A, y, kb, 1.0, 1, s, H, seed=8, prec="fp64", loss=2)
        assert pl.enqueue(4) == 4
        st, _ = pl.run(3)
        assert pl.enqueue(2) == 2
        st, _ = pl.run(-1)
        assert st["iters_done"] == H and st["outer_steps"] == 14
        side.synchronize()
        assert torch.equal(ref.alpha, pl.alpha) and torch.equal(ref.grad, pl.grad)
        ref.close()
        pl.close()


@pytest.mark.parametrize("prec,fp8,s,b", [("fp64", False, 8, 8), ("bf16x3", False, 48, 32), ("fp8", True, 40, 32),
                                          ("fp16", False, 64, 32)])
def test_krr_lookahead_off_the_cluster_path_matches_one_stream_steps(prec, fp8, s, b):
    """K-RR steps that do not take the single-cluster recurrence (FP64, or s b
    above one cluster: the blocked recurrence) get the in-order look-ahead:
    the iterates equal the one-stream steps' bit for bit, with residual
    checks, gradient recomputations and a short last step."""
    p = inputs.krr_dense(m=3000, n=64, seed=23, dtype=np.float32)
    kb = B().kernel("rbf", gamma=0.5)
    H = 5 * s + 3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        if fp8:
            q, sc = oracle.quantize_e4m3_rows(p.A)
            A = B().Fp8(dev(q), dev(sc))
        else:
            A = dev(p.A.astype(np.float64) if prec == "fp64" else p.A)
        y = dev(p.y)
        runs = []
        for flags in (B().FLAG_NO_GRAPH, 0):
            al, gr, st, rc = B().krr_solve(A, y, kb, 1e-2, b, s, H, seed=5, prec=prec, tol=1e-3, check_every=2,
                                           flags=flags | B().FLAG_REFRESH, stream=side.cuda_stream)
            runs.append((al, gr, st))
        side.synchronize()
    (a0, g0, s0), (a1, g1, s1) = runs
    assert s0["iters_done"] == s1["iters_done"] and s0["refreshes"] == s1["refreshes"]
    assert torch.equal(a0, a1) and torch.equal(g0, g1)


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
def test_deferred_steps_split_over_calls_match_one_call(prec):
    """The deferred look-ahead keeps the recurrence and x computed ahead across
    dcd_plan_enqueue / dcd_plan_run calls: a solve split into pieces (with a
    final short step) gives the bits of the same solve in one call."""
    p = inputs.krr_dense(m=2000, n=48, seed=29, dtype=np.float32)
    kb = B().kernel("rbf", gamma=0.5)
    b, s, H = 16, 64, 64 * 11 + 16 * 3
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A, y = dev(p.A), dev(p.y)
        ref = B().Plan(1, A, y, kb, 1e-3, b, s, H, seed=4, prec=prec)
        ref.run(-1)
        pl = B().Plan(1, A, y, kb, 1e-3, b, s, H, seed=4, prec=prec)
        assert pl.enqueue(3) == 3
        st, _ = pl.run(2)
        assert pl.enqueue(4) == 4
        st, _ = pl.run(-1)
        assert st["iters_done"] == H and st["outer_steps"] == 12
        side.synchronize()
        assert torch.equal(ref.alpha, pl.alpha) and torch.equal(ref.grad, pl.grad)
        ref.close()
        pl.close()


# The deferred gradient evaluates the block's part at the next step's rows in
# a separate s b x s b product whose FP32 epilogue groups other rows into
# warps: where a warp's RBF terms decide between the factored and the clamped
# exponent form differently, the kernel value differs by FP32 rounding
# (~1e-7 relative), and the iterates drift from the in-order steps' by a few
# 1e-7 (measured 3e-7).  A dropped or misplaced term (the cross product, the
# update's repeat term) changes them at order 1, far above this tolerance and
# the mixed forms' error against the oracle (1e-4).
DEFER_TOL = 1e-5


@pytest.mark.parametrize("prec", ["fp16", "bf16x3"])
@pytest.mark.parametrize("m,s,b,H", [(2000, 64, 16, 64 * 9), (600, 40, 16, 40 * 7 + 13), (5000, 16, 8, 16 * 12)])
def test_deferred_gradient_matches_in_order_steps(prec, m, s, b, H):
    """The recurrence of step k+1 computed beside the block of step k, from the
    gradient before that block, the s b x s b cross product at the rows step
    k+1 samples and the update's repeat term: the iterates equal those of the
    in-order steps up to rounding (DEFER_TOL).  m = 600 with s b = 640
    repeats most rows within and across consecutive steps (the repeat term);
    the ragged budget ends on a short step after the deferred ones."""
    p = inputs.krr_dense(m=m, n=40, seed=41, dtype=np.float32)
    kb = B().kernel("rbf", gamma=0.5)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A, y = dev(p.A), dev(p.y)
        runs = [B().krr_solve(A, y, kb, 1e-3, b, s, H, seed=9, prec=prec, flags=f, stream=side.cuda_stream)
                for f in (B().FLAG_NO_DEFER, 0)]
        side.synchronize()
    (a1, g1, s1, _), (a2, g2, s2, _) = runs
    assert s1["iters_done"] == s2["iters_done"] == H
    assert rel(a2.cpu().numpy(), a1.cpu().numpy()) < DEFER_TOL
    assert np.linalg.norm(g2.cpu().numpy() - g1.cpu().numpy()) <= DEFER_TOL * np.linalg.norm(p.y)


@pytest.mark.parametrize("kind,kw", [("poly", dict(coef0=1.0, degree=3)), ("linear", {})])
@pytest.mark.parametrize("prec", ["fp16", "bf16x3", "fp8"])
def test_deferred_gradient_other_kernels_match_oracle(kind, kw, prec):
    """The deferred look-ahead with the polynomial and linear kernels (the cross
    product's epilogue takes their forms, with no own-sample rule), at the
    bench's (s, b) = (64, 16): against the FP64 oracle (Algorithm 3) within
    the mixed forms' tolerances, and against the in-order steps (DEFER_TOL).
    fp8: the oracle runs on the dequantised rows."""
    p = inputs.krr_dense(m=2000, n=48, seed=37, dtype=np.float32)
    A32 = p.A
    b, s, H, lam = 16, 64, 64 * 8 + 16, 1e-2
    kb, ko = B().kernel(kind, **kw), oracle.kernel(kind, **kw)
    if prec == "fp8":
        q, sc = oracle.quantize_e4m3_rows(A32)
        A64 = oracle.dequantize_e4m3_rows(q, sc)
    else:
        A64 = A32.astype(np.float64)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A = B().Fp8(dev(q), dev(sc)) if prec == "fp8" else dev(A32)
        runs = [B().krr_solve(A, dev(p.y), kb, lam, b, s, H, seed=5, prec=prec, flags=f, stream=side.cuda_stream)
                for f in (B().FLAG_NO_DEFER, 0)]
        side.synchronize()
    (a1, _, _, _), (a2, _, st2, _) = runs
    assert st2["iters_done"] == H
    assert rel(a2.cpu().numpy(), a1.cpu().numpy()) < DEFER_TOL
    want = oracle.bdcd_krr(A64, p.y, ko, lam, b, H, seed=5)
    a = a2.cpu().numpy()
    assert rel(a, want) < (ALPHA_TOL["fp16"] if prec in ("fp16", "fp8") else 1e-4)
    f_got = oracle.krr_objective(A64, p.y, ko, lam, a)
    f_want = oracle.krr_objective(A64, p.y, ko, lam, want)
    assert abs(f_got - f_want) <= 1e-6 * abs(f_want)


def test_nonzero_alpha0_gradient_pass():
    p = inputs.blobs(m=260, n=9, seed=10)
    kb, ko = B().kernel("rbf", gamma=0.3), oracle.kernel("rbf", gamma=0.3)
    a0 = np.random.default_rng(0).uniform(0, 0.5, 260)
    al, gr, _, _ = B().svm_solve(dev(p.A), dev(p.y), kb, 1, 1.0, 4, 301, seed=3, prec="fp64", alpha=dev(a0))
    want = oracle.dcd_svm(p.A, p.y, ko, 1, 1.0, 301, seed=3, alpha0=a0)
    assert rel(al.cpu().numpy(), want) < 1e-10
    gw = oracle.svm_gradient(p.A, p.y, ko, 1, 1.0, want)
    assert np.linalg.norm(gr.cpu().numpy() - gw) < 1e-10 * np.sqrt(len(gw))


def test_host_io_matches_device_path():
    p = inputs.krr_dense(m=200, n=10, seed=11, dtype=np.float64)
    kb = B().kernel("rbf", gamma=0.5)
    ad, gd, _, _ = B().krr_solve(dev(p.A), dev(p.y), kb, 0.05, 4, 4, 50, seed=1, prec="fp64")
    ah, gh, _, _ = B().krr_solve(np.ascontiguousarray(p.A), p.y.copy(), kb, 0.05, 4, 4, 50, seed=1, prec="fp64",
                                 flags=B().FLAG_HOST_IO)
    assert np.array_equal(ad.cpu().numpy(), ah) and np.array_equal(gd.cpu().numpy(), gh)


def test_svm_rejects_non_binary_labels():
    p = inputs.blobs(m=50, n=3, seed=1)
    y = p.y.copy()
    y[3] = 0.5
    with pytest.raises(B().DcdError) as e:
        B().svm_solve(dev(p.A), dev(y), B().kernel("linear"), 1, 1.0, 1, 10, prec="fp64")
    assert e.value.status == B().EINVAL


# --------------------------------------------------- mixed-form solves ----
# Error of each tensor-core precision against the FP64 oracle on the same
# index stream.  bf16x3 is the mixed form held to the targets (dual objective
# 1e-6, alpha 1e-4); plain bf16 / tf32 perturb the data by 2^-9 / 2^-11 and
# are held to the error levels that perturbation implies (measured on GB300:
# bf16 ~6e-4, tf32 ~3e-4 in alpha).
# The split forms are held to the mixed-precision targets (objective 1e-6,
# alpha 1e-4; split tf32 to alpha 1e-5): their kernel entries carry the FP32
# epilogue's ~2.5e-7 relative error, which bounds the objective at long
# chains (s = 32) near 1e-7.
# fp16 (11 significant bits, per-row power-of-two scales) meets the objective
# target; its alpha error reaches 3.3e-4 to 3.8e-4 on the long K-SVM and
# look-ahead runs here (measured on GB300), so it is held to 1e-3 there.
ALPHA_TOL = {"tf32x3": 1e-5, "bf16x3": 1e-4, "tf32": 1e-3, "bf16": 3e-3, "fp16": 1e-3}
OBJ_TOL = {"tf32x3": 1e-6, "bf16x3": 1e-6, "tf32": 1e-4, "bf16": 3e-4, "fp16": 1e-6}


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "bf16", "fp16"])
@pytest.mark.parametrize("s,b", [(1, 16), (16, 16), (7, 8), (40, 4), (9, 12), (64, 16)])
def test_bdcd_mixed_matches_oracle(prec, s, b):
    """s = 1: the single-block path; (7, 8): the one-CTA refined chain with an
    odd number of streamed panels; (16, 16), (40, 4), (9, 12): the cluster
    recurrence with 16 and 9 CTAs and several blocks per CTA; (64, 16): the
    bench's shape, 32 super-blocks of two blocks on a full 16-CTA cluster."""
    p = inputs.krr_dense(m=1000, n=64, seed=12, dtype=np.float32)
    A64 = p.A.astype(np.float64)
    lam, H = 1e-2, 640
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    al, gr, st, _ = B().krr_solve(dev(p.A), dev(p.y), kb, lam, b, s, H, seed=3, prec=prec)
    want = oracle.bdcd_krr(A64, p.y, ko, lam, b, H, seed=3)
    a = al.cpu().numpy()
    assert rel(a, want) < ALPHA_TOL[prec]
    f_got = oracle.krr_objective(A64, p.y, ko, lam, a)
    f_want = oracle.krr_objective(A64, p.y, ko, lam, want)
    assert abs(f_got - f_want) <= OBJ_TOL[prec] * abs(f_want)


@pytest.mark.parametrize("sigma,s", [(10.0, 8), (10.0, 32), (100.0, 8), (100.0, 32)])
def test_bdcd_fp64_small_m_lambda(sigma, s):
    """The FP64 form at small m * lambda (m = 1000, lambda = 1e-6, b = 32, the
    corner of the batched sweep): G_jj = K_jj / lambda + m I is dominated by
    the kernel block.  sigma = 100 makes K nearly all ones, cond(G_jj) ~ 8e3,
    where two FP32-chain refinements leave ~1e-8; the rounds are decided on
    the device until the correction is at FP64 accuracy.  Iterates within
    1e-10 of the oracle (Algorithm 3)."""
    g = np.random.default_rng(17)
    A = g.standard_normal((1000, 128))
    y = g.standard_normal(1000)
    gam = 1.0 / (2 * sigma * sigma)
    kb, ko = B().kernel("rbf", gamma=gam), oracle.kernel("rbf", gamma=gam)
    H = 3 * s + 5  # ragged last outer step
    al, gr, st, _ = B().krr_solve(dev(A), dev(y), kb, 1e-6, 32, s, H, seed=4, prec="fp64")
    want = oracle.bdcd_krr(A, y, ko, 1e-6, 32, H, seed=4)
    assert rel(al.cpu().numpy(), want) < 1e-10


def test_bdcd_fp64_near_singular_blocks_fall_back():
    """K ~ J with lambda = 1e-7: cond(G_jj) ~ 1e6, where the FP32 chain
    contracts the error by only ~1e-2 per refinement round and four rounds
    leave ~1e-8, so the step falls back to the FP64 Cholesky kernels.  Both
    sides then solve the same ill-conditioned block systems in FP64; their
    iterates agree to about cond(G_jj) * 2^-53 (tolerance 1e-8)."""
    g = np.random.default_rng(18)
    A = g.standard_normal((300, 16)) * 0.01
    y = g.standard_normal(300)
    kb, ko = B().kernel("rbf", gamma=1e-3), oracle.kernel("rbf", gamma=1e-3)
    al, _, st, _ = B().krr_solve(dev(A), dev(y), kb, 1e-7, 32, 4, 18, seed=2, prec="fp64")
    want = oracle.bdcd_krr(A, y, ko, 1e-7, 32, 18, seed=2)
    assert np.all(np.isfinite(al.cpu().numpy()))
    assert rel(al.cpu().numpy(), want) < 1e-8


@pytest.mark.parametrize("prec,fp8", [("bf16x3", False), ("tf32x3", False), ("fp8", True), ("fp16", False)])
def test_lookahead_solve_matches_oracle(prec, fp8):
    """The look-ahead step the bench times (next step's products on a second
    stream, the block as the chain's programmatic dependent, even/odd step
    graphs) at the bench's (s, b) = (64, 16), compared directly with the FP64
    oracle (Algorithm 3) on the same index stream: alpha within 1e-4 and the
    dual objective within 1e-6 (fp8: on the dequantised rows)."""
    p = inputs.krr_dense(m=2000, n=48, seed=31, dtype=np.float32)
    b, s, H, lam = 16, 64, 23 * 64 + 16 * 5, 1e-3
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    if fp8:
        q, sc = oracle.quantize_e4m3_rows(p.A)
        A64 = oracle.dequantize_e4m3_rows(q, sc)
    else:
        A64 = p.A.astype(np.float64)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        A = B().Fp8(dev(q), dev(sc)) if fp8 else dev(p.A)
        al, gr, st, rc = B().krr_solve(A, dev(p.y), kb, lam, b, s, H, seed=7, prec=prec, stream=side.cuda_stream)
        side.synchronize()
    assert st["iters_done"] == H
    want = oracle.bdcd_krr(A64, p.y, ko, lam, b, H, seed=7)
    a = al.cpu().numpy()
    assert rel(a, want) < (ALPHA_TOL["fp16"] if prec == "fp16" else 1e-4)
    f_got = oracle.krr_objective(A64, p.y, ko, lam, a)
    f_want = oracle.krr_objective(A64, p.y, ko, lam, want)
    assert abs(f_got - f_want) <= 1e-6 * abs(f_want)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "fp8"])
@pytest.mark.parametrize("m,s,b", [(3000, 48, 32), (700, 128, 32), (5000, 100, 16), (2500, 300, 8)])
def test_bdcd_long_chain_blocked_panels(prec, m, s, b):
    """s*b above one cluster launch (1024 rows): diagonal panels of the
    cluster recurrence joined by FP64 updates of the later right-hand sides;
    m = 700 with s*b = 4096 repeats every index several times per step, also
    across panels.  fp8: the oracle runs on the dequantised rows."""
    p = inputs.krr_dense(m=m, n=64, seed=21, dtype=np.float32)
    lam, H = 1e-2, 2 * s
    kb, ko = B().kernel("rbf", gamma=0.5), oracle.kernel("rbf", gamma=0.5)
    if prec == "fp8":
        q, sc = oracle.quantize_e4m3_rows(p.A)
        A64 = oracle.dequantize_e4m3_rows(q, sc)
        Ad = B().Fp8(dev(q), dev(sc))
    else:
        A64 = p.A.astype(np.float64)
        Ad = dev(p.A)
    al, gr, st, _ = B().krr_solve(Ad, dev(p.y), kb, lam, b, s, H, seed=5, prec=prec)
    want = oracle.bdcd_krr(A64, p.y, ko, lam, b, H, seed=5)
    a = al.cpu().numpy()
    assert rel(a, want) < ALPHA_TOL.get(prec, 1e-4)
    f_got = oracle.krr_objective(A64, p.y, ko, lam, a)
    f_want = oracle.krr_objective(A64, p.y, ko, lam, want)
    assert abs(f_got - f_want) <= OBJ_TOL.get(prec, 1e-6) * abs(f_want)


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3", "tf32", "bf16", "fp16"])
@pytest.mark.parametrize("s", [8, 32])
@pytest.mark.parametrize("deferred", [False, True])
def test_dcd_mixed_matches_oracle(prec, s, deferred):
    """K-SVM-L1 on the blobs; s = 32 is the CSR workload's step size (the
    register-resident chain reading an FP32 Gram).  On the default stream the
    steps run in order; on a stream of the caller's, as the deferred K-SVM
    step (the chain one step ahead, beside the block)."""
    p = inputs.blobs(m=700, n=64, seed=13)
    kb, ko = B().kernel("rbf", gamma=1 / 128), oracle.kernel("rbf", gamma=1 / 128)
    side = torch.cuda.Stream() if deferred else None
    with torch.cuda.stream(side or torch.cuda.current_stream()):
        al, _, st, _ = B().svm_solve(dev(p.A.astype(np.float32)), dev(p.y), kb, 1, 1.0, s, 2000, seed=0, prec=prec,
                                     stream=side.cuda_stream if deferred else None)
        torch.cuda.synchronize()
    want = oracle.sstep_dcd_svm(p.A.astype(np.float32).astype(np.float64), p.y, ko, 1, 1.0, s, 2000, seed=0)
    a = al.cpu().numpy()
    A64 = p.A.astype(np.float32).astype(np.float64)
    f = oracle.svm_objectives(A64, p.y, ko, 1, 1.0, a)
    fw = oracle.svm_objectives(A64, p.y, ko, 1, 1.0, want)
    assert abs(f["dual"] - fw["dual"]) <= OBJ_TOL[prec] * abs(fw["dual"])
    assert rel(a, want) < ALPHA_TOL[prec]
