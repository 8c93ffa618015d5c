"""Row-sharded outer steps (the multi-GPU layout): rows of A, y, alpha and g
split over ranks, one all-gather of the sampled rows per outer step, the
Gram and the recurrence repeated on every rank, the kernel block applied to
each rank's own rows.

On the CPU the driver (`paper_2406_18001_gb300.sharded`) runs with the step's
pieces written out in numpy here (kernel values from the FP64 oracle), as
emulated ranks in one process and as world_size-2 gloo ranks: the solve
must not depend on the number of ranks at all (bit for bit), and must match
the oracle's Algorithms 2 and 4.  On the GPU the same driver runs the pieces
through the library's C ABI.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_2406_18001_gb300 import sharded as SH


class NumpyShardOps:
    """The pieces of a sharded step on the CPU (torch CPU tensors in and out):
    the sample stream and the kernel values from the oracle, the rest written
    out from Algorithms 2 and 4 and the step's description."""

    def __init__(self, kernel):
        self.ko = kernel

    def sample(self, problem, seed, m, b, first, count, device):
        if problem == SH.KRR:
            S = oracle.sample_bdcd(seed, m, b, first, count).reshape(-1)
        else:
            S = oracle.sample_dcd(seed, m, first, count)
        return torch.from_numpy(np.asarray(S, dtype=np.int32))

    def contribute(self, A, row0, m, S, g, alpha, y):
        A, S = A.numpy(), S.numpy()
        buf = np.zeros((S.size, A.shape[1] + 4))
        for j, key in enumerate(S):
            assert 0 <= key < m
            r = key - row0
            if 0 <= r < A.shape[0]:
                buf[j, :4] = (1.0, g[r], alpha[r], y[r])
                buf[j, 4:] = A[r]
        return torch.from_numpy(buf)

    def assemble(self, gathered, nranks, S, n):
        S = S.numpy()
        cnt = S.size
        parts = gathered.numpy().reshape(nranks, cnt, n + 4)
        own = parts[:, :, 0]
        assert np.all(own.sum(0) == 1.0) and np.all((own == 0.0) | (own == 1.0))
        pick = parts[own.argmax(0), np.arange(cnt)]
        first = np.array([int(np.argmax(S == key)) for key in S], dtype=np.int32)
        return (torch.from_numpy(pick[:, 4:].copy()), torch.from_numpy(pick[:, 1].copy()),
                torch.from_numpy(pick[:, 2].copy()), torch.from_numpy(pick[:, 3].copy()), torch.from_numpy(first))

    def gram(self, A_S, first, k):
        return torch.from_numpy(oracle.kernel_block(self.ko, A_S.numpy(), first.numpy(), rows=first.numpy()))

    def krr_recurrence(self, Kss, S, b, lam, m, g_S):
        # Algorithm 4's step: G_jt = K_jt / lambda + m [S_p == S_q]; block j solves
        # G_jj delta_j = -g_S[j] - sum_{t<j} G_jt delta_t
        K, S, g = Kss.numpy(), S.numpy(), g_S.numpy()
        G = K / lam + m * (S[:, None] == S[None, :])
        s = S.size // b
        delta = np.zeros(S.size)
        for j in range(s):
            J = slice(j * b, (j + 1) * b)
            rhs = -g[J] - G[J, : j * b] @ delta[: j * b]
            delta[J] = np.linalg.solve(G[J, J], rhs)
        return torch.from_numpy(delta), torch.from_numpy(delta / lam)

    def svm_recurrence(self, Kss, S, y_S, a_S, g_S, loss, C_):
        # Algorithm 2's inner loop on the gathered values
        K, S, y, a, g = Kss.numpy(), S.numpy(), y_S.numpy(), a_S.numpy(), g_S.numpy()
        omega, nu = (0.5 / C_, np.inf) if loss == 2 else (0.0, C_)
        th = np.zeros(S.size)
        for j in range(S.size):
            prev = [t for t in range(j) if S[t] == S[j]]
            rho = a[j] + sum(th[t] for t in prev)
            gj = g[j] + sum(y[j] * y[t] * K[j, t] * th[t] for t in range(j)) + omega * (rho - a[j])
            eta = K[j, j] + omega
            pg = min(gj, 0.0) if rho == 0.0 else (max(gj, 0.0) if rho == nu else gj)
            if eta <= 0.0 or pg == 0.0:
                continue
            th[j] = min(max(rho - gj / eta, 0.0), nu) - rho
        return torch.from_numpy(th), torch.from_numpy(y * th)

    def apply(self, A, row0, A_S, S, k, w, rowscale, g):
        A, P = A.numpy(), A_S.numpy()
        both = np.vstack([A, P])
        Kb = oracle.kernel_block(self.ko, both, np.arange(A.shape[0], both.shape[0]), rows=np.arange(A.shape[0]))
        s = (Kb * w.numpy()[None, :]).sum(axis=1)  # per-row sums: independent of the other rows
        g += torch.from_numpy(s * (rowscale.numpy() if rowscale is not None else 1.0))

    def update(self, S, delta, diag, row0, alpha, g):
        S, d = S.numpy(), delta.numpy()
        for p, key in enumerate(S):
            r = key - row0
            if not (0 <= r < alpha.numel()) or key in S[:p]:
                continue
            tot = 0.0
            for q in range(p, S.size):
                if S[q] == key:
                    tot += d[q]
            alpha[r] += tot
            g[r] += diag * tot


def _problem(kind, m=90, n=7, seed=3):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * 0.6
    if kind == SH.KRR:
        y = np.sin(A @ rng.standard_normal(n)) + 0.1 * rng.standard_normal(m)
    else:
        y = np.where(A[:, 0] + 0.3 * rng.standard_normal(m) >= 0, 1.0, -1.0)
    return A, y


def _solve_local(kind, A, y, nranks, spec, ko, kd):
    ops = NumpyShardOps(ko)
    shards = [SH.RowShard(ops, spec, torch.from_numpy(A[r0:r0 + c].copy()), torch.from_numpy(y[r0:r0 + c].copy()),
                          r0, kd) for r0, c in SH.split_rows(A.shape[0], nranks)]
    SH.run_local(shards)
    return (np.concatenate([sh.alpha.numpy() for sh in shards]), np.concatenate([sh.g.numpy() for sh in shards]))


KERNELS = [("rbf", dict(gamma=0.4)), ("poly", dict(coef0=1.0, degree=3)), ("linear", {})]


@pytest.mark.parametrize("kname,kw", KERNELS)
def test_krr_sharded_solve_is_independent_of_rank_count_and_matches_algorithm_4(kname, kw):
    A, y = _problem(SH.KRR)
    m = A.shape[0]
    ko = oracle.kernel(kname, **kw)
    spec = SH.ShardSpec(SH.KRR, m=m, b=3, s=4, H=26, param=0.05, seed=9)  # 26 blocks: a short last step
    base = _solve_local(SH.KRR, A, y, 1, spec, ko, None)
    for P in (2, 3, 5):
        got = _solve_local(SH.KRR, A, y, P, spec, ko, None)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
    want = oracle.sstep_bdcd_krr(A, y, ko, 0.05, 3, 4, 26, seed=9)
    assert np.linalg.norm(base[0] - want) <= 1e-11 * np.linalg.norm(want)
    # the cached gradient is the gradient of the final alpha
    gw = oracle.krr_gradient(A, y, ko, 0.05, base[0])
    assert np.linalg.norm(base[1] - gw) <= 1e-10 * np.linalg.norm(gw)


@pytest.mark.parametrize("loss", [1, 2])
def test_svm_sharded_solve_is_independent_of_rank_count_and_matches_algorithm_2(loss):
    A, y = _problem(SH.SVM)
    m = A.shape[0]
    ko = oracle.kernel("rbf", gamma=0.3)
    spec = SH.ShardSpec(SH.SVM, m=m, b=1, s=8, H=203, param=0.7, loss=loss, seed=4)
    base = _solve_local(SH.SVM, A, y, 1, spec, ko, None)
    for P in (2, 4):
        got = _solve_local(SH.SVM, A, y, P, spec, ko, None)
        assert np.array_equal(got[0], base[0]) and np.array_equal(got[1], base[1])
    want = oracle.sstep_dcd_svm(A, y, ko, loss, 0.7, 8, 203, seed=4)
    assert np.max(np.abs(base[0] - want)) <= 1e-11 * max(1.0, np.max(np.abs(want)))
    gw = oracle.svm_gradient(A, y, ko, loss, 0.7, base[0])
    assert np.max(np.abs(base[1] - gw)) <= 1e-10 * max(1.0, np.max(np.abs(gw)))


def test_sampled_rows_repeat_across_blocks_and_ranks():
    # m small against s*b: the s blocks of a step overlap, and a row sampled twice
    # may belong to either rank
    A, y = _problem(SH.KRR, m=12, n=4, seed=5)
    ko = oracle.kernel("rbf", gamma=0.5)
    spec = SH.ShardSpec(SH.KRR, m=12, b=4, s=5, H=15, param=0.1, seed=2)
    S = oracle.sample_bdcd(2, 12, 4, 0, 5).reshape(-1)
    assert len(set(S.tolist())) < S.size
    base = _solve_local(SH.KRR, A, y, 1, spec, ko, None)
    got = _solve_local(SH.KRR, A, y, 3, spec, ko, None)
    assert np.array_equal(got[0], base[0])
    want = oracle.sstep_bdcd_krr(A, y, ko, 0.1, 4, 5, 15, seed=2)
    assert np.linalg.norm(base[0] - want) <= 1e-11 * np.linalg.norm(want)


def test_split_rows_covers_every_row_once():
    for m, P in ((10, 3), (7, 7), (5, 1), (100, 8)):
        parts = SH.split_rows(m, P)
        assert len(parts) == P
        assert parts[0][0] == 0 and sum(c for _, c in parts) == m
        assert all(parts[i][0] + parts[i][1] == parts[i + 1][0] for i in range(P - 1))
        assert max(c for _, c in parts) - min(c for _, c in parts) <= 1


# ----------------------------------------------------- world_size 2, gloo --
def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _gloo_rank(rank, ws, port, kind, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        A, y = _problem(kind)
        if kind == SH.KRR:
            ko = oracle.kernel("rbf", gamma=0.4)
            spec = SH.ShardSpec(SH.KRR, m=A.shape[0], b=3, s=4, H=26, param=0.05, seed=9)
        else:
            ko = oracle.kernel("rbf", gamma=0.3)
            spec = SH.ShardSpec(SH.SVM, m=A.shape[0], b=1, s=8, H=203, param=0.7, loss=1, seed=4)
        r0, cnt = SH.split_rows(A.shape[0], ws)[rank]
        shard = SH.RowShard(NumpyShardOps(ko), spec, torch.from_numpy(A[r0:r0 + cnt].copy()),
                            torch.from_numpy(y[r0:r0 + cnt].copy()), r0, None)
        SH.run_dist(shard, SH.DistExchange())
        np.save(os.path.join(out_dir, f"{kind}_alpha{rank}.npy"), shard.alpha.numpy())
        np.save(os.path.join(out_dir, f"{kind}_g{rank}.npy"), shard.g.numpy())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", [SH.KRR, SH.SVM])
def test_gloo_two_ranks_match_the_single_rank_solve_bit_for_bit(kind, tmp_path):
    ws = 2
    mp.start_processes(_gloo_rank, args=(ws, _free_port(), kind, str(tmp_path)), nprocs=ws, start_method="spawn")
    alpha = np.concatenate([np.load(tmp_path / f"{kind}_alpha{r}.npy") for r in range(ws)])
    g = np.concatenate([np.load(tmp_path / f"{kind}_g{r}.npy") for r in range(ws)])
    A, y = _problem(kind)
    if kind == SH.KRR:
        ko = oracle.kernel("rbf", gamma=0.4)
        spec = SH.ShardSpec(SH.KRR, m=A.shape[0], b=3, s=4, H=26, param=0.05, seed=9)
    else:
        ko = oracle.kernel("rbf", gamma=0.3)
        spec = SH.ShardSpec(SH.SVM, m=A.shape[0], b=1, s=8, H=203, param=0.7, loss=1, seed=4)
    base = _solve_local(kind, A, y, 1, spec, ko, None)
    assert np.array_equal(alpha, base[0]) and np.array_equal(g, base[1])


# ------------------------------------------------------------------ GPU --
def _gpu_case(kind, prec, nranks, m, n, b, s, H, param, kd, seed=0, loss=1):
    from paper_2406_18001_gb300 import binding as B  # noqa: F401
    A, y = _problem(kind, m=m, n=n, seed=seed + 1)
    dev = torch.device("cuda")
    ops = SH.CudaShardOps(prec)
    spec = SH.ShardSpec(kind, m=m, b=b, s=s, H=H, param=param, loss=loss, seed=seed)
    At, yt = torch.from_numpy(A).to(dev), torch.from_numpy(y).to(dev)
    shards = [SH.RowShard(ops, spec, At[r0:r0 + c], yt[r0:r0 + c], r0, kd) for r0, c in SH.split_rows(m, nranks)]
    SH.run_local(shards)
    alpha = torch.cat([sh.alpha for sh in shards]).cpu().numpy()
    g = torch.cat([sh.g for sh in shards]).cpu().numpy()
    return A, y, alpha, g


@pytest.mark.gpu
@pytest.mark.parametrize("kind", [SH.KRR, SH.SVM])
def test_gpu_sharded_fp64_matches_the_plan_and_is_rank_independent(kind):
    from paper_2406_18001_gb300 import binding as B
    m, n = 1500, 48
    if kind == SH.KRR:
        kd = B.kernel("rbf", gamma=0.3)
        args = dict(b=8, s=4, H=60, param=1e-2)
    else:
        kd = B.kernel("rbf", gamma=0.3)
        args = dict(b=1, s=8, H=400, param=1.0)
    A, y, a1, g1 = _gpu_case(kind, "fp64", 1, m, n, kd=kd, **args)
    _, _, a2, g2 = _gpu_case(kind, "fp64", 2, m, n, kd=kd, **args)
    _, _, a3, g3 = _gpu_case(kind, "fp64", 3, m, n, kd=kd, **args)
    assert np.array_equal(a1, a2) and np.array_equal(a1, a3)
    assert np.array_equal(g1, g2) and np.array_equal(g1, g3)
    dev = torch.device("cuda")
    At, yt = torch.from_numpy(A).to(dev), torch.from_numpy(y).to(dev)
    if kind == SH.KRR:
        ap, _, _, _ = B.krr_solve(At, yt, kd, args["param"], args["b"], args["s"], args["H"], seed=0, prec="fp64")
        ko = oracle.kernel("rbf", gamma=0.3)
        want = oracle.sstep_bdcd_krr(A, y, ko, args["param"], args["b"], args["s"], args["H"], seed=0)
    else:
        ap, _, _, _ = B.svm_solve(At, yt, kd, 1, args["param"], args["s"], args["H"], seed=0, prec="fp64")
        ko = oracle.kernel("rbf", gamma=0.3)
        want = oracle.sstep_dcd_svm(A, y, ko, 1, args["param"], args["s"], args["H"], seed=0)
    ap = ap.cpu().numpy()
    scale = max(1.0, np.max(np.abs(want)))
    assert np.max(np.abs(a1 - ap)) <= 1e-12 * scale
    assert np.max(np.abs(a1 - want)) <= 1e-10 * scale


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["bf16x3", "bf16"])
def test_gpu_sharded_tensor_core_step_matches_the_plan(prec):
    from paper_2406_18001_gb300 import binding as B
    m, n = 3000, 64
    kd = B.kernel("rbf", gamma=0.25)
    args = dict(b=16, s=8, H=64, param=1e-3)
    A, y, a2, _ = _gpu_case(SH.KRR, prec, 2, m, n, kd=kd, **args)
    dev = torch.device("cuda")
    At, yt = torch.from_numpy(A).to(dev), torch.from_numpy(y).to(dev)
    ap, _, _, _ = B.krr_solve(At, yt, kd, args["param"], args["b"], args["s"], args["H"], seed=0, prec=prec)
    ap = ap.cpu().numpy()
    ko = oracle.kernel("rbf", gamma=0.25)
    want = oracle.sstep_bdcd_krr(A, y, ko, args["param"], args["b"], args["s"], args["H"], seed=0)
    tol = 1e-4 if prec == "bf16x3" else 1e-2
    err_plan = np.linalg.norm(a2 - ap) / np.linalg.norm(ap)
    err_oracle = np.linalg.norm(a2 - want) / np.linalg.norm(want)
    assert err_plan <= tol and err_oracle <= tol, (err_plan, err_oracle)


@pytest.mark.gpu
def test_gpu_assemble_rejects_rows_claimed_twice_or_not_at_all():
    from paper_2406_18001_gb300 import binding as B
    dev = torch.device("cuda")
    cnt, n = 3, 5
    S = torch.tensor([4, 9, 4], dtype=torch.int32, device=dev)
    buf = torch.zeros((2, cnt, n + 4), dtype=torch.float64, device=dev)
    buf[0, :, 0] = 1.0
    buf[1, 1, 0] = 1.0  # position 1 claimed by both ranks; 0 and 2 by rank 0 only
    out = [torch.empty((cnt, n), dtype=torch.float64, device=dev)] + [
        torch.empty(cnt, dtype=torch.float64, device=dev) for _ in range(3)]
    with pytest.raises(B.DcdError) as e:
        B.shard_assemble(buf, 2, S, n, *out)
    assert e.value.status == B.EINVAL
    buf[1, 1, 0] = 0.0
    first = torch.empty(cnt, dtype=torch.int32, device=dev)
    B.shard_assemble(buf, 2, S, n, *out, first_pos=first)
    assert first.cpu().tolist() == [0, 1, 0]
    buf[0, 2, 0] = 0.0  # position 2 claimed by no rank
    with pytest.raises(B.DcdError):
        B.shard_assemble(buf, 2, S, n, *out)
