"""Row-sharded outer steps: the multi-GPU layout of s-step (B)DCD.

The rows of A -- and of y, alpha and the cached gradient g -- are split over
ranks: rank p holds rows [row0_p, row0_p + m_p).  One outer step (Algorithm 2
for K-SVM, Algorithm 4 for K-RR) then needs one exchange:

  1. every rank draws the same sample S (the counter-based stream depends on
     the seed and the iteration number only);
  2. the owner of each sampled row contributes it, with g, alpha and y there;
     one all-gather gives every rank all of them (s*b*(n + 4) words per rank,
     independent of m);
  3. every rank forms the sampled Gram and runs the recurrence -- redundantly,
     as the paper's ranks repeat the s-step recurrence (Section 4);
  4. every rank applies the kernel block of its own rows to the step's
     coefficients (g_i += sum_j K(a_i, a_{S_j}) w_j, the gradient form of the
     alpha update) and updates alpha and g at the sampled rows it owns.

The paper's own layout splits the columns (features) of A instead and
all-reduces the m x s*b block every outer step (Section 4, Theorem 2); with
m >> n the row split moves far fewer words.  Every number a rank computes for
its rows is the single-rank number: the Gram and the recurrence see the same
inputs on every rank, and a row's kernel-block sum does not depend on the
other rows.

The arithmetic lives in `ops`: `CudaShardOps` runs each piece through the
library's C ABI on this rank's GPU; a test may pass its own implementation of
the same methods.  The all-gather lives in `exchange`: `DistExchange` uses a
torch.distributed process group (NCCL between GPUs); `run_local` emulates
several ranks in one process, one rank after another.
"""
from __future__ import annotations

from dataclasses import dataclass

from . import binding as B

KRR, SVM = "krr", "svm"


class CudaShardOps:
    """The pieces of a sharded outer step through the C ABI (device tensors)."""

    def __init__(self, prec="fp64"):
        self.prec = prec

    def sample(self, problem, seed, m, b, first, count, device):
        return B.sample_indices(1 if problem == KRR else 0, seed, m, b, first, count, device=device)

    def contribute(self, A, row0, m, S, g, alpha, y):
        import torch
        buf = torch.empty((S.numel(), A.shape[1] + 4), dtype=torch.float64, device=A.device)
        return B.shard_contribute(A, row0, m, S, g, alpha, y, buf)

    def assemble(self, gathered, nranks, S, n):
        import torch
        cnt, dev = S.numel(), S.device
        A_S = torch.empty((cnt, n), dtype=torch.float64, device=dev)
        g_S, a_S, y_S = (torch.empty(cnt, dtype=torch.float64, device=dev) for _ in range(3))
        first = torch.empty(cnt, dtype=torch.int32, device=dev)
        B.shard_assemble(gathered, nranks, S, n, A_S, g_S, a_S, y_S, first)
        return A_S, g_S, a_S, y_S, first

    def gram(self, A_S, first, k):
        return B.kernel_block(A_S, k, self.prec, first, rows=first)

    def krr_recurrence(self, Kss, S, b, lam, m, g_S):
        import torch
        delta = torch.empty(S.numel(), dtype=torch.float64, device=S.device)
        w = torch.empty_like(delta)
        B.bdcd_recurrence(Kss, S, b, lam, float(m), g_S, delta, w)
        return delta, w

    def svm_recurrence(self, Kss, S, y_S, a_S, g_S, loss, C_):
        import torch
        theta = torch.empty(S.numel(), dtype=torch.float64, device=S.device)
        w = torch.empty_like(theta)
        B.dcd_recurrence(Kss, S, y_S, a_S, g_S, loss, C_, theta, w)
        return theta, w

    def apply(self, A, row0, A_S, S, k, w, rowscale, g):
        B.kernel_block_apply_points(A, row0, A_S, S, k, self.prec, w, g, rowscale=rowscale)

    def update(self, S, delta, diag, row0, alpha, g):
        B.shard_update(S, delta, diag, row0, alpha, g)


@dataclass
class ShardSpec:
    problem: str          # KRR or SVM
    m: int                # rows of the whole problem
    b: int                # block size (1 for K-SVM)
    s: int                # blocks (coordinates) per outer step
    H: int                # iterations in all: blocks (K-RR) or coordinates (K-SVM)
    param: float          # lambda (K-RR) or C (K-SVM)
    loss: int = 1         # K-SVM: 1 hinge, 2 squared hinge
    seed: int = 0


class RowShard:
    """One rank's rows [row0, row0 + A.shape[0]) of a K-RR or K-SVM problem,
    solved from alpha = 0 (g = -y for K-RR, g = -1 for K-SVM) by row-sharded
    outer steps.  `alpha` and `g` are this rank's parts."""

    def __init__(self, ops, spec: ShardSpec, A, y, row0, k):
        import torch
        self.ops, self.spec, self.A, self.y, self.row0, self.k = ops, spec, A, y, int(row0), k
        if spec.problem not in (KRR, SVM):
            raise ValueError("problem must be 'krr' or 'svm'")
        if spec.problem == SVM and spec.b != 1:
            raise ValueError("K-SVM samples single coordinates (b = 1)")
        self.alpha = torch.zeros(A.shape[0], dtype=torch.float64, device=A.device)
        self.g = -y.to(torch.float64).clone() if spec.problem == KRR else -torch.ones_like(self.alpha)
        self.diag = float(spec.m) if spec.problem == KRR else (0.5 / spec.param if spec.loss == 2 else 0.0)
        self.done = 0
        self._S = None

    def steps(self):
        """Outer steps in the whole solve (the last one shorter when s does not divide H)."""
        return -(-self.spec.H // self.spec.s)

    def contribute(self):
        """Phase 1 of the next outer step: the sample and this rank's buffer."""
        sp = self.spec
        cnt = min(sp.s, sp.H - self.done)
        self._S = self.ops.sample(sp.problem, sp.seed, sp.m, sp.b, self.done, cnt, self.A.device)
        return self.ops.contribute(self.A, self.row0, sp.m, self._S, self.g, self.alpha, self.y)

    def finish(self, gathered, nranks):
        """Phase 2: Gram, recurrence, kernel block on this rank's rows, update."""
        sp, S = self.spec, self._S
        A_S, g_S, a_S, y_S, first = self.ops.assemble(gathered, nranks, S, self.A.shape[1])
        Kss = self.ops.gram(A_S, first, self.k)
        if sp.problem == KRR:
            delta, w = self.ops.krr_recurrence(Kss, S, sp.b, sp.param, sp.m, g_S)
            self.ops.apply(self.A, self.row0, A_S, S, self.k, w, None, self.g)
        else:
            delta, w = self.ops.svm_recurrence(Kss, S, y_S, a_S, g_S, sp.loss, sp.param)
            self.ops.apply(self.A, self.row0, A_S, S, self.k, w, self.y, self.g)
        self.ops.update(S, delta, self.diag, self.row0, self.alpha, self.g)
        self.done += S.numel() // sp.b
        self._S = None


class DistExchange:
    """All-gather over a torch.distributed process group (every rank's buffer
    has the same shape: one row per sampled position)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist, self.group = dist, group
        self.size = dist.get_world_size(group)

    def all_gather(self, buf):
        import torch
        parts = [torch.empty_like(buf) for _ in range(self.size)]
        self.dist.all_gather(parts, buf.contiguous(), group=self.group)
        return torch.cat(parts, 0)


def run_dist(shard: RowShard, exchange: DistExchange, steps=None):
    """This rank's part of the row-sharded solve (every rank calls it)."""
    n = shard.steps() if steps is None else steps
    for _ in range(n):
        if shard.done >= shard.spec.H:
            break
        gathered = exchange.all_gather(shard.contribute())
        shard.finish(gathered, exchange.size)
    return shard


def run_local(shards, steps=None):
    """Several ranks emulated in one process: each outer step runs phase 1 on
    every shard, concatenates the buffers in rank order (the all-gather) and
    runs phase 2 on every shard."""
    import torch
    n = shards[0].steps() if steps is None else steps
    for _ in range(n):
        if shards[0].done >= shards[0].spec.H:
            break
        gathered = torch.cat([sh.contribute() for sh in shards], 0)
        for sh in shards:
            sh.finish(gathered, len(shards))
    return shards


def split_rows(m, nranks):
    """Contiguous row ranges [(row0, rows)] of nearly equal size, in rank order."""
    base, extra = divmod(int(m), int(nranks))
    out, r0 = [], 0
    for p in range(nranks):
        cnt = base + (1 if p < extra else 0)
        out.append((r0, cnt))
        r0 += cnt
    return out
