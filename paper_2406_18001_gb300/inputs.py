"""Seeded synthetic inputs for the s-step DCD / BDCD solvers.

This module only draws data: it holds none of the solvers' arithmetic (no
kernel function, no coordinate sampling, no update rule).  Both the CUDA
path's tests and the FP64 oracle take their inputs from here, so the two
sides see bit-identical matrices.  Every generator is a pure function of its
seed (numpy's PCG64 stream), independent of the machine it runs on.

The workloads mirror the shapes of the paper's experiments (Section 5): dense
blobs for K-SVM, a dense Gaussian regression matrix for K-RR, a uniformly
sparse CSR matrix like the paper's synthetic 2000 x 800000 set (Table of
performance datasets, Section 5.2), a sweep of uneven problems, and an
ill-conditioned dense matrix.  The LIBSVM sets the paper uses are not
available; these synthetic matrices stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int, stream: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([int(seed) & 0xFFFFFFFF, int(stream)]))


@dataclass
class DenseProblem:
    A: np.ndarray          # (m, n) row-major
    y: np.ndarray          # (m,) float64: +-1 labels or regression targets
    meta: dict = field(default_factory=dict)


@dataclass
class CsrProblem:
    row_ptr: np.ndarray    # (m+1,) int64
    col_idx: np.ndarray    # (nnz,) int32, sorted within each row
    values: np.ndarray     # (nnz,) float32
    n: int
    y: np.ndarray          # (m,) float64 labels
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return self.row_ptr.shape[0] - 1

    def to_dense(self, dtype=np.float64) -> np.ndarray:
        out = np.zeros((self.m, self.n), dtype=dtype)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        out[rows, self.col_idx] = self.values
        return out


def blobs(m: int = 2000, n: int = 64, seed: int = 0, dtype=np.float64) -> DenseProblem:
    """Two Gaussian blobs (means +-0.5 in every coordinate, unit variance).

    The first half of the rows is labelled +1 and centred at +0.5, the second
    half -1 at -0.5; rows are then shuffled by the seed.
    """
    g = _rng(seed, 1)
    half = m // 2
    y = np.empty(m)
    y[:half] = 1.0
    y[half:] = -1.0
    A = g.standard_normal((m, n)) + 0.5 * y[:, None]
    perm = g.permutation(m)
    return DenseProblem(A[perm].astype(dtype), y[perm].copy(), {"kind": "blobs", "m": m, "n": n, "seed": seed})


def krr_dense(m: int = 50000, n: int = 512, seed: int = 0, noise: float = 0.1,
              dtype=np.float32) -> DenseProblem:
    """A ~ N(0,1)/sqrt(n); y = sin(A w) + noise * N(0,1) with w ~ N(0, I)."""
    g = _rng(seed, 2)
    A = (g.standard_normal((m, n), dtype=np.float32) / np.float32(np.sqrt(n))).astype(np.float32)
    w = g.standard_normal(n)
    y = np.sin(A.astype(np.float64) @ w) + noise * g.standard_normal(m)
    return DenseProblem(A.astype(dtype), y, {"kind": "krr_dense", "m": m, "n": n, "seed": seed})


def sparse_csr(m: int = 200000, n: int = 50000, nnz_per_row: int = 50, seed: int = 0,
               w_density: float = 0.01, flip: float = 0.05) -> CsrProblem:
    """Uniformly sparse rows (nnz_per_row distinct random columns, values
    U(0,1), each row scaled to unit 2-norm); labels are the sign of a_i.w for
    a sparse Gaussian w (sign(0) = +1), with a fraction `flip` flipped."""
    g = _rng(seed, 3)
    k = int(nnz_per_row)
    if k > n:
        raise ValueError("nnz_per_row > n")
    cols = np.sort(g.integers(0, n, size=(m, k), dtype=np.int64), axis=1)
    while True:  # redraw rows with repeated columns until every row is distinct
        dup = np.any(cols[:, 1:] == cols[:, :-1], axis=1) if k > 1 else np.zeros(m, bool)
        bad = np.nonzero(dup)[0]
        if bad.size == 0:
            break
        cols[bad] = np.sort(g.integers(0, n, size=(bad.size, k), dtype=np.int64), axis=1)
    vals = g.random((m, k))
    vals /= np.linalg.norm(vals, axis=1, keepdims=True)
    vals = vals.astype(np.float32)
    w = np.zeros(n)
    nw = max(1, int(round(w_density * n)))
    w[g.choice(n, nw, replace=False)] = g.standard_normal(nw)
    score = np.sum(vals.astype(np.float64) * w[cols], axis=1)
    y = np.where(score >= 0, 1.0, -1.0)
    nflip = int(round(flip * m))
    y[g.choice(m, nflip, replace=False)] *= -1.0
    row_ptr = np.arange(0, (m + 1) * k, k, dtype=np.int64)
    return CsrProblem(row_ptr, cols.reshape(-1).astype(np.int32), vals.reshape(-1), n, y,
                      {"kind": "sparse_csr", "m": m, "n": n, "nnz_per_row": k, "seed": seed})


def sweep_problem(p: int, n: int = 128, m_lo: int = 1000, m_hi: int = 20000,
                  dtype=np.float32) -> DenseProblem:
    """Problem p of the batched K-RR sweep: m_p ~ U{m_lo..m_hi} drawn from
    seed p, A ~ N(0,1) (m_p x n), y ~ N(0,1)."""
    g = _rng(p, 4)
    mp = int(g.integers(m_lo, m_hi + 1))
    A = g.standard_normal((mp, n), dtype=np.float32).astype(dtype)
    y = g.standard_normal(mp)
    return DenseProblem(A, y, {"kind": "sweep", "p": p, "m": mp, "n": n})


def sweep_grid(count: int = 256, sig_lo: float = 0.1, sig_hi: float = 10.0,
               lam_lo: float = 1e-6, lam_hi: float = 1e-1):
    """(sigma, lambda) pairs on a log x log grid, one pair per problem."""
    side = int(round(np.sqrt(count)))
    sig = np.logspace(np.log10(sig_lo), np.log10(sig_hi), side)
    lam = np.logspace(np.log10(lam_lo), np.log10(lam_hi), side)
    pairs = [(float(s), float(l)) for s in sig for l in lam]
    return pairs[:count]


def ill_conditioned_mixer(n: int, seed: int = 0, cond: float = 1e4, row_norm2: float = 64.0) -> np.ndarray:
    """The n x n factor diag(sig) W^T of ill_conditioned (float32): rows of
    A are z^T diag(sig) W^T with z ~ N(0, I)."""
    gw = _rng(seed, 5)
    W, _ = np.linalg.qr(gw.standard_normal((n, n)))
    sig = np.logspace(-np.log10(cond), 0.0, n)
    sig *= np.sqrt(row_norm2 / np.sum(sig ** 2))
    return (sig[:, None] * W.T).astype(np.float32)


def ill_conditioned(m: int, n: int, seed: int = 0, cond: float = 1e4, row_norm2: float = 64.0,
                    dtype=np.float32, row_start: int = 0, chunk: int = 65536) -> np.ndarray:
    """A = Z diag(sig) W^T with Z ~ N(0,1), W a seeded random orthogonal n x n
    matrix and sig log-spaced over [1/cond, 1] * c, where c makes the expected
    squared row norm equal to row_norm2.  Rows are drawn in fixed chunks from
    per-chunk streams, so any row range is reproducible on its own."""
    B = ill_conditioned_mixer(n, seed, cond, row_norm2)
    out = np.empty((m, n), dtype=dtype)
    r = 0
    while r < m:
        gi = (row_start + r) // chunk
        off = (row_start + r) % chunk
        take = min(chunk - off, m - r)
        gz = _rng(seed, 1000 + gi)
        Z = gz.standard_normal((chunk, n), dtype=np.float32)[off:off + take]
        out[r:r + take] = (Z @ B).astype(dtype)
        r += take
    return out


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round float32 values to bfloat16 (nearest even) and return the 16-bit
    patterns as uint16 (storage conversion only)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16).astype(np.uint16)
    nan = np.isnan(x)
    if np.any(nan):
        r[nan] = 0x7FC0
    return r


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (b.astype(np.uint32) << 16).view(np.float32)
