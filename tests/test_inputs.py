"""The seeded input recipes hold the shapes and statistics the workloads are
stated with: determinism per seed, the blobs' halves and means, the K-RR
targets, the CSR pattern (distinct columns, unit rows, labels with the
stated flip fraction), the sweep's sizes and log grid, the ill-conditioned
matrix's spectrum and row norms (chunk-independent), and bf16 rounding."""
import os
import sys

import numpy as np
import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_2406_18001_gb300 import inputs  # noqa: E402


def test_every_recipe_is_a_function_of_its_seed():
    a, b = inputs.blobs(m=50, n=4, seed=3), inputs.blobs(m=50, n=4, seed=3)
    assert np.array_equal(a.A, b.A) and np.array_equal(a.y, b.y)
    assert not np.array_equal(a.A, inputs.blobs(m=50, n=4, seed=4).A)
    c, d = inputs.sparse_csr(m=40, n=100, nnz_per_row=5, seed=2), inputs.sparse_csr(m=40, n=100, nnz_per_row=5, seed=2)
    assert np.array_equal(c.col_idx, d.col_idx) and np.array_equal(c.values, d.values)


def test_blobs_halves_and_means():
    p = inputs.blobs(m=4000, n=8, seed=1)
    assert p.A.shape == (4000, 8) and np.sum(p.y == 1) == 2000 and np.sum(p.y == -1) == 2000
    for lab, mu in ((1.0, 0.5), (-1.0, -0.5)):
        rows = p.A[p.y == lab]
        assert np.all(np.abs(rows.mean(axis=0) - mu) < 5 / np.sqrt(2000))  # 5 standard errors
        assert np.all(np.abs(rows.std(axis=0) - 1.0) < 0.1)
    assert not np.all(p.y[:2000] == 1)  # shuffled


def test_krr_dense_scale_and_targets():
    p = inputs.krr_dense(m=3000, n=64, seed=0)
    assert p.A.dtype == np.float32 and p.A.shape == (3000, 64)
    assert abs(np.mean(np.sum(p.A.astype(np.float64) ** 2, axis=1)) - 1.0) < 0.02  # N(0,1)/sqrt(n) rows
    assert np.all(np.abs(p.y) < 1.0 + 6 * 0.1)  # sin(.) + 0.1 N(0,1)


def test_sparse_csr_pattern_norms_and_labels():
    m, n, k = 2000, 500, 20
    p = inputs.sparse_csr(m=m, n=n, nnz_per_row=k, seed=5, flip=0.05)
    assert np.array_equal(p.row_ptr, np.arange(0, (m + 1) * k, k))
    cols = p.col_idx.reshape(m, k)
    assert np.all(np.diff(cols, axis=1) > 0) and cols.min() >= 0 and cols.max() < n  # distinct, sorted
    vals = p.values.reshape(m, k).astype(np.float64)
    assert np.all(vals > 0) and np.allclose(np.linalg.norm(vals, axis=1), 1.0, atol=1e-6)
    assert set(np.unique(p.y)) <= {-1.0, 1.0}
    dense = p.to_dense()
    assert np.array_equal(np.count_nonzero(dense, axis=1), np.full(m, k))


def test_sparse_csr_flip_fraction():
    a = inputs.sparse_csr(m=1000, n=300, nnz_per_row=10, seed=9, flip=0.0)
    b = inputs.sparse_csr(m=1000, n=300, nnz_per_row=10, seed=9, flip=0.05)
    assert np.array_equal(a.col_idx, b.col_idx)
    assert np.sum(a.y != b.y) == 50


def test_sweep_sizes_and_grid():
    ms = [inputs.sweep_problem(p, n=16).A.shape[0] for p in range(64)]
    assert min(ms) >= 1000 and max(ms) <= 20000 and len(set(ms)) > 50
    grid = inputs.sweep_grid()
    assert len(grid) == 256 and len(set(grid)) == 256
    sig = sorted({s for s, _ in grid})
    lam = sorted({l for _, l in grid})
    assert len(sig) == 16 and len(lam) == 16
    assert sig[0] == pytest.approx(0.1) and sig[-1] == pytest.approx(10.0)
    assert lam[0] == pytest.approx(1e-6) and lam[-1] == pytest.approx(1e-1)
    assert np.allclose(np.diff(np.log(sig)), np.log(sig[1] / sig[0]))  # log-spaced


def test_ill_conditioned_spectrum_and_row_norms():
    n, cond = 32, 1e4
    B = inputs.ill_conditioned_mixer(n, seed=1, cond=cond, row_norm2=64.0).astype(np.float64)
    sv = np.linalg.svd(B, compute_uv=False)
    assert sv.max() / sv.min() == pytest.approx(cond, rel=1e-3)
    assert np.sum(sv ** 2) == pytest.approx(64.0, rel=1e-5)  # E ||a||^2 = ||diag(sig)||_F^2
    A = inputs.ill_conditioned(4000, n, seed=1, chunk=1000).astype(np.float64)
    assert np.mean(np.sum(A ** 2, axis=1)) == pytest.approx(64.0, rel=0.05)


def test_ill_conditioned_rows_do_not_depend_on_the_range_drawn():
    full = inputs.ill_conditioned(300, 16, seed=2, chunk=128)
    part = inputs.ill_conditioned(100, 16, seed=2, chunk=128, row_start=150)
    assert np.array_equal(full[150:250], part)


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e38, 1e-40], dtype=np.float32)
    r = inputs.bf16_bits_to_f32(inputs.to_bf16_bits(x))
    # ties go to the even mantissa: 1 + 2^-8 -> 1, 1 + 3 * 2^-8 -> 1 + 2^-6
    assert r[0] == 1.0 and r[1] == 1.0 and r[2] == np.float32(1.0 + 2.0 ** -6) and r[3] == -2.5
    # half an ulp: 2^-8 relative for normal values, 2^-134 absolute among the subnormals
    assert np.all(np.abs(r.astype(np.float64) - x) <= np.maximum(np.abs(x.astype(np.float64)) * 2.0 ** -8, 2.0 ** -134))
    assert inputs.to_bf16_bits(np.array([np.nan], dtype=np.float32))[0] == 0x7FC0
