"""dcd_kernel_block_static (no device allocation) against dcd_kernel_block.

The static entry point is for callers that cannot allocate device memory
when they need a kernel block -- a framework that has reserved the device
memory for its own caching pool, or a deployment that forbids allocation
after start-up.  It keeps its scratch in one library-owned device array, so
it must produce the same block as the allocating entry point, call after
call, while that array is reused.  Both entry points run the same pack,
norm and block kernels with the same arguments, so the blocks are compared
bit for bit.  This file is collected last: if it fails, a run that stops at
the first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16", "bf16x3", "fp64"])
def test_static_scratch_matches_allocating_entry_point(prec):
    from paper_2406_18001_gb300 import binding as B
    g = np.random.default_rng(11)
    k = B.kernel("rbf", gamma=0.3)
    dt = np.float64 if prec == "fp64" else np.float32
    # the start-up call a caller that must not allocate later makes: an empty
    # request, which looks up (and makes resident) the scratch array
    A0 = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    c0 = torch.zeros(2, dtype=torch.int32, device="cuda")
    o0 = torch.full((1, 2), -7.0, device="cuda", dtype=torch.float64 if prec == "fp64" else torch.float32)
    B.kernel_block_static(A0, k, prec, c0, nrows=0, out=o0)
    assert torch.all(o0 == -7.0)  # nothing written
    # two calls in a row with different shapes: the second reuses (and must
    # not be disturbed by) what the first left in the shared scratch array
    for m, n, nc, nr in ((300, 77, 70, 133), (517, 40, 103, 260)):
        A = torch.from_numpy((g.standard_normal((m, n)) * 0.2).astype(dt)).cuda()
        cols = torch.from_numpy(g.integers(0, m, size=nc).astype(np.int32)).cuda()
        rows = torch.from_numpy(g.integers(0, m, size=nr).astype(np.int32)).cuda()
        want = B.kernel_block(A, k, prec, cols, rows=rows).cpu().numpy()
        got = B.kernel_block_static(A, k, prec, cols, rows=rows).cpu().numpy()
        assert got.shape == want.shape
        assert np.array_equal(got, want)


def test_static_scratch_rejects_requests_beyond_its_size():
    from paper_2406_18001_gb300 import binding as B
    # 40000 bf16 rows of 512 features need ~41 MB of scratch > 32 MiB
    A = torch.zeros((40000, 512), dtype=torch.float32, device="cuda")
    cols = torch.arange(8, dtype=torch.int32, device="cuda")
    with pytest.raises(B.DcdError) as e:
        B.kernel_block_static(A, B.kernel("linear"), "bf16", cols)
    assert e.value.status == B.EINVAL


def test_static_scratch_checks_arguments_as_the_allocating_entry_point():
    from paper_2406_18001_gb300 import binding as B
    A = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    cols = torch.arange(3, dtype=torch.int32, device="cuda")
    bad = B.kernel("poly", coef0=float("inf"), degree=3)
    for fn in (B.kernel_block, B.kernel_block_static):
        with pytest.raises(B.DcdError) as e:
            fn(A, bad, "bf16", cols)
        assert e.value.status == B.EINVAL
