"""Failure paths, tested without faulting, trapping or hanging a GPU.

A bounded device wait that runs out must come back as DCD_ETIMEOUT with the
stream still usable; a device allocation that fails (injected on the host)
must come back as DCD_ENOMEM, and the next call must work again.
"""
import numpy as np
import pytest

from paper_2406_18001_gb300 import inputs

torch = pytest.importorskip("torch")


def B():
    from paper_2406_18001_gb300 import binding
    return binding


def test_injection_hook_argument_checks():
    assert B().lib().dcd_inject_alloc_failures(-1) == B().EINVAL
    assert B().lib().dcd_inject_alloc_failures(0) == B().OK
    assert B().lib().dcd_selftest_bounded_wait(10, None) == B().EINVAL  # below 1 us


@pytest.mark.gpu
def test_bounded_wait_gives_up_and_reports_a_timeout():
    assert B().selftest_bounded_wait(1_000_000) == B().ETIMEOUT  # ~1 ms bound
    # the context and stream stay usable: a solve right after it succeeds
    p = inputs.krr_dense(m=200, n=8, seed=1, dtype=np.float64)
    al, _, st, rc = B().krr_solve(torch.from_numpy(p.A).cuda(), torch.from_numpy(p.y).cuda(),
                                  B().kernel("rbf", gamma=0.5), 0.05, 4, 4, 40, prec="fp64")
    assert rc == B().OK and np.all(np.isfinite(al.cpu().numpy()))


@pytest.mark.gpu
def test_allocation_failure_reports_enomem_then_recovers():
    p = inputs.krr_dense(m=200, n=8, seed=2, dtype=np.float32)
    A, y = torch.from_numpy(p.A).cuda(), torch.from_numpy(p.y).cuda()
    k = B().kernel("rbf", gamma=0.5)
    B().inject_alloc_failures(1)
    with pytest.raises(B().DcdError) as e:
        B().krr_solve(A, y, k, 0.05, 4, 4, 40, prec="bf16x3")
    assert e.value.status == B().ENOMEM
    al, _, st, rc = B().krr_solve(A, y, k, 0.05, 4, 4, 40, prec="bf16x3")
    assert rc == B().OK
    B().inject_alloc_failures(1)
    with pytest.raises(B().DcdError) as e:
        B().kernel_block(A, k, "bf16", torch.arange(8, dtype=torch.int32, device="cuda"))
    assert e.value.status == B().ENOMEM
    B().inject_alloc_failures(0)
