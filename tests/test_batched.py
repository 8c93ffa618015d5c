"""Batched K-RR (bdcd_krr_solve_batched): every problem of a batch must give
exactly what a single bdcd_krr_solve with the same arguments gives, and the
autotuner's choice must be a valid s."""
import numpy as np
import pytest

import oracle
from paper_2406_18001_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def B():
    from paper_2406_18001_gb300 import binding
    return binding


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def sweep(count, seed=0, n=24, m_lo=150, m_hi=900):
    """A small sweep in the config's shape: uneven m, (sigma, lambda) on a log
    grid, b in {8, 32}."""
    g = np.random.default_rng(seed)
    side = int(np.ceil(np.sqrt(count)))
    grid = inputs.sweep_grid(side * side, sig_lo=0.3, sig_hi=3.0, lam_lo=1e-4, lam_hi=1e-1)
    probs = []
    for p in range(count):
        m = int(g.integers(m_lo, m_hi + 1))
        A = g.standard_normal((m, n)).astype(np.float32) / np.sqrt(n)
        y = g.standard_normal(m)
        sig, lam = grid[p]
        b = 8 if p % 2 == 0 else 32
        probs.append(dict(A=dev(A), y=dev(y), k=B().kernel("rbf", gamma=1.0 / (2 * sig * sig)), lam=lam, b=b,
                          H=int(g.integers(3, 12)) * 4 + 1, seed=p, A_np=A, y_np=y, gamma=1.0 / (2 * sig * sig)))
    return probs


def single(p, s, prec):
    al, gr, st, _ = B().krr_solve(p["A"], p["y"], p["k"], p["lam"], p["b"], s, p["H"], seed=p["seed"], prec=prec)
    return al, gr


@pytest.mark.parametrize("prec", ["bf16x3", "fp64"])
def test_batch_equals_single_solves(prec):
    probs = sweep(9, seed=1)
    for i, p in enumerate(probs):
        p["s"] = [1, 4, 8, 16][i % 4]
    # 3 streams, 2 outer steps per graph replay: several recaptures as budgets run out
    al, gr, st, rc = B().krr_solve_batched(probs, prec=prec, streams=3, rounds_per_graph=2)
    assert rc == B().OK
    for i, p in enumerate(probs):
        a1, g1 = single(p, p["s"], prec)
        assert st[i]["iters_done"] == p["H"] and st[i]["s_used"] == p["s"]
        assert torch.equal(al[i], a1) and torch.equal(gr[i], g1), i


def test_batch_autotuned_s_matches_single_solve_with_that_s():
    probs = sweep(4, seed=2)
    for p in probs:
        p["s"] = 0
    al, gr, st, rc = B().krr_solve_batched(probs, prec="bf16x3", streams=2)
    for i, p in enumerate(probs):
        s = int(st[i]["s_used"])
        assert s >= 1 and s & (s - 1) == 0 and s * p["b"] <= 8192
        a1, _ = single(p, s, "bf16x3")
        assert torch.equal(al[i], a1)


def test_batch_tolerance_drops_converged_problems():
    probs = sweep(6, seed=3, m_lo=150, m_hi=400)
    for p in probs:
        p["s"] = 4
        p["H"] = 200000
    al, gr, st, rc = B().krr_solve_batched(probs, prec="bf16x3", tol=1e-5, check_every=1, rounds_per_graph=4,
                                           flags=B().FLAG_REFRESH)
    assert rc == B().OK
    for i, p in enumerate(probs):
        assert st[i]["converged"] == 1 and st[i]["final_metric"] <= 1e-5
        ko = oracle.kernel("rbf", gamma=p["gamma"])
        gw = oracle.krr_gradient(p["A_np"], p["y_np"], ko, p["lam"], al[i].cpu().numpy())
        assert np.linalg.norm(gw) / np.linalg.norm(p["y_np"]) <= 2e-5


def test_batch_matches_the_oracle():
    probs = sweep(3, seed=4, m_lo=200, m_hi=300)
    for p in probs:
        p["s"] = 8
    al, _, _, _ = B().krr_solve_batched(probs, prec="fp64")
    for i, p in enumerate(probs):
        ko = oracle.kernel("rbf", gamma=p["gamma"])
        want = oracle.bdcd_krr(p["A_np"].astype(np.float64), p["y_np"], ko, p["lam"], p["b"], p["H"],
                               seed=p["seed"])
        a = al[i].cpu().numpy()
        assert np.linalg.norm(a - want) <= 1e-10 * np.linalg.norm(want)


def test_autotune_returns_a_power_of_two():
    p = sweep(1, seed=5, m_lo=2000, m_hi=2000)[0]
    s = B().krr_autotune_s(p["A"], p["y"], p["k"], p["lam"], 16)
    assert s >= 1 and s & (s - 1) == 0 and s <= 128
