"""The planner's cost model: CPU reference pinned by finite differences; GPU forward,
backward and Adam kernels against the CPU reference."""
import numpy as np
import pytest

from oracle import mlp_oracle as M


def random_problem(seed, n=12, d=7):
    r = np.random.default_rng(seed)
    x = r.standard_normal((n, d))
    t = r.standard_normal(n)
    npar = d * 64 + 64 + 64 * 64 + 64 + 64 + 1
    p = r.standard_normal(npar) * 0.3
    return x, t, p


@pytest.mark.parametrize("seed", range(3))
def test_reference_gradient_matches_finite_differences(seed):
    x, t, p = random_problem(seed)
    g = M.gradient(x, t, p)
    r = np.random.default_rng(100 + seed)
    idx = r.choice(len(p), 60, replace=False)
    eps = 1e-6
    for i in idx:
        e = np.zeros_like(p)
        e[i] = eps
        fd = (M.loss(x, t, p + e) - M.loss(x, t, p - e)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


@pytest.mark.gpu
def test_gpu_forward_backward_match_reference():
    import torch
    from paper_2008_08657_b300.lmfao import CostModel
    x, t, p = random_problem(7, n=300, d=19)
    m = CostModel(19)
    m.params.copy_(torch.tensor(p, dtype=torch.float32))
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    y, h1, h2 = m.forward(xt, keep=True)
    yref, _ = M.forward(x.astype(np.float32).astype(np.float64), p.astype(np.float32).astype(np.float64))
    np.testing.assert_allclose(y.cpu().numpy(), yref, rtol=1e-4, atol=1e-4 * np.abs(yref).max())
    gy = torch.tensor(2.0 * (yref - t) / len(t), dtype=torch.float32, device="cuda")
    g = m.backward(xt, h1, h2, gy).cpu().numpy()
    gref = M.gradient(x.astype(np.float32).astype(np.float64), t, p.astype(np.float32).astype(np.float64))
    scale = np.abs(gref).max()
    np.testing.assert_allclose(g, gref, rtol=1e-3, atol=2e-4 * scale)


@pytest.mark.gpu
def test_gpu_training_reduces_loss_and_overfits_small_set():
    import torch
    from paper_2008_08657_b300.lmfao import CostModel
    r = np.random.default_rng(3)
    x = r.standard_normal((64, 10))
    t = np.sin(x[:, 0]) + 0.5 * x[:, 1] ** 2
    m = CostModel(10, seed=1)
    xt = torch.tensor(x, dtype=torch.float32, device="cuda")
    tt = torch.tensor(t, dtype=torch.float32, device="cuda")
    first = float(m.train_step(xt, tt, lr=3e-3).item())
    for _ in range(1500):
        last = m.train_step(xt, tt, lr=3e-3)
    last = float(last.item())
    assert last < 0.05 * first and last < 0.02
