"""The planner's cost model: CPU reference pinned by finite differences, by networks that
realise known functions and by Adam's closed-form first steps; GPU forward, backward and
Adam kernels against the CPU reference."""
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


def _params(d, W1=None, b1=None, W2=None, b2=None, W3=None, b3=0.0):
    H = M.H
    parts = [np.zeros((d, H)) if W1 is None else W1, np.zeros(H) if b1 is None else b1,
             np.zeros((H, H)) if W2 is None else W2, np.zeros(H) if b2 is None else b2,
             np.zeros(H) if W3 is None else W3, [b3]]
    return np.concatenate([np.ravel(a) for a in parts])


def test_reference_forward_realises_known_functions():
    """Networks whose weights realise a known function of x: sum of ReLUs of the inputs
    (first layer copies x and -x, so relu(x) + relu(-x) = |x|), the output bias alone, and a
    hidden bias that reaches the output only through the ReLU. A dropped bias, a transposed
    weight matrix or a missing ReLU fails one of them."""
    d, H = 3, M.H
    r = np.random.default_rng(0)
    x = r.standard_normal((20, d))
    # |x_0| + 2 |x_1| + 3 |x_2| + 0.5
    W1 = np.zeros((d, H))
    for i in range(d):
        W1[i, i] = 1.0
        W1[i, d + i] = -1.0
    W2 = np.eye(H)
    W3 = np.zeros(H)
    for i in range(d):
        W3[i] = W3[d + i] = i + 1.0
    y, _ = M.forward(x, _params(d, W1=W1, W2=W2, W3=W3, b3=0.5))
    np.testing.assert_allclose(y, np.abs(x) @ np.array([1.0, 2.0, 3.0]) + 0.5, rtol=1e-12)
    # zero weights: the output is b3 whatever x is
    y, _ = M.forward(x, _params(d, b3=-1.25))
    np.testing.assert_array_equal(y, np.full(len(x), -1.25))
    # hidden biases only: y = relu(b2) . W3 + b3 (negative b2 entries are cut by the ReLU)
    b2 = np.linspace(-1.0, 1.0, H)
    W3 = np.ones(H)
    y, _ = M.forward(x, _params(d, b2=b2, W3=W3, b3=0.0))
    np.testing.assert_allclose(y, np.full(len(x), np.maximum(b2, 0).sum()), rtol=1e-12)
    # layer-1 bias: relu(x_0 + 1) through W2 = identity and W3 = e_0
    W1 = np.zeros((d, H))
    W1[0, 0] = 1.0
    b1 = np.zeros(H)
    b1[0] = 1.0
    W3 = np.zeros(H)
    W3[0] = 1.0
    y, _ = M.forward(x, _params(d, W1=W1, b1=b1, W2=np.eye(H), W3=W3))
    np.testing.assert_allclose(y, np.maximum(x[:, 0] + 1.0, 0.0), rtol=1e-12)


def test_reference_adam_first_steps_have_closed_forms():
    """From m = v = 0 the bias-corrected first step is lr * g / (|g| + eps), i.e. lr * sign(g);
    under a constant gradient every later step is the same; a zero gradient moves nothing."""
    g = np.array([3.0, -0.5, 1e-3, 0.0, -7.0])
    p0 = np.array([1.0, 2.0, -3.0, 4.0, 0.0])
    m = v = np.zeros_like(g)
    p, lr = p0, 0.01
    for step in range(1, 6):
        p, m, v = M.adam_step(p, g, m, v, step, lr)
        want = p0 - lr * step * g / (np.abs(g) + 1e-8)
        np.testing.assert_allclose(p, want, rtol=1e-9, atol=1e-12)
    assert p[3] == p0[3]


@pytest.mark.gpu
def test_gpu_adam_matches_reference():
    import torch
    from paper_2008_08657_b300.lmfao import library
    lib = library()
    r = np.random.default_rng(5)
    n = 5000
    p = r.standard_normal(n)
    m = np.zeros(n)
    v = np.zeros(n)
    tp = torch.tensor(p, dtype=torch.float32, device="cuda")
    tm = torch.zeros(n, dtype=torch.float32, device="cuda")
    tv = torch.zeros(n, dtype=torch.float32, device="cuda")
    import ctypes
    for step in range(1, 8):
        g = r.standard_normal(n) * (10.0 ** r.uniform(-3, 1, n))
        tg = torch.tensor(g, dtype=torch.float32, device="cuda")
        rc = lib.lmfao_mlp_adam(ctypes.c_void_p(tp.data_ptr()), ctypes.c_void_p(tg.data_ptr()),
                                ctypes.c_void_p(tm.data_ptr()), ctypes.c_void_p(tv.data_ptr()),
                                ctypes.c_int64(n), step, ctypes.c_float(1e-2), None)
        assert rc == 0
        p, m, v = M.adam_step(p, g.astype(np.float32).astype(np.float64), m, v, step, 1e-2)
    torch.cuda.synchronize()
    np.testing.assert_allclose(tp.cpu().numpy(), p, rtol=1e-5, atol=1e-5)
    np.testing.assert_allclose(tm.cpu().numpy(), m, rtol=1e-4, atol=1e-6 * np.abs(m).max())


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
