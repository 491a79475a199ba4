"""CPU reference of the planner's cost model (test infrastructure only).

A 3-layer perceptron of width 64, h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2),
y = h2 W3 + b3, with the mean squared error loss and its gradient, in float64 numpy,
written from the definitions (chain rule). Parameters are one flat vector in the layout
W1 (d x 64) | b1 | W2 (64 x 64) | b2 | W3 (64) | b3, the layout of the CUDA kernels.
"""
import numpy as np

H = 64


def unpack(p, d):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + d * H].reshape(d, H); o += d * H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def forward(x, p):
    x = np.asarray(x, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p, x.shape[1])
    z1 = x @ W1 + b1
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    y = h2 @ W3 + b3
    return y, (x, z1, h1, z2, h2)


def loss(x, t, p):
    y, _ = forward(x, p)
    return float(np.mean((y - np.asarray(t, dtype=np.float64)) ** 2))


def gradient(x, t, p):
    """d loss / d p for loss = mean((y - t)^2)."""
    y, (x, z1, h1, z2, h2) = forward(x, p)
    n, d = x.shape
    W1, b1, W2, b2, W3, b3 = unpack(p, d)
    gy = 2.0 * (y - np.asarray(t, dtype=np.float64)) / n
    gW3 = h2.T @ gy
    gb3 = gy.sum()
    dz2 = np.outer(gy, W3) * (z2 > 0)
    gW2 = h1.T @ dz2
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    gW1 = x.T @ dz1
    gb1 = dz1.sum(axis=0)
    return np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, "Adam: A Method for Stochastic Optimization", 2015,
    Algorithm 1): exponential moving averages of the gradient and of its square, bias
    correction by 1 - beta^step, and p - lr * m_hat / (sqrt(v_hat) + eps). Returns the new
    (p, m, v) in float64."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
