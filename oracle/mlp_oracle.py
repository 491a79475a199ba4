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
