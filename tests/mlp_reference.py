"""Plain NumPy statement of the budget perceptron the library trains
(test infrastructure): forward with BF16-rounded weights, the pinball loss,
backward, full-batch Adam.  Float64 by default; float32 when asked."""
import numpy as np

H = 64


def bf16(x):
    """Round float32 values to the nearest BF16 (ties to even), as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) >> 16
    return (rounded << 16).astype(np.uint32).view(np.float32)


def unpack(p, f):
    o = 0
    W1 = p[o:o + H * f].reshape(H, f); o += H * f
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    w3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, w3, b3


def forward(p, X, dtype=np.float64, round_weights=True):
    f = X.shape[1]
    W1, b1, W2, b2, w3, b3 = unpack(p, f)
    r = bf16 if round_weights else (lambda a: np.asarray(a, dtype))
    W1, W2, w3 = (r(W1).astype(dtype), r(W2).astype(dtype), r(w3).astype(dtype))
    X = X.astype(dtype)
    h1 = np.maximum(X @ W1.T + b1.astype(dtype), 0)
    h2 = np.maximum(h1 @ W2.T + b2.astype(dtype), 0)
    return h2 @ w3 + dtype(b3), (h1, h2, W2, w3)


def loss_and_grad(p, X, y, quantile, dtype=np.float64, round_weights=True):
    n, f = X.shape
    yh, (h1, h2, W2, w3) = forward(p, X, dtype, round_weights)
    err = y.astype(dtype) - yh
    loss = np.mean(np.where(err > 0, quantile * err, (quantile - 1) * err))
    g = np.where(err > 0, -quantile, np.where(err < 0, 1 - quantile, 0.0)).astype(dtype) / n
    d2 = np.where(h2 > 0, g[:, None] * w3[None, :], 0)
    d1 = np.where(h1 > 0, d2 @ W2, 0)
    grads = [d1.T @ X.astype(dtype), d1.sum(0), d2.T @ h1, d2.sum(0), h2.T @ g, np.array([g.sum()])]
    return loss, np.concatenate([a.ravel() for a in grads])


def train(p, X, y, epochs, lr, quantile, dtype=np.float32):
    p = p.astype(np.float32).copy()
    m1 = np.zeros_like(p)
    m2 = np.zeros_like(p)
    b1p = b2p = 1.0
    losses = []
    for _ in range(epochs):
        loss, g = loss_and_grad(p, X, y, quantile, dtype)
        losses.append(loss)
        g = g.astype(np.float32)
        b1p *= 0.9
        b2p *= 0.999
        m1 = 0.9 * m1 + 0.1 * g
        m2 = 0.999 * m2 + 0.001 * g * g
        p = p - lr * (m1 / (1 - b1p)) / (np.sqrt(m2 / (1 - b2p)) + 1e-8)
    return p, np.array(losses)
