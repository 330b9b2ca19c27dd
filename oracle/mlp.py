"""float64 reference of the per-phase policy network (TEST INFRASTRUCTURE ONLY).

Layout of the weight vector (float, input index first):
    W1[8][32], b1[32], W2[32][32], b2[32], W3[32][4], b3[4]     (1476 values)
Network: h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2), y = h2 W3 + b3,
relu'(0) = 0.  Loss of a batch with arm a_b and target t_b:
    L = (1/B) sum_b (y_b[a_b] - t_b)^2.
The gradient is the textbook chain rule written out layer by layer; the tests
pin it against central finite differences and closed forms.
"""
from __future__ import annotations

import numpy as np

F, H, A = 8, 32, 4
SIZES = [("W1", (F, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, A)), ("b3", (A,))]
NWEIGHTS = sum(int(np.prod(s)) for _, s in SIZES)  # 1476


def unpack(w):
    w = np.asarray(w, dtype=np.float64)
    assert w.size == NWEIGHTS
    out, off = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = w[off:off + k].reshape(shape)
        off += k
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(parts[name], dtype=np.float64).reshape(-1) for name, _ in SIZES])


def forward(w, x):
    """Outputs y[B, 4] and the intermediates (z1, h1, z2, h2)."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ p["W1"] + p["b1"]
    h1 = np.maximum(z1, 0.0)
    z2 = h1 @ p["W2"] + p["b2"]
    h2 = np.maximum(z2, 0.0)
    y = h2 @ p["W3"] + p["b3"]
    return y, (z1, h1, z2, h2)


def loss(w, x, target, arm):
    y, _ = forward(w, x)
    b = np.arange(len(arm))
    err = y[b, np.asarray(arm)] - np.asarray(target, dtype=np.float64)
    return float(np.mean(err * err))


def backward(w, x, target, arm):
    """(loss, gradient) of the masked mean squared error."""
    p = unpack(w)
    x = np.asarray(x, dtype=np.float64)
    arm = np.asarray(arm)
    B = x.shape[0]
    y, (z1, h1, z2, h2) = forward(w, x)
    err = y[np.arange(B), arm] - np.asarray(target, dtype=np.float64)
    dy = np.zeros_like(y)
    dy[np.arange(B), arm] = 2.0 * err / B           # dL/dy
    g = {}
    g["W3"] = h2.T @ dy
    g["b3"] = dy.sum(axis=0)
    dz2 = (dy @ p["W3"].T) * (z2 > 0)               # through relu
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(axis=0)
    dz1 = (dz2 @ p["W2"].T) * (z1 > 0)
    g["W1"] = x.T @ dz1
    g["b1"] = dz1.sum(axis=0)
    return float(np.mean(err * err)), pack(g)


def init(seed: int, scale: float = 0.3) -> np.ndarray:
    """Seeded random weights (uniform in [-scale, scale], biases small)."""
    rng = np.random.default_rng(seed)
    parts = {}
    for name, shape in SIZES:
        fan_in = shape[0] if len(shape) == 2 else 1
        lim = scale if len(shape) == 2 else 0.05
        parts[name] = rng.uniform(-lim, lim, size=shape) * (1.0 if len(shape) == 1 else np.sqrt(8.0 / max(fan_in, 8)))
    return pack(parts)
