"""The float64 policy-network oracle against finite differences and closed forms."""
import numpy as np

from oracle import mlp


def _batch(seed, B=64):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(B, mlp.F))
    t = rng.normal(0, 1, size=B)
    a = rng.integers(0, mlp.A, size=B)
    return x, t, a


def test_gradient_matches_central_differences():
    w = mlp.init(3)
    x, t, a = _batch(4)
    L, g = mlp.backward(w, x, t, a)
    assert abs(L - mlp.loss(w, x, t, a)) < 1e-12
    rng = np.random.default_rng(5)
    idx = np.concatenate([rng.choice(mlp.NWEIGHTS, 200, replace=False), np.arange(mlp.NWEIGHTS - 40, mlp.NWEIGHTS)])
    eps = 1e-6
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += eps
        wm[i] -= eps
        fd = (mlp.loss(wp, x, t, a) - mlp.loss(wm, x, t, a)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_zero_output_layer_closed_form():
    """W3 = 0: y = b3, so dL/db3[k] = (2/B) sum_{a_b = k} (b3[k] - t_b) and every
    other gradient is 0."""
    p = mlp.unpack(mlp.init(7))
    p["W3"][:] = 0.0
    p["b3"][:] = [0.5, -1.0, 2.0, 0.25]
    w = mlp.pack(p)
    x, t, a = _batch(8, B=50)
    L, g = mlp.backward(w, x, t, a)
    gp = mlp.unpack(g)
    for k in range(mlp.A):
        sel = a == k
        assert np.isclose(gp["b3"][k], 2.0 / len(a) * np.sum(p["b3"][k] - t[sel]))
    for name in ("W1", "b1", "W2", "b2"):
        assert np.all(gp[name] == 0.0)
    assert np.isclose(L, np.mean((p["b3"][a] - t) ** 2))


def test_all_active_network_is_the_linear_composition():
    """Positive inputs and non-negative weights keep every ReLU active, so the
    network equals x W1 W2 W3 + (b1 W2 + b2) W3 + b3."""
    rng = np.random.default_rng(9)
    p = {name: rng.uniform(0.01, 0.2, size=shape) for name, shape in mlp.SIZES}
    w = mlp.pack(p)
    x = rng.uniform(0.1, 1.0, size=(10, mlp.F))
    y, _ = mlp.forward(w, x)
    ref = x @ p["W1"] @ p["W2"] @ p["W3"] + (p["b1"] @ p["W2"] + p["b2"]) @ p["W3"] + p["b3"]
    assert np.allclose(y, ref, rtol=1e-12)


def test_gradient_step_lowers_the_loss():
    w = mlp.init(11)
    x, t, a = _batch(12)
    L0, g = mlp.backward(w, x, t, a)
    assert mlp.loss(w - 1e-3 * g, x, t, a) < L0
