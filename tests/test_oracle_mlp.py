"""Pins of the FP64 MLP oracle: hand-built networks, finite differences, Adam."""
import numpy as np

from oracle import mlp
import seeded_inputs as si


def test_param_count():
    assert mlp.n_params() == 9282


def test_forward_hand_built_network():
    """Weights that route relu(x0), relu(-x1) and x2 through the network give
    y0 = relu(x0) + 2 relu(-x1), y1 = 3 relu(x2)."""
    ps = [np.zeros(s) for s in mlp.param_shapes()]
    W1, W2, W3, W4 = ps[0], ps[2], ps[4], ps[6]
    W1[0, 0] = 1.0
    W1[1, 1] = -1.0
    W1[2, 2] = 1.0
    for W in (W2, W3):
        W[0, 0] = W[1, 1] = W[2, 2] = 1.0
    W4[0, 0] = 1.0
    W4[0, 1] = 2.0
    W4[1, 2] = 3.0
    ps[7][:] = [0.5, -0.25]
    flat = mlp.flatten(ps)
    x = np.zeros((4, 12))
    x[:, 0] = [1.0, -1.0, 2.0, 0.0]
    x[:, 1] = [-2.0, 3.0, 0.5, -1.0]
    x[:, 2] = [0.0, 4.0, -3.0, 1.5]
    y, _ = mlp.forward(flat, x)
    r = lambda v: np.maximum(v, 0.0)
    exp0 = r(x[:, 0]) + 2 * r(-x[:, 1]) + 0.5
    exp1 = 3 * r(x[:, 2]) - 0.25
    assert np.allclose(y[:, 0], exp0, rtol=0, atol=1e-15)
    assert np.allclose(y[:, 1], exp1, rtol=0, atol=1e-15)


def test_backward_matches_central_differences():
    flat = mlp.init_params(si.uniform01(5, mlp.n_params()))
    flat = flat + 0.01 * (si.uniform01(6, flat.size) - 0.5)   # non-zero biases
    x = 2 * si.uniform01(7, 8 * 12).reshape(8, 12) - 1
    t = si.uniform01(8, 16).reshape(8, 2)
    g = mlp.backward(flat, x, t)
    h = 1e-6
    idx = np.unique(np.linspace(0, flat.size - 1, 400).astype(int))
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (mlp.loss(flat + e, x, t) - mlp.loss(flat - e, x, t)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_adam_first_step_closed_form():
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -1e-3, 0.0])
    lr, eps = 0.01, 1e-8
    p1, m, v = mlp.adam_step(p, g, np.zeros(3), np.zeros(3), 1, lr=lr, eps=eps)
    assert np.allclose(p1, p - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)


def test_training_reduces_loss():
    flat = mlp.init_params(si.uniform01(9, mlp.n_params()))
    x = 2 * si.uniform01(10, 64 * 12).reshape(64, 12) - 1
    t = np.stack([x[:, 0] + 0.5 * x[:, 1], x[:, 2] * x[:, 3]], axis=1)
    m = np.zeros_like(flat)
    v = np.zeros_like(flat)
    l0 = mlp.loss(flat, x, t)
    for s in range(1, 201):
        flat, m, v = mlp.adam_step(flat, mlp.backward(flat, x, t), m, v, s, lr=3e-3)
    assert mlp.loss(flat, x, t) < 0.2 * l0
