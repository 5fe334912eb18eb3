"""FP64 reference of the learned cost model (TEST INFRASTRUCTURE ONLY).

The paper tunes leaf tile sizes by exhaustive exploration (Sec. 5.1.5); the
engine adds a small learned model of the tuner's own records.  This module is
the plain NumPy float64 definition of that model, used only to check the CUDA
kernels of the library.

Network: x (12) -> Linear(64) -> ReLU -> Linear(64) -> ReLU -> Linear(64)
-> ReLU -> Linear(2).  Weights W_l have shape (out, in), y = W x + b.
Loss over a batch of B samples with targets t (B, 2):
    L = (1 / B) * sum_b sum_o 0.5 * (y_bo - t_bo)^2
Adam (Kingma and Ba, 2015) with bias correction:
    m = b1 m + (1 - b1) g ; v = b2 v + (1 - b2) g^2
    p -= lr * (m / (1 - b1^s)) / (sqrt(v / (1 - b2^s)) + eps)
Parity status: forward pinned by hand-built networks with known outputs,
backward pinned by central finite differences of the loss, Adam pinned by the
first-step closed form p -= lr * g / (|g| + eps).
"""
from __future__ import annotations

import numpy as np

LAYERS = (12, 64, 64, 64, 2)


def param_shapes(layers=LAYERS):
    out = []
    for i in range(len(layers) - 1):
        out.append((layers[i + 1], layers[i]))
        out.append((layers[i + 1],))
    return out


def n_params(layers=LAYERS):
    return int(sum(int(np.prod(s)) for s in param_shapes(layers)))


def unflatten(flat, layers=LAYERS):
    """Split the flat parameter vector (W1, b1, W2, b2, ...) into arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for s in param_shapes(layers):
        k = int(np.prod(s))
        out.append(flat[o:o + k].reshape(s))
        o += k
    if o != flat.size:
        raise ValueError("parameter vector has the wrong length")
    return out


def flatten(params):
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in params])


def forward(flat, x, layers=LAYERS):
    """Returns (y, activations) with activations[l] the input of layer l."""
    ps = unflatten(flat, layers)
    h = np.asarray(x, dtype=np.float64)
    acts = [h]
    nl = len(layers) - 1
    for l in range(nl):
        W, b = ps[2 * l], ps[2 * l + 1]
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if l < nl - 1 else z
        acts.append(h)
    return h, acts


def loss(flat, x, t, layers=LAYERS):
    y, _ = forward(flat, x, layers)
    B = y.shape[0]
    return float(np.sum(0.5 * (y - t) ** 2) / B)


def backward(flat, x, t, layers=LAYERS):
    """Gradient of ``loss`` with respect to the flat parameter vector."""
    ps = unflatten(flat, layers)
    y, acts = forward(flat, x, layers)
    B = y.shape[0]
    nl = len(layers) - 1
    grads = [None] * (2 * nl)
    d = (y - t) / B                          # dL/dz of the last layer
    for l in range(nl - 1, -1, -1):
        h_in = acts[l]
        grads[2 * l] = d.T @ h_in            # dL/dW = d^T h
        grads[2 * l + 1] = d.sum(axis=0)
        if l > 0:
            d = (d @ ps[2 * l]) * (acts[l] > 0.0)   # back through W, then the ReLU of layer l-1
    return flatten(grads)


def adam_step(flat, grad, m, v, step, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update; returns new (params, m, v).  ``step`` counts from 1."""
    m = b1 * m + (1.0 - b1) * grad
    v = b2 * v + (1.0 - b2) * grad * grad
    mh = m / (1.0 - b1 ** step)
    vh = v / (1.0 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed_uniform, layers=LAYERS):
    """He-uniform weights and zero biases from a vector of U[0,1) draws."""
    u = np.asarray(seed_uniform, dtype=np.float64)
    out, o = [], 0
    for i in range(len(layers) - 1):
        fan_in, fan_out = layers[i], layers[i + 1]
        k = fan_in * fan_out
        lim = np.sqrt(6.0 / fan_in)
        out.append((2.0 * u[o:o + k] - 1.0).reshape(fan_out, fan_in) * lim)
        o += k
        out.append(np.zeros(fan_out))
    return flatten(out)
