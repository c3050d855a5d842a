"""FP64 oracle of the patch-scoring MLP (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module; it shares no code with the CUDA MLP.

Network (the learned proposal is not in the paper; this is its reading: a
patch of 16 x 16 sky points x 32 frequencies of the coarse 2F map, ReLU
hidden layers, a sigmoid output trained with binary cross-entropy): 8192
inputs -> 256 ReLU -> 256 ReLU -> 1 logit s; p = sigmoid(s); loss = mean
binary cross-entropy with a positive-class weight w+:
    L = mean_i  w_i (softplus(s_i) - y_i s_i),  w_i = w+ if y_i = 1 else 1.
Parameters: W1 [8192, 256], b1 [256], W2 [256, 256], b2 [256], w3 [256], b3.
Adam: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr m_hat / (sqrt(v_hat) + eps).

`store` (optional, default none): a function applied to the first hidden
activation h1 where it is stored for the second layer and for W2's gradient,
for a device that keeps h1 in a narrower type.  The backward pass treats it as
the identity (its derivative is one almost everywhere for a rounding), so the
ReLU decisions of layer 2 are taken on the stored h1 as on such a device.
"""
from __future__ import annotations

import numpy as np

NAMES = ("W1", "b1", "W2", "b2", "w3", "b3")


def relu(x):
    return np.maximum(x, 0.0)


def softplus(s):
    return np.maximum(s, 0.0) + np.log1p(np.exp(-np.abs(s)))


def sigmoid(s):
    return 1.0 / (1.0 + np.exp(-s))


def forward(params, X, store=None):
    """Logits s [B] and the hidden activations (z1, h1, z2, h2); h1 as stored."""
    z1 = X @ params["W1"] + params["b1"]
    h1 = relu(z1)
    if store is not None:
        h1 = store(h1)
    z2 = h1 @ params["W2"] + params["b2"]
    h2 = relu(z2)
    s = h2 @ params["w3"] + params["b3"]
    return s, (z1, h1, z2, h2)


def loss(params, X, y, pos_weight: float = 1.0, store=None):
    s, _ = forward(params, X, store)
    w = np.where(y > 0.5, pos_weight, 1.0)
    return float(np.mean(w * (softplus(s) - y * s)))


def backward(params, X, y, pos_weight: float = 1.0, store=None):
    """Gradients of `loss` with respect to every parameter (FP64)."""
    B = X.shape[0]
    s, (z1, h1, z2, h2) = forward(params, X, store)
    w = np.where(y > 0.5, pos_weight, 1.0)
    ds = w * (sigmoid(s) - y) / B                 # dL/ds
    g = {}
    g["w3"] = h2.T @ ds
    g["b3"] = np.array(np.sum(ds))
    dz2 = np.outer(ds, params["w3"]) * (z2 > 0)
    g["W2"] = h1.T @ dz2
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ params["W2"].T) * (z1 > 0)
    g["W1"] = X.T @ dz1
    g["b1"] = dz1.sum(0)
    return g


def adam_step(params, grads, state, lr: float, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8):
    """One Adam update in place; state holds m, v per parameter and the step t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        params[k] = params[k] - lr * mh / (np.sqrt(vh) + eps)
    return params
