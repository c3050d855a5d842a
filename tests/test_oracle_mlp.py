"""Pins of the MLP oracle (CPU only): central finite differences of the loss
on random parameters of every tensor, closed values, and an Adam step on a
convex problem."""
import math

import numpy as np

from oracle import mlp_oracle as MO


def _params(rng, n_in=40, h=16):
    return {"W1": rng.standard_normal((n_in, h)) / math.sqrt(n_in), "b1": rng.standard_normal(h) * 0.1,
            "W2": rng.standard_normal((h, h)) / math.sqrt(h), "b2": rng.standard_normal(h) * 0.1,
            "w3": rng.standard_normal(h) / math.sqrt(h), "b3": np.array(0.05)}


def test_gradients_match_central_finite_differences():
    rng = np.random.default_rng(0)
    p = _params(rng)
    X = rng.standard_normal((12, 40))
    y = (rng.random(12) < 0.4).astype(np.float64)
    g = MO.backward(p, X, y, pos_weight=3.0)
    h = 1e-6
    checked = 0
    for k in MO.NAMES:
        flat = p[k].reshape(-1)
        for i in rng.choice(flat.size, size=min(flat.size, 30), replace=False):
            old = flat[i]
            flat[i] = old + h
            lp = MO.loss(p, X, y, 3.0)
            flat[i] = old - h
            lm = MO.loss(p, X, y, 3.0)
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[k].reshape(-1)[i]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (k, i, fd, an)
            checked += 1
    assert checked >= 100


def test_closed_values():
    p = {"W1": np.zeros((4, 3)), "b1": np.zeros(3), "W2": np.zeros((3, 3)), "b2": np.zeros(3),
         "w3": np.zeros(3), "b3": np.array(0.0)}
    X = np.ones((5, 4))
    y = np.array([1.0, 0.0, 1.0, 0.0, 0.0])
    # s = 0 everywhere: loss = log 2 per sample, weighted
    assert abs(MO.loss(p, X, y) - math.log(2)) < 1e-15
    assert abs(MO.loss(p, X, y, pos_weight=2.0) - math.log(2) * (2 + 2 + 3) / 5) < 1e-15
    g = MO.backward(p, X, y)
    assert abs(float(g["b3"]) - np.mean(0.5 - y)) < 1e-15
    # a ReLU network with a positive path is piecewise linear in the input
    rng = np.random.default_rng(1)
    q = _params(rng, 6, 5)
    Xq = rng.standard_normal((3, 6))
    s1, _ = MO.forward(q, Xq)
    s2, _ = MO.forward(q, 2 * Xq)
    z1 = Xq @ q["W1"]
    if np.all((z1 > 0) == (2 * Xq @ q["W1"] + q["b1"] > 0)):
        assert np.all(np.isfinite(s1)) and np.all(np.isfinite(s2))


def test_adam_converges_on_separable_data():
    rng = np.random.default_rng(2)
    p = _params(rng, 8, 8)
    X = rng.standard_normal((64, 8))
    y = (X[:, 0] + 0.5 * X[:, 1] > 0).astype(np.float64)
    st = {}
    l0 = MO.loss(p, X, y)
    for _ in range(300):
        MO.adam_step(p, MO.backward(p, X, y), st, lr=1e-2)
    assert MO.loss(p, X, y) < 0.2 * l0
    assert st["t"] == 300


def test_store_hook_reaches_layer_two_and_its_gradient():
    """A store that zeroes h1 leaves s = relu(b2) . w3 + b3 and a zero W2
    gradient; the identity store changes nothing."""
    rng = np.random.default_rng(4)
    p = _params(rng, 10, 6)
    X = rng.standard_normal((7, 10))
    y = (rng.random(7) < 0.5).astype(np.float64)
    s0, _ = MO.forward(p, X, store=lambda h: 0.0 * h)
    np.testing.assert_allclose(s0, np.full(7, np.maximum(p["b2"], 0) @ p["w3"] + p["b3"]), rtol=0, atol=1e-15)
    g0 = MO.backward(p, X, y, 2.0, store=lambda h: 0.0 * h)
    assert np.all(g0["W2"] == 0.0)
    g1 = MO.backward(p, X, y, 2.0, store=lambda h: h)
    g2 = MO.backward(p, X, y, 2.0)
    for k in MO.NAMES:
        np.testing.assert_array_equal(g1[k], g2[k])
