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


# ---------------------------------------------------------------- Adam closed forms

def _adam_closed_form_error(step, eps=1e-8, beta1=0.9, beta2=0.999):
    """Largest deviation of an Adam implementation `step(params, grads,
    state, lr, beta1, beta2, eps)` from Adam's closed forms, over:
      * step 1 from zero moments: p1 - p0 = -lr g1 / (|g1| + eps);
      * step 2: m_hat = (beta1 g1 + g2) / (1 + beta1),
                v_hat = (beta2 g1^2 + g2^2) / (1 + beta2),
        p2 - p1 = -lr m_hat / (sqrt(v_hat) + eps);
      * a constant gradient for 5 steps: every step moves -lr g / (|g| + eps)
        (bias correction makes m_hat = g, v_hat = g^2 at every t).
    Gradients span magnitudes from 1e-6 to 1 so that eps matters for some."""
    rng = np.random.default_rng(21)
    shapes = {"W1": (5, 4), "b1": (4,), "W2": (4, 4), "b2": (4,), "w3": (4,), "b3": ()}
    lr = 1e-3

    def grads():
        return {k: rng.standard_normal(s) * 10.0 ** rng.uniform(-6, 0, s) for k, s in shapes.items()}

    p0 = {k: rng.standard_normal(s) for k, s in shapes.items()}
    g1, g2 = grads(), grads()
    st = {}
    p = {k: v.copy() for k, v in p0.items()}
    p = step(p, g1, st, lr, beta1, beta2, eps)
    err = 0.0
    for k in shapes:
        want = -lr * g1[k] / (np.abs(g1[k]) + eps)
        err = max(err, float(np.max(np.abs((p[k] - p0[k]) - want))) / lr)
    p1 = {k: v.copy() for k, v in p.items()}
    p = step(p, g2, st, lr, beta1, beta2, eps)
    for k in shapes:
        mh = (beta1 * g1[k] + g2[k]) / (1 + beta1)
        vh = (beta2 * g1[k] ** 2 + g2[k] ** 2) / (1 + beta2)
        want = -lr * mh / (np.sqrt(vh) + eps)
        err = max(err, float(np.max(np.abs((p[k] - p1[k]) - want))) / lr)
    st = {}
    p = {k: v.copy() for k, v in p0.items()}
    for _ in range(5):
        prev = {k: v.copy() for k, v in p.items()}
        p = step(p, g1, st, lr, beta1, beta2, eps)
        for k in shapes:
            want = -lr * g1[k] / (np.abs(g1[k]) + eps)
            err = max(err, float(np.max(np.abs((p[k] - prev[k]) - want))) / lr)
    return err


def _adam_no_bias_correction(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    for k in MO.NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        params[k] = params[k] - lr * m / (np.sqrt(v) + eps)
    return params


def _adam_swapped_betas(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    return MO.adam_step(params, grads, state, lr, beta2, beta1, eps)


def _adam_eps_inside_sqrt(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in MO.NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        params[k] = params[k] - lr * (m / (1 - beta1 ** t)) / np.sqrt(v / (1 - beta2 ** t) + eps)
    return params


def _adam_first_moment_only_bias(params, grads, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in MO.NAMES:
        m = state.setdefault("m_" + k, np.zeros_like(params[k]))
        v = state.setdefault("v_" + k, np.zeros_like(params[k]))
        m[...] = beta1 * m + (1 - beta1) * grads[k]
        v[...] = beta2 * v + (1 - beta2) * grads[k] ** 2
        params[k] = params[k] - lr * (m / (1 - beta1 ** t)) / (np.sqrt(v) + eps)
    return params


def test_adam_matches_closed_forms():
    assert _adam_closed_form_error(MO.adam_step) < 1e-12


def test_adam_closed_forms_catch_planted_mistakes():
    for bad in (_adam_no_bias_correction, _adam_swapped_betas, _adam_eps_inside_sqrt,
                _adam_first_moment_only_bias):
        assert _adam_closed_form_error(bad) > 1e-2, bad.__name__
