"""Patch-scoring network on the GPU (through the C ABI) against the FP64 MLP
oracle, patch extraction against a numpy gather, and a small learned-proposal
run that must beat a random choice of patches."""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as MO
from oracle import quantize as Q
from workload import config4_workunit

pytestmark = pytest.mark.gpu


def _params(rng, I, H):
    return {"W1": rng.standard_normal((I, H)) * math.sqrt(2.0 / I), "b1": rng.standard_normal(H) * 0.1,
            "W2": rng.standard_normal((H, H)) * math.sqrt(2.0 / H), "b2": rng.standard_normal(H) * 0.1,
            "w3": rng.standard_normal(H) * math.sqrt(1.0 / H), "b3": np.array([0.1])}


def _exact_layer1(rng, p, B, I):
    """Inputs and first-layer parameters on which FP32 accumulation is exact:
    X small integers, W1 and b1 integer multiples of 2^-e with fewer than 8
    significant bits (exact in BF16).  Then z1 = X W1 + b1 is the same number
    on the device as in FP64 whatever the summation order, so the device's
    BF16 h1 equals the oracle's and the comparison isolates the backward
    pass and the optimiser."""
    e = int(round(math.log2(24.0 / math.sqrt(2.0 / I))))
    step = 2.0 ** -e
    q = dict(p)
    q["W1"] = np.clip(np.round(p["W1"] / step), -255, 255) * step
    q["b1"] = np.clip(np.round(p["b1"] / step), -255, 255) * step
    X = np.clip(np.round(rng.standard_normal((B, I))), -3, 3)
    return q, X


def _bf16(x):
    bits = Q.f32_to_bf16_bits(np.asarray(x, dtype=np.float32))
    return bits, Q.bf16_bits_to_f32(bits).astype(np.float64)


SIG_BF16 = 2.0 ** -9 / math.sqrt(3.0)   # standard deviation of one BF16 rounding, relative
N_SIGMA = 10.0


def _grad_sigma(p, X, y, pw, store):
    """Per-element standard deviation of (GPU gradient - FP64 gradient) from
    the device's BF16 storage of the backward operands dz2 and dz1 (each
    rounding an independent relative error of standard deviation 2^-9/sqrt 3),
    propagated through the products by root-sum-square.  h1 is rounded the
    same way on both sides (the oracle's store hook), so its rounding adds
    nothing; FP32 accumulation adds 1e-6 of the sum of |terms|."""
    W1, b1, W2, b2, w3, b3 = (p[k] for k in MO.NAMES)
    B = X.shape[0]
    z1 = X @ W1 + b1
    h1 = store(np.maximum(z1, 0.0))
    z2 = h1 @ W2 + b2
    h2 = np.maximum(z2, 0.0)
    s = h2 @ w3 + b3
    wt = np.where(y > 0.5, pw, 1.0)
    ds = wt * (1.0 / (1.0 + np.exp(-s)) - y) / B
    dz2 = np.outer(ds, w3) * (z2 > 0)
    dz1 = (dz2 @ W2.T) * (z1 > 0)
    acc = 1e-6
    sd = {"w3": acc * (h2.T @ np.abs(ds)), "b3": np.array([acc * np.abs(ds).sum()]),
          "b2": acc * np.abs(dz2).sum(0)}
    sd["W2"] = SIG_BF16 * np.sqrt((h1 ** 2).T @ (dz2 ** 2)) + acc * (h1.T @ np.abs(dz2))
    var_dz1 = (SIG_BF16 ** 2) * ((dz2 ** 2) @ (W2 ** 2).T) * (z1 > 0)
    sd["b1"] = np.sqrt(var_dz1.sum(0)) + acc * np.abs(dz1).sum(0)
    sd["W1"] = np.sqrt((X ** 2).T @ (var_dz1 + SIG_BF16 ** 2 * dz1 ** 2)) + acc * (np.abs(X).T @ np.abs(dz1))
    return sd


@pytest.mark.parametrize("I,H,B", [(64, 32, 40), (8192, 256, 512)])
def test_forward_and_gradients_match_oracle(lib, I, H, B):
    """Forward logits and loss, then every gradient element against the FP64
    oracle: |g - g_ref| <= 1e-2 |g_ref| + 8 sigma, sigma the element's
    rounding spread from the BF16 backward operands; and at least 95 % of
    the larger half of each tensor within the relative 1e-2 alone."""
    rng = np.random.default_rng(I + H)
    p, X0 = _exact_layer1(rng, _params(rng, I, H), B, I)
    # the oracle sees the BF16-rounded weights and inputs the GPU multiplies
    pq = dict(p)
    pq["W1"] = _bf16(p["W1"])[1]
    pq["W2"] = _bf16(p["W2"])[1]
    pq["b3"] = np.float64(p["b3"][0])
    xbits, X = _bf16(X0)
    assert np.array_equal(pq["W1"], p["W1"]) and np.array_equal(X, X0)
    y = (rng.random(B) < 0.3).astype(np.float64)
    m = lib.MLP(I, H, 1024)
    try:
        m.set_params(p)
        # the device keeps h1 in BF16 (round to nearest even) between the layers
        store = lambda h: _bf16(h)[1]  # noqa: E731
        s = m.forward(xbits).astype(np.float64)
        s_ref, _ = MO.forward(pq, X, store)
        assert np.max(np.abs(s - s_ref)) <= 2e-2 * np.max(np.abs(s_ref)) + 1e-3
        loss = m.train_step(xbits, y, 2.5, 1e-3)
        assert abs(loss - MO.loss(pq, X, y, 2.5, store)) <= 1e-2 * abs(loss) + 1e-4
        g = m.get_grads()
    finally:
        m.close()
    gr = MO.backward(pq, X, y, 2.5, store)
    sd = _grad_sigma(pq, X, y, 2.5, store)
    for k in MO.NAMES:
        a = np.asarray(g[k], np.float64).ravel()
        b = np.asarray(gr[k], np.float64).ravel()
        e = N_SIGMA * np.asarray(sd[k], np.float64).ravel()
        err = np.abs(a - b)
        bad = np.nonzero(err > 1e-2 * np.abs(b) + e + 1e-10)[0]
        assert bad.size == 0, (k, bad[:5], a[bad[:5]], b[bad[:5]], e[bad[:5]])
        big = np.abs(b) >= np.median(np.abs(b))
        assert np.mean(err[big] <= 1e-2 * np.abs(b[big])) >= 0.95, k


def _adam_step_range(grads, bounds, t, lr):
    """Element-wise [min, max] of the displacement of Adam step t (1-based)
    over the centre and every corner path of the box g_i +- b_i of the
    gradients of steps 1..t, by mlp_oracle.adam_step from zero moments (the
    elements are independent, so one path covers all of them at once)."""
    lo = hi = None
    for corner in range(2 ** t + 1):
        st = {}
        pp = {k: np.zeros(np.shape(grads[0][k])) for k in MO.NAMES}
        for i in range(t):
            sgn = 0.0 if corner == 2 ** t else (1.0 if (corner >> i) & 1 else -1.0)
            gi = {k: grads[i][k] + sgn * bounds[i][k] for k in MO.NAMES}
            before = {k: np.array(pp[k], copy=True) for k in MO.NAMES}
            pp = MO.adam_step(pp, gi, st, lr)
        d = {k: pp[k] - before[k] for k in MO.NAMES}
        lo = d if lo is None else {k: np.minimum(lo[k], d[k]) for k in MO.NAMES}
        hi = d if hi is None else {k: np.maximum(hi[k], d[k]) for k in MO.NAMES}
    return lo, hi


def test_three_adam_steps_match_oracle(lib):
    """Three training steps on the GPU, each on its own batch so that the
    gradients change from step to step, against Adam on the FP64 oracle's
    gradients (mlp_oracle.adam_step along the oracle's own trajectory).  Each
    step's displacement of every weight whose gradients stay clear of zero
    (|g| > 10 sigma at every step) must lie in the range Adam gives over the
    gradients' rounding spread; every weight must move less than 1.1 lr.
    lr is small (1e-5), so a weight whose tiny gradient takes the other sign
    on the device (and moves the other way) changes the next steps' gradients
    by far less than their rounding spread.  Step 1 is lr sign(g), and the
    later steps mix three different gradients: a missing bias correction
    (3.2 lr at step 1), swapped moment decays (0.003 lr) or a wrong moment
    recursion cannot pass."""
    I, H, B, lr, pw = 64, 32, 40, 1e-5, 2.5
    rng = np.random.default_rng(7)
    p, X0 = _exact_layer1(rng, _params(rng, I, H), B, I)
    batches = [X0] + [np.clip(np.round(rng.standard_normal((B, I))), -3, 3) for _ in range(2)]
    ys = [(rng.random(B) < 0.3).astype(np.float64) for _ in range(3)]
    store = lambda h: _bf16(h)[1]  # noqa: E731
    m = lib.MLP(I, H, 64)
    gpu = [{k: np.asarray(v, np.float64) for k, v in p.items()}]
    try:
        m.set_params(p)
        for X, y in zip(batches, ys):
            m.train_step(_bf16(X)[0], y, pw, lr, want_loss=False)
            gpu.append({k: np.asarray(v, np.float64) for k, v in m.get_params().items()})
    finally:
        m.close()
    ref = {k: np.asarray(v, np.float64).reshape(np.shape(gpu[0][k])).copy() for k, v in p.items()}
    st, grads, bounds = {}, [], []
    clear = {k: np.ones(np.shape(ref[k]), bool) for k in MO.NAMES}
    for t, (X, y) in enumerate(zip(batches, ys)):
        pq = dict(ref)
        pq["W1"] = _bf16(ref["W1"])[1]
        pq["W2"] = _bf16(ref["W2"])[1]
        pq["b3"] = np.float64(ref["b3"].reshape(-1)[0])
        gr = MO.backward(pq, X, y, pw, store)
        sd = _grad_sigma(pq, X, y, pw, store)
        gr = {k: np.asarray(gr[k], np.float64).reshape(np.shape(ref[k])) for k in MO.NAMES}
        bd = {k: N_SIGMA * np.asarray(sd[k], np.float64).reshape(np.shape(ref[k])) + 1e-3 * np.abs(gr[k])
              for k in MO.NAMES}
        grads.append(gr)
        bounds.append(bd)
        ref = MO.adam_step(ref, gr, st, lr)
        lo, hi = _adam_step_range(grads, bounds, t + 1, lr)
        for k in MO.NAMES:
            clear[k] &= np.abs(gr[k]) > bd[k]
            d = gpu[t + 1][k] - gpu[t][k]
            pad = 1e-3 * lr + 0.1 * (hi[k] - lo[k]) + 2.0 ** -23 * np.abs(gpu[t + 1][k])
            c = clear[k]
            assert np.all(d[c] >= lo[k][c] - pad[c]) and np.all(d[c] <= hi[k][c] + pad[c]), (k, t)
            assert np.all(np.abs(d) <= 1.1 * lr), (k, t)
    for k in ("W1", "W2"):
        assert clear[k].mean() >= 0.8, (k, clear[k].mean())


def test_training_separates_a_toy_problem(lib):
    rng = np.random.default_rng(3)
    I, H, B = 64, 32, 256
    X = rng.standard_normal((B, I))
    y = (X[:, 0] - X[:, 3] > 0).astype(np.float32)
    xbits, _ = _bf16(X)
    m = lib.MLP(I, H, B)
    try:
        m.set_params(_params(rng, I, H))
        l0 = m.train_step(xbits, y, 1.0, 5e-3)
        for _ in range(300):
            l1 = m.train_step(xbits, y, 1.0, 5e-3, want_loss=False)
        l1 = m.train_step(xbits, y, 1.0, 5e-3)
        assert l1 < 0.3 * l0
        acc = np.mean((m.forward(xbits) > 0) == (y > 0.5))
        assert acc > 0.95
    finally:
        m.close()


def test_patch_extraction_matches_gather(lib):
    torch = pytest.importorskip("torch")
    from workload import DET_H, DetectorData, TemplateBank, cn_noise, T0, T_SFT
    n_a, n_d, n_f = 8, 4, 64
    a = (np.arange(n_a) + 0.5) * 2 * math.pi / n_a
    sd = -1 + (np.arange(n_d) + 0.5) * 2 / n_d
    A, S = np.meshgrid(a, sd, indexing="ij")
    sky = np.stack([A.ravel(), np.arcsin(S.ravel())], 1)
    det = DetectorData(DET_H["lat"], 0.0, DET_H["az"], T0 + T_SFT * np.arange(30), cn_noise(4, 1, (30, 140)))
    g = lib.FStat(0, topk=1)
    try:
        lib.fstat_set_sfts(g.ctx, 0, det.lat, det.lon, det.az, T_SFT, 180000, det.t_start, det.bins)
        g.set_bank(TemplateBank(sky, (180000 + 30) / T_SFT, 1 / T_SFT, n_f, np.zeros(1), T0))
        g.compute()
        twoF = g.twoF().reshape(n_a, n_d, n_f)
        fst = np.array([0, 16, 48], dtype=np.int32)
        out = torch.empty((2 * 2 * 3, 4 * 2 * 16), dtype=torch.int16, device="cuda")
        lib.fstat_extract_patches(g.ctx, n_a, n_d, 4, 2, 16, fst, 4.0, 0.125, out)
        got = out.cpu().numpy().view(np.uint16)
        for pa in range(2):
            for pd in range(2):
                for q, f in enumerate(fst):
                    blk = twoF[pa * 4:(pa + 1) * 4, pd * 2:(pd + 1) * 2, f:f + 16].reshape(-1)
                    x = np.maximum(blk - np.float32(4.0), np.float32(0.0)) * np.float32(0.125)
                    want = Q.f32_to_bf16_bits(x.astype(np.float32))
                    np.testing.assert_array_equal(got[(pa * 2 + pd) * 3 + q], want)
    finally:
        g.close()


def test_learned_proposal_beats_random_choice(lib):
    """Small learned-proposal run: trained on windows of coarse maps (eight
    signals per training workunit, and up to three detector lines), the
    network's 8 best patches of 232 hold most of the held-out signals the
    exhaustive fine grid detects, far more than 8 random patches, at a
    fraction of the exhaustive grid's cost.  With detector lines in the
    held-out data the coarse-max ranking spends its budget on line patches
    and the network does not: it recovers clearly more signals."""
    pytest.importorskip("torch")
    from paper_0904_1826_gb300 import proposal as PR
    search = PR.ProposalSearch(0, hidden=64, max_batch=512)
    try:
        train = [config4_workunit(i, True, n_sft=150, n_signals=8, n_lines=3) for i in range(60)]
        X, y = search.training_set(train, np.random.default_rng(5), 16, 256)
        search.init_params(np.random.default_rng(1))
        hist = search.train(X, y, steps=1200, batch=256, lr=3e-4, pos_frac=0.25, seed=2)
        assert hist[-1] < 0.3 * hist[0]
        test = [config4_workunit(i, False, n_sft=150) for i in range(16)]
        res = PR.evaluate(search, test, n_refine=8, noise_patches_per_wu=24)
        assert res["n_detected_exhaustive"] >= 6
        assert res["recall_nn"] >= 0.5
        assert res["recall_nn"] >= res["recall_random"] + 0.3
        assert res["speedup"] > 10
        test_l = [config4_workunit(i, False, n_sft=150, n_lines=3) for i in range(16)]
        rl = PR.evaluate(search, test_l, n_refine=8, noise_patches_per_wu=24)
        assert rl["n_detected_exhaustive"] >= 6
        assert rl["recall_nn"] >= rl["recall_coarse_max"] + 0.2, (rl["recall_nn"], rl["recall_coarse_max"])
        top = rl["line_patches_in_top"]
        assert top["nn"] * 2 < top["cm"], top
    finally:
        search.close()
