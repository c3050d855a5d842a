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


def _bf16(x):
    bits = Q.f32_to_bf16_bits(np.asarray(x, dtype=np.float32))
    return bits, Q.bf16_bits_to_f32(bits).astype(np.float64)


@pytest.mark.parametrize("I,H,B", [(64, 32, 40), (8192, 256, 512)])
def test_forward_and_gradients_match_oracle(lib, I, H, B):
    rng = np.random.default_rng(I + H)
    p = _params(rng, I, H)
    # the oracle sees the BF16-rounded weights and inputs the GPU multiplies
    pq = dict(p)
    pq["W1"] = _bf16(p["W1"])[1]
    pq["W2"] = _bf16(p["W2"])[1]
    xbits, X = _bf16(rng.standard_normal((B, I)))
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
        gr = MO.backward(pq, X, y, 2.5, store)
        for k in MO.NAMES:
            a, b = np.asarray(g[k], np.float64).ravel(), np.asarray(gr[k], np.float64).ravel()
            assert np.linalg.norm(a - b) <= 2e-2 * np.linalg.norm(b) + 1e-6, k
        # the step applied Adam: first step moves each weight by about lr
        p2 = m.get_params()
        step = np.abs(p2["W2"] - p["W2"].astype(np.float32))
        assert np.median(step[np.abs(gr["W2"]) > 1e-6]) == pytest.approx(1e-3, rel=0.05)
    finally:
        m.close()


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
    signals per training workunit), the network's 8 best patches of 232 hold
    most of the held-out signals the exhaustive fine grid detects, far more
    than 8 random patches, at a fraction of the exhaustive grid's cost."""
    pytest.importorskip("torch")
    from paper_0904_1826_gb300 import proposal as PR
    search = PR.ProposalSearch(0, hidden=64, max_batch=512)
    try:
        train = [config4_workunit(i, True, n_sft=150, n_signals=8) for i in range(40)]
        X, y = search.training_set(train, np.random.default_rng(5), 16, 256)
        search.init_params(np.random.default_rng(1))
        hist = search.train(X, y, steps=800, batch=256, lr=3e-4, pos_frac=0.25, seed=2)
        assert hist[-1] < 0.3 * hist[0]
        test = [config4_workunit(i, False, n_sft=150) for i in range(16)]
        res = PR.evaluate(search, test, n_refine=8, noise_patches_per_wu=24)
        assert res["n_detected_exhaustive"] >= 6
        assert res["recall_nn"] >= 0.5
        assert res["recall_nn"] >= res["recall_random"] + 0.3
        assert res["speedup"] > 10
    finally:
        search.close()
