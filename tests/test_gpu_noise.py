"""Noise-floor normalisation and noise weights on the GPU (fstat_set_noise_floor)
against the oracle (oracle/noise_oracle.py) on non-stationary data: two
detectors whose SFT noise levels differ by up to 10x, with signals."""
import dataclasses

import numpy as np
import pytest

from oracle import fstat_oracle as O
from oracle import noise_oracle as N
from workload import config_mid

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3
W = 16


def _case(seed=31):
    w = config_mid(seed=seed, n_sft=40, n_sky=3, n_f=60, n_fdot=2, n_bins=200)
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    rng = np.random.default_rng(seed)
    scaled = []
    for d, b in zip(w.detectors, bins):
        g = np.sqrt(rng.uniform(1.0, 10.0, d.n_sft))[:, None]
        scaled.append((b * g).astype(np.complex64))
    dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, scaled)]
    return w, scaled, dets


def test_floor_and_weights_match_oracle(lib):
    w, scaled, dets = _case()
    g = lib.FStat(0, dterms=w.dterms, topk=10)
    try:
        g.load_workload(w, bins_override=scaled)
        lib.fstat_set_noise_floor(g.ctx, W)
        g.compute()
        fl, wt = lib.fstat_get_noise(g.ctx, w.n_sft_total, w.n_bins)
    finally:
        g.close()
    ref_fl = np.concatenate([N.running_median_floor(d.bins, W) for d in dets])
    np.testing.assert_array_equal(fl, ref_fl)                       # FP32 selection, bit for bit
    ref_w = np.concatenate(N.noise_weights([N.running_median_floor(d.bins, W) for d in dets]))
    np.testing.assert_allclose(wt, ref_w, rtol=1e-12)


@pytest.mark.parametrize("algo", ["auto", "farpoly", "direct"])
def test_weighted_2F_matches_oracle(lib, algo):
    w, scaled, dets = _case(seed=32)
    ref = O.compute_fstat_freq_band(N.weighted_detectors(dets, W), w.T, w.k_lo, w.dterms, w.bank).ravel()
    g = lib.FStat(0, dterms=w.dterms, topk=10, algo=algo)
    try:
        g.load_workload(w, bins_override=scaled)
        lib.fstat_set_noise_floor(g.ctx, W)
        g.compute()
        got = g.twoF().astype(np.float64)
        assert g.error_flags() == 0
        # switching it off gives the plain statistic again
        lib.fstat_set_noise_floor(g.ctx, 0)
        g.compute()
        plain = g.twoF().astype(np.float64)
    finally:
        g.close()
    err = np.abs(got - ref)
    assert np.all(err <= REL * ref + ABS), float(np.max(err / (REL * ref + ABS)))
    ref_plain = O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank).ravel()
    assert np.all(np.abs(plain - ref_plain) <= REL * ref_plain + ABS)


def test_noise_floor_errors(lib):
    g = lib.FStat(0)
    try:
        with pytest.raises(lib.FstatError) as e:
            lib.fstat_set_noise_floor(g.ctx, 65)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError) as e:
            lib.fstat_get_noise(g.ctx, 1, 1)
        assert e.value.code == lib.FSTAT_ESTATE
    finally:
        g.close()
