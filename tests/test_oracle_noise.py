"""Pins of the noise-floor / noise-weight oracle (CPU only)."""
import dataclasses
import math

import numpy as np

from oracle import fstat_oracle as O
from oracle import noise_oracle as N
from workload import config_mid

LN2 = math.log(2.0)


def test_running_median_of_a_ramp_is_closed_form():
    # power 1..9 in one SFT (bins with |X|^2 = k exactly), half window 1:
    # medians 1.5 (clipped, averaged), 2, 3, ..., 8, 8.5
    p = np.arange(1, 10, dtype=np.float64)
    bins = (np.sqrt(p).astype(np.float32) + 0j).astype(np.complex64)[None, :]
    want_med = np.array([1.5, 2, 3, 4, 5, 6, 7, 8, 8.5])
    got = N.running_median_floor(bins, 1)[0].astype(np.float64)
    pw = N.power_f32(bins)[0].astype(np.float64)           # |sqrt(k)|^2 in FP32, within an ulp of k
    assert np.allclose(pw, p, rtol=3e-7)
    assert np.allclose(got * LN2, want_med, rtol=1e-6)


def test_constant_power_gives_constant_floor_and_exact_weights():
    c = np.array([1.0, 4.0, 0.25, 9.0])
    rng = np.random.default_rng(0)
    ph = np.exp(2j * np.pi * rng.random((4, 50)))
    bins = (np.sqrt(c)[:, None] * ph).astype(np.complex64)
    f = N.running_median_floor(bins, 5).astype(np.float64)
    for s in range(4):
        assert np.allclose(f[s], c[s] / LN2, rtol=1e-6)
    w = N.noise_weights([f[:2], f[2:]])
    inv = 1.0 / c
    np.testing.assert_allclose(np.concatenate(w), inv / inv.mean(), rtol=1e-6)
    xw = N.whiten(bins, f)
    np.testing.assert_allclose(np.abs(xw) ** 2, LN2, rtol=1e-5)


def test_stationary_whitening_scales_2F_by_one_over_the_floor():
    """With one floor value s for every bin, whitening divides X by sqrt(s)
    and the weights are 1, so 2F is exactly the unweighted 2F divided by s."""
    w = config_mid(n_sft=12, n_sky=1, n_f=10, n_fdot=1)
    s = 3.0
    dets_w = [N.WeightedDetector(d.lat, d.lon, d.az, d.t_start, d.bins.astype(np.complex128) / math.sqrt(s),
                                 np.ones(d.n_sft))
              for d in w.detectors]
    ref = O.compute_fstat_freq_band(w.detectors, w.T, w.k_lo, w.dterms, w.bank)
    got = O.compute_fstat_freq_band(dets_w, w.T, w.k_lo, w.dterms, w.bank)
    np.testing.assert_allclose(got, ref / s, rtol=1e-10)


def test_weighted_2F_has_chi2_4_mean_on_nonstationary_noise():
    """SFT noise levels differing by up to 10x: after whitening and weighting,
    2F on noise keeps its chi^2_4 mean of about 4 (as D -> inf; D = 8 here)."""
    w = config_mid(seed=9, n_sft=60, n_sky=2, n_f=150, n_fdot=1, n_bins=220)
    rng = np.random.default_rng(4)
    dets = []
    for d in w.detectors:
        g = np.sqrt(rng.choice([1.0, 10.0], size=d.n_sft))[:, None]
        dets.append(dataclasses.replace(d, bins=(d.bins * g).astype(np.complex64)))
    wd = N.weighted_detectors(dets, 16)
    two = O.compute_fstat_freq_band(wd, w.T, w.k_lo, w.dterms, w.bank)
    assert abs(two.mean() - 4.0) < 0.25


def test_weights_recover_signal_to_noise_on_nonstationary_data():
    """A signal in noise whose level jumps 20x in half of the SFTs: the
    weighted statistic at the true template is far above the unweighted one,
    which the noisy half dilutes."""
    from workload import Injection
    w = config_mid(seed=11, n_sft=80, n_sky=1, n_f=20, n_fdot=1, n_bins=220)
    inj = Injection(w.bank.sky[0, 0], w.bank.sky[0, 1], 0.2, 0.4, 0.7, w.bank.f0 + 7 * w.bank.df, 0.0, 12.0)
    bins = O.inject(w.detectors, w.T, w.k_lo, [inj], w.bank.t_ref)
    dets = []
    for d, b in zip(w.detectors, bins):
        g = np.ones(d.n_sft)
        g[d.n_sft // 2:] = math.sqrt(20.0)
        noise = (d.bins * (g[:, None] - 1.0)).astype(np.complex64)   # extra noise in the second half
        dets.append(dataclasses.replace(d, bins=(b + noise).astype(np.complex64)))
    raw = O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank)[0, 0]
    wd = N.weighted_detectors(dets, 16)
    wgt = O.compute_fstat_freq_band(wd, w.T, w.k_lo, w.dterms, w.bank)[0, 0]
    # compare each at its own noise scale: the unweighted statistic sees a mean
    # noise level of (1 + 20)/2 per SFT, so divide it by its noise-only mean
    assert wgt[7] > 3.0 * raw[7] / 10.5


def test_noise_free_weighted_2F_matches_the_whitened_snr_closed_form():
    """Signal only, SFT alpha whitened by its own floor S_alpha and weighted by
    w_alpha ~ 1/S_alpha: at the true template (D large) the statistic is the
    whitened optimal SNR, (T^2/2) sum_alpha (a^2|c_a|^2 + b^2|c_b|^2 +
    2 a b Re(c_a c_b*)) / S_alpha."""
    from workload import Injection, TemplateBank
    w = config_mid(seed=21, n_sft=20, n_sky=1, n_f=1, n_fdot=1, n_bins=200)
    inj = Injection(0.9, -0.3, 0.35, 0.25, 1.1, (w.k_lo + 100.3) / w.T, 0.0, 10.0)
    zero = [dataclasses.replace(d, bins=np.zeros_like(d.bins)) for d in w.detectors]
    bins = O.inject(zero, w.T, w.k_lo, [inj], w.bank.t_ref)
    rng = np.random.default_rng(5)
    S = [rng.uniform(1.0, 10.0, d.n_sft) for d in w.detectors]
    inv = np.concatenate([1.0 / s for s in S])
    wd = [N.WeightedDetector(d.lat, d.lon, d.az, d.t_start, b.astype(np.complex128) / np.sqrt(s)[:, None],
                             (1.0 / s) / inv.mean()) for d, b, s in zip(w.detectors, bins, S)]
    bank = TemplateBank(np.array([[inj.alpha, inj.delta]]), inj.f, 1.0 / w.T, 1, np.zeros(1), w.bank.t_ref)
    got = O.compute_fstat_freq_band(wd, w.T, w.k_lo, 48, bank)[0, 0, 0]
    h0 = O.injection_h0(zero, w.T, inj, w.bank.t_ref)
    ca, cb = O.signal_amplitudes(inj.psi, inj.cosi, inj.phi0, h0)
    q = 0.0
    for d, s in zip(w.detectors, S):
        _, _, a, b = O.sft_timing_antenna(d, w.T, inj.alpha, inj.delta, w.bank.t_ref)
        q += np.sum((a * a * abs(ca) ** 2 + b * b * abs(cb) ** 2 + 2 * a * b * (ca * np.conj(cb)).real) / s)
    want = w.T ** 2 / 2.0 * q
    assert abs(got / want - 1.0) < 0.01, (got, want)
