"""Pins of the per-SFT frequency-coverage oracle (CPU only).

Coverage that holds every SFT must reproduce the plain oracle; coverage that
splits the SFTs must reproduce the plain oracle on each subset (a template's
A, B, C come from its own SFTs); an SFT covering nothing must be as if it
were absent; a frequency covered by nothing has 2F = 0; and on noise the
per-template normalisation keeps E[2F] = 4 where only half the SFTs remain.
"""
import math

import numpy as np

from oracle import coverage_oracle as CO
from oracle import fstat_oracle as O
from workload import DET_H, DET_L, DetectorData, TemplateBank, cn_noise, gapped_timestamps

T = 1800.0
T_REF = 8.0e8
K_LO = 180000


def _dets(seed=31, n=20, nb=90):
    out = []
    for i, g in enumerate((DET_H, DET_L)):
        t = gapped_timestamps(seed, i, T_REF, T, n)
        out.append(DetectorData(g["lat"], g["lon"], g["az"], t, cn_noise(seed, 10 + i, (n, nb))))
    return out


def _bank(n_f=24):
    sky = np.array([[1.1, 0.4], [4.0, -0.7]])
    return TemplateBank(sky=sky, f0=(K_LO + 30.3) / T, df=1.0 / T, n_f=n_f, fdot=np.array([-4e-10, 0.0]),
                        t_ref=T_REF)


def test_full_coverage_is_the_plain_oracle():
    dets, bank = _dets(), _bank()
    n = sum(len(d.t_start) for d in dets)
    got = CO.compute_fstat_coverage(dets, T, K_LO, 8, bank, np.zeros(n), np.full(n, bank.n_f))
    want = O.compute_fstat_freq_band(dets, T, K_LO, 8, bank)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)


def test_detector_split_gives_each_detector_alone():
    dets, bank = _dets(), _bank()
    n0, n1 = len(dets[0].t_start), len(dets[1].t_start)
    J = 10
    lo = np.r_[np.zeros(n0), np.full(n1, J)]
    hi = np.r_[np.full(n0, J), np.full(n1, bank.n_f)]
    got = CO.compute_fstat_coverage(dets, T, K_LO, 8, bank, lo, hi)
    only0 = O.compute_fstat_freq_band(dets[:1], T, K_LO, 8, bank)
    only1 = O.compute_fstat_freq_band(dets[1:], T, K_LO, 8, bank)
    np.testing.assert_allclose(got[..., :J], only0[..., :J], rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(got[..., J:], only1[..., J:], rtol=1e-11, atol=1e-12)


def test_sft_covering_nothing_is_absent_and_uncovered_frequency_is_zero():
    dets, bank = _dets(), _bank()
    n0, n1 = len(dets[0].t_start), len(dets[1].t_start)
    lo = np.zeros(n0 + n1)
    hi = np.full(n0 + n1, bank.n_f - 3)      # the last three frequencies: no SFT
    lo[4], hi[4] = 7, 7                       # SFT 4 of detector 0 covers nothing
    got = CO.compute_fstat_coverage(dets, T, K_LO, 8, bank, lo, hi)
    keep = np.ones(n0, bool)
    keep[4] = False
    d0 = DetectorData(dets[0].lat, dets[0].lon, dets[0].az, dets[0].t_start[keep], dets[0].bins[keep])
    want = O.compute_fstat_freq_band([d0, dets[1]], T, K_LO, 8, bank)
    np.testing.assert_allclose(got[..., :-3], want[..., :-3], rtol=1e-11, atol=1e-12)
    assert np.all(got[..., -3:] == 0.0)


def test_noise_mean_stays_four_where_half_the_sfts_remain():
    # D = 256 windows on templates 520 bins apart: independent chi^2_4 draws
    D, n_sft, nb, spacing = 256, 8, 20000, 520
    t_start = gapped_timestamps(5, 2, T_REF, T, n_sft)
    first = K_LO + D + 40
    n_f = (nb - 2 * D - 80) // spacing
    bank = TemplateBank(sky=np.array([[2.1, -0.5]]), f0=(first + 0.5) / T, df=spacing / T, n_f=n_f,
                        fdot=np.zeros(1), t_ref=T_REF)
    lo = np.zeros(n_sft)
    hi = np.where(np.arange(n_sft) < n_sft // 2, n_f, n_f // 2)   # the later SFTs stop half way
    low, high = [], []
    for seed in range(14):
        det = DetectorData(DET_L["lat"], 0.0, DET_L["az"], t_start, cn_noise(700 + seed, 3, (n_sft, nb)))
        x = CO.compute_fstat_coverage([det], T, K_LO, D, bank, lo, hi)[0, 0]
        low.append(x[:n_f // 2])
        high.append(x[n_f // 2:])
    low, high = np.concatenate(low), np.concatenate(high)
    for x in (low, high):
        assert abs(x.mean() - 4.0) < 4 * math.sqrt(8.0 / x.shape[0])


def test_full_coverage_with_noise_weights_is_the_weighted_oracle():
    # per-SFT noise weights (attribute `weights`) enter A, B, C and Fa, Fb the
    # same way in both oracles
    from oracle import noise_oracle as N
    dets = _dets(seed=41)
    rng = np.random.default_rng(4)
    dets = [DetectorData(d.lat, d.lon, d.az, d.t_start,
                         (d.bins * np.sqrt(rng.uniform(1, 5, len(d.t_start)))[:, None]).astype(np.complex64))
            for d in dets]
    wd = N.weighted_detectors(dets, 8)
    bank = _bank()
    n = sum(len(d.t_start) for d in wd)
    got = CO.compute_fstat_coverage(wd, T, K_LO, 8, bank, np.zeros(n), np.full(n, bank.n_f))
    want = O.compute_fstat_freq_band(wd, T, K_LO, 8, bank)
    np.testing.assert_allclose(got, want, rtol=1e-11, atol=1e-12)
