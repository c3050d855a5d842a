"""Pins of the FP64 oracle against what the mathematics fixes (CPU only).

Each test checks the oracle against something other than itself: closed
forms, a published antenna-pattern formula, brute-force time-domain
demodulation, the chi^2_4 noise law, exhaustive sorting.
"""
import math

import numpy as np
import pytest

from oracle import fstat_oracle as O
from workload import (DET_H, DET_L, DetectorData, TemplateBank, Injection, cn_noise,
                      gapped_timestamps, config0)

T = 1800.0
T_REF = 8.0e8


def _zero_ephemeris(monkeypatch):
    def zero(lat, lon, t):
        z = np.zeros(np.shape(t) + (3,))
        return z, z.copy()
    monkeypatch.setattr(O, "detector_position_velocity", zero)


# ---------------------------------------------------------------- kinematics

def test_orbit_and_rotation_closed_forms():
    t = T_REF + np.linspace(0, 3e7, 101)
    r, v = O.detector_position_velocity(DET_H["lat"], 0.0, t)
    # Earth-centre part: |r_orb| = AU, |v_orb| = 2 pi AU / year
    r_c, v_c = O.detector_position_velocity(math.pi / 2, 0.0, t)   # pole: rotation adds R_E z only
    r_orb = r_c - np.array([0, 0, O.EARTH_R])
    np.testing.assert_allclose(np.linalg.norm(r_orb, axis=1), O.AU_M, rtol=1e-13)
    np.testing.assert_allclose(np.linalg.norm(v_c, axis=1), 2 * math.pi * O.AU_M / O.YEAR_S, rtol=1e-13)
    # rotation: |r - r_orb| = R_E, speed R_E Omega cos(lat)
    rr = r - r_orb
    # (the subtraction of AU-sized vectors leaves ~1e-5 m of FP64 rounding)
    np.testing.assert_allclose(np.linalg.norm(rr, axis=1), O.EARTH_R, rtol=1e-11)
    vr = v - v_c
    np.testing.assert_allclose(np.linalg.norm(vr, axis=1),
                               O.EARTH_R * O.SIDEREAL_W * math.cos(DET_H["lat"]), rtol=1e-10)
    # orbit lies in the ecliptic: normal (0, -sin eps, cos eps)
    nrm = np.array([0.0, -math.sin(O.OBLIQUITY), math.cos(O.OBLIQUITY)])
    assert np.max(np.abs(r_orb @ nrm)) < 1e-4 * O.AU_M * 1e-6


def test_velocity_is_derivative_of_position():
    t = T_REF + np.linspace(0, 3e7, 37)
    h = 0.5
    for lat in (DET_H["lat"], DET_L["lat"]):
        r1, _ = O.detector_position_velocity(lat, 0.3, t - h)
        r2, _ = O.detector_position_velocity(lat, 0.3, t + h)
        _, v = O.detector_position_velocity(lat, 0.3, t)
        fd = (r2 - r1) / (2 * h)
        np.testing.assert_allclose(fd, v, atol=1e-6 * np.max(np.abs(v)))


def test_tdot_is_derivative_of_dtau():
    det = DetectorData(DET_L["lat"], DET_L["lon"], DET_L["az"], T_REF + T * np.arange(0, 2000, 97.0),
                       np.zeros((21, 1), np.complex64))
    h = 1.0
    d1 = DetectorData(det.lat, det.lon, det.az, det.t_start - h, det.bins)
    d2 = DetectorData(det.lat, det.lon, det.az, det.t_start + h, det.bins)
    for alpha, delta in [(0.3, 0.9), (4.0, -1.2), (2.0, 0.0)]:
        dt1, _, _, _ = O.sft_timing_antenna(d1, T, alpha, delta, T_REF)
        dt2, _, _, _ = O.sft_timing_antenna(d2, T, alpha, delta, T_REF)
        _, tdot, _, _ = O.sft_timing_antenna(det, T, alpha, delta, T_REF)
        np.testing.assert_allclose((dt2 - dt1) / (2 * h), tdot, atol=1e-9)
        assert np.all(np.abs(tdot - 1) < 1.1e-4)


def test_roemer_delay_bounds_and_pole():
    det = DetectorData(DET_H["lat"], 0.0, DET_H["az"], T_REF + T * np.arange(0, 20000, 10.0),
                       np.zeros((2000, 1), np.complex64))
    tm = det.t_start + T / 2
    # ecliptic pole: orbital Roemer delay vanishes, only the rotation term remains
    pole = O.sky_unit_vector(-math.pi / 2, math.pi / 2 - O.OBLIQUITY)
    dtau, _, _, _ = O.sft_timing_antenna(det, T, -math.pi / 2, math.pi / 2 - O.OBLIQUITY, T_REF)
    roemer = dtau - (tm - T_REF)
    assert np.max(np.abs(roemer)) <= O.EARTH_R / O.C_LIGHT * (1 + 1e-9)
    # in the ecliptic plane the amplitude reaches AU/c
    dtau, _, _, _ = O.sft_timing_antenna(det, T, 0.0, 0.0, T_REF)
    roemer = dtau - (tm - T_REF)
    assert np.max(np.abs(roemer)) > 0.99 * O.AU_M / O.C_LIGHT
    assert np.max(np.abs(roemer)) <= (O.AU_M + O.EARTH_R) / O.C_LIGHT * (1 + 1e-12)
    del pole


# ---------------------------------------------------------------- antenna patterns

def _jks_ab(lat, gamma, alpha, delta, lst):
    """Jaranowski-Krolak-Schutz (PRD 58, 063001, 1998) antenna coefficients of an
    interferometer with perpendicular arms; gamma measured counter-clockwise
    from East to the arms' bisector."""
    h = alpha - lst
    s2g, c2g = math.sin(2 * gamma), math.cos(2 * gamma)
    a = (s2g * (3 - math.cos(2 * lat)) * (3 - np.cos(2 * delta)) * np.cos(2 * h) / 16
         - c2g * math.sin(lat) * (3 - np.cos(2 * delta)) * np.sin(2 * h) / 4
         + s2g * math.sin(2 * lat) * np.sin(2 * delta) * np.cos(h) / 4
         - c2g * math.cos(lat) * np.sin(2 * delta) * np.sin(h) / 2
         + 3 * s2g * math.cos(lat) ** 2 * np.cos(delta) ** 2 / 4)
    b = (c2g * math.sin(lat) * np.sin(delta) * np.cos(2 * h)
         + s2g * (3 - math.cos(2 * lat)) * np.sin(delta) * np.sin(2 * h) / 4
         + c2g * math.cos(lat) * np.cos(delta) * np.cos(h)
         + s2g * math.sin(2 * lat) * np.cos(delta) * np.sin(h) / 2)
    return a, b


@pytest.mark.parametrize("geom", [DET_H, DET_L, dict(lat=-0.4, lon=1.3, az=2.5)])
def test_antenna_matches_jks(geom):
    rng = np.random.default_rng(7)
    t = T_REF + rng.uniform(0, 3e7, 200)
    alpha = rng.uniform(0, 2 * math.pi, 200)
    delta = np.arcsin(rng.uniform(-1, 1, 200))
    Dt = O.detector_tensor(geom["lat"], geom["lon"], geom["az"], t)
    a, b = O.antenna_ab(Dt, alpha, delta)
    lst = geom["lon"] + O.SIDEREAL_W * t
    aj, bj = _jks_ab(geom["lat"], math.pi / 4 - geom["az"], alpha, delta, lst)
    # one fixed convention: the oracle's + polarisation axis is JKS's rotated by 90 degrees
    np.testing.assert_allclose(a, -aj, atol=2e-11)
    np.testing.assert_allclose(b, bj, atol=2e-11)


def test_antenna_rotation_invariance_and_bounds():
    rng = np.random.default_rng(8)
    t = T_REF + rng.uniform(0, 3e7, 50)
    alpha = rng.uniform(0, 2 * math.pi, 50)
    delta = np.arcsin(rng.uniform(-1, 1, 50))
    Dt = O.detector_tensor(DET_H["lat"], 0.0, DET_H["az"], t)
    a, b = O.antenna_ab(Dt, alpha, delta)
    for psi in np.linspace(0, math.pi, 7):
        fp = a * math.cos(2 * psi) + b * math.sin(2 * psi)
        fx = b * math.cos(2 * psi) - a * math.sin(2 * psi)
        np.testing.assert_allclose(fp ** 2 + fx ** 2, a ** 2 + b ** 2, rtol=1e-12)
    assert np.all(a ** 2 + b ** 2 <= 1 + 1e-12)
    # source at zenith of the detector: a^2 + b^2 = 1 (full response)
    tt = np.array([T_REF])
    lst = O.SIDEREAL_W * tt
    Dz = O.detector_tensor(DET_H["lat"], 0.0, DET_H["az"], tt)
    az_, bz_ = O.antenna_ab(Dz, lst, np.array([DET_H["lat"]]))
    np.testing.assert_allclose(az_ ** 2 + bz_ ** 2, 1.0, rtol=1e-12)


def test_detector_tensor_structure():
    t = T_REF + np.array([0.0, 1e5, 3e6])
    Dt = O.detector_tensor(DET_L["lat"], 0.2, DET_L["az"], t)
    np.testing.assert_allclose(Dt, np.swapaxes(Dt, -1, -2), atol=1e-15)
    np.testing.assert_allclose(np.trace(Dt, axis1=-2, axis2=-1), 0.0, atol=1e-15)
    # local vertical is in the kernel of D
    phi = 0.2 + O.SIDEREAL_W * t
    up = np.stack([math.cos(DET_L["lat"]) * np.cos(phi), math.cos(DET_L["lat"]) * np.sin(phi),
                   math.sin(DET_L["lat"]) * np.ones_like(phi)], -1)
    np.testing.assert_allclose(np.einsum("...ij,...j->...i", Dt, up), 0.0, atol=1e-15)


# ---------------------------------------------------------------- demodulation

def _brute_force_case(monkeypatch, doppler, f_s, df_off, fdot=0.0, N=4096, nsft=4):
    """Complex time series of three tones, SFTs by the DFT definition, and the
    matched filter sum_j a x(t_j) e^{-i Phi(t_j)} dt over the unsplit series."""
    t_start = T_REF + T * np.array([0.0, 1.0, 3.0, 4.0])[:nsft]
    alpha, delta = 1.0, 0.3
    dt = T / N
    nvec = O.sky_unit_vector(alpha, delta)
    ephem = O.detector_position_velocity

    def tau(t):
        if not doppler:
            return t - T_REF
        r, _ = ephem(DET_H["lat"], DET_H["lon"], t)
        return (t - T_REF) + r @ nvec / O.C_LIGHT

    tones = [(f_s + 0.3 / T, 1.0 + 0.5j), (f_s + 2.7 / T, -0.4 + 0.2j), (f_s - 5.1 / T, 0.3j)]
    kc = int(round(f_s * T))
    nb = N + 64
    k_lo = kc - N // 2 - 32
    bins = np.zeros((nsft, nb), np.complex128)
    f_t = f_s + df_off
    Dt = O.detector_tensor(DET_H["lat"], DET_H["lon"], DET_H["az"], t_start + T / 2)
    a, b = O.antenna_ab(Dt, alpha, delta)
    Fa_bf = 0.0
    Fb_bf = 0.0
    for s in range(nsft):
        tj = t_start[s] + dt * np.arange(N)
        tt = tau(tj)
        x = sum(A * np.exp(2j * math.pi * (f * tt + 0.5 * fdot * tt * tt)) for f, A in tones)
        X = dt * np.fft.fft(x)
        bins[s] = X[(k_lo + np.arange(nb)) % N]
        m = np.sum(x * np.exp(-2j * math.pi * (f_t * tt + 0.5 * fdot * tt * tt))) * dt
        Fa_bf += a[s] * m
        Fb_bf += b[s] * m
    scale = T * np.sum(np.abs(a) + np.abs(b)) * sum(abs(A) for _, A in tones)
    det = DetectorData(DET_H["lat"], DET_H["lon"], DET_H["az"], t_start, bins)
    if not doppler:
        _zero_ephemeris(monkeypatch)
    Fa, Fb, _, _ = O.compute_fa_fb(det, T, k_lo, N // 2, alpha, delta, np.array([f_t]),
                                   np.array([fdot]), T_REF)
    return Fa[0], Fb[0], Fa_bf, Fb_bf, scale


@pytest.mark.parametrize("df_off", [0.0, 0.3 / T, 1.37 / T, -2.6 / T])
@pytest.mark.parametrize("f_s", [10.0, 100.0])
def test_brute_force_demodulation_linear_phase(monkeypatch, f_s, df_off):
    """No Doppler, no spindown: the phase is exactly linear inside each SFT, so
    the SFT method with D = N/2 equals the time-domain sum up to the
    discrete-vs-continuous kernel (O(1/N))."""
    Fa, Fb, Fa_bf, Fb_bf, scale = _brute_force_case(monkeypatch, False, f_s, df_off)
    assert abs(Fa - Fa_bf) < 1e-3 * scale
    assert abs(Fb - Fb_bf) < 1e-3 * scale


@pytest.mark.parametrize("df_off", [0.0, 0.3 / T, -1.1 / T])
def test_brute_force_demodulation_with_doppler(monkeypatch, df_off):
    """Doppler on: the method linearises the phase about each SFT midpoint;
    the curvature left inside an 1800 s SFT at 10 Hz is ~5e-4 cycles."""
    Fa, Fb, Fa_bf, Fb_bf, scale = _brute_force_case(monkeypatch, True, 10.0, df_off, fdot=-1e-9)
    assert abs(Fa - Fa_bf) < 1e-2 * scale
    assert abs(Fb - Fb_bf) < 1e-2 * scale


def test_kappa_zero_reduces_to_bin_sum(monkeypatch):
    """A template exactly on a bin with no Doppler: each SFT term is the bin
    itself, (-1)^k0 e^{-i Phi} X_k0 (the exact limit of the Dirichlet kernel)."""
    _zero_ephemeris(monkeypatch)
    rng = np.random.default_rng(3)
    t_start = T_REF + T * np.array([0.0, 2.0, 5.0, 6.0, 9.0])
    nb = 40
    k_lo = 180000
    bins = (rng.standard_normal((5, nb)) + 1j * rng.standard_normal((5, nb))).astype(np.complex64)
    det = DetectorData(DET_H["lat"], 0.0, DET_H["az"], t_start, bins)
    k = 180017
    f = k / T
    Fa, Fb, a, b = O.compute_fa_fb(det, T, k_lo, 8, 0.7, -0.2, np.array([f]), np.array([0.0]), T_REF)
    tm = t_start + T / 2
    z = (-1.0) ** k * np.exp(-2j * math.pi * f * (tm - T_REF)) * bins[:, k - k_lo].astype(np.complex128)
    # f dtau ~ 1.6e6 cycles: FP64 leaves ~4e-10 cycles of phase rounding
    np.testing.assert_allclose(Fa[0], np.sum(a * z), rtol=1e-8)
    np.testing.assert_allclose(Fb[0], np.sum(b * z), rtol=1e-8)


def test_kappa_limit_is_continuous():
    """Just above the kappa threshold the full Dirichlet sum equals the limit
    used below it (the sum is continuous at integer kappa_hat)."""
    rng = np.random.default_rng(4)
    row = (rng.standard_normal(64) + 1j * rng.standard_normal(64)).astype(np.complex64)
    k_lo = 1000
    kh = np.array([1030.0, 1030.0 + 2.0 ** -23, 1030.0 + 1e-6, 1031.0 - 1e-7])
    z = O.some_calculations(row, k_lo, kh, np.zeros(4), 8)
    np.testing.assert_allclose(z[1], z[0], rtol=1e-6)
    np.testing.assert_allclose(z[2], z[0], rtol=1e-5)
    z1 = O.some_calculations(row, k_lo, np.array([1031.0]), np.zeros(1), 8)
    np.testing.assert_allclose(z[3], z1[0], rtol=1e-5)


# ---------------------------------------------------------------- injections and 2F

def _noise_free(w, inj):
    dets = []
    h0 = O.injection_h0(w.detectors, w.T, inj, w.bank.t_ref)
    for d in w.detectors:
        sb = O.signal_bins(d, w.T, w.k_lo, w.n_bins, inj, h0, w.bank.t_ref)
        dets.append(DetectorData(d.lat, d.lon, d.az, d.t_start, sb))
    return dets, h0


def test_closed_form_fa_fb_noise_free():
    """O1: noise-free model-exact injection; demodulated Fa, Fb at the true
    template equal (T/2) sum a t (a c_a + b c_b) (t the window's kernel mass)."""
    w = config0()
    inj = w.injections[0]
    dets, h0 = _noise_free(w, inj)
    twoF, parts = O.compute_fstat(dets, w.T, w.k_lo, w.dterms, inj.alpha, inj.delta,
                                  np.array([inj.f]), np.array([inj.fdot]), w.bank.t_ref, return_parts=True)
    Fa, Fb = O.closed_form_fa_fb(dets, w.T, w.dterms, inj, h0, w.bank.t_ref)
    np.testing.assert_allclose(parts["Fa"][0], Fa, rtol=1e-10)
    np.testing.assert_allclose(parts["Fb"][0], Fb, rtol=1e-10)
    assert 0.9 * inj.rho ** 2 < twoF[0] < inj.rho ** 2


def test_large_dterms_recovers_rho2():
    """O1 as D -> infinity: the noise-free 2F at the true template tends to
    rho^2 = (T^2/2) c^H M c, computed without the demodulation or combine."""
    rng = np.random.default_rng(11)
    n_sft, nb, D = 30, 6000, 2900
    t_start = gapped_timestamps(77, 1, T_REF, T, n_sft)
    k_lo = 180000 - nb // 2
    for geom in (DET_H, DET_L):
        inj = Injection(rng.uniform(0, 6.28), math.asin(rng.uniform(-1, 1)), rng.uniform(-0.7, 0.7),
                        rng.uniform(-1, 1), rng.uniform(0, 6.28), 100.0 + 0.37 / T, -3e-10, 12.0)
        det = DetectorData(geom["lat"], 0.0, geom["az"], t_start, np.zeros((n_sft, nb), np.complex64))
        h0 = O.injection_h0([det], T, inj, T_REF)
        det.bins = O.signal_bins(det, T, k_lo, nb, inj, h0, T_REF)
        twoF = O.compute_fstat([det], T, k_lo, D, inj.alpha, inj.delta, np.array([inj.f]),
                               np.array([inj.fdot]), T_REF)
        np.testing.assert_allclose(twoF[0], inj.rho ** 2, rtol=2e-4)


def test_noisy_injection_recovers_4_plus_rho2():
    """O2: noisy injection, 2F at the true template within 4 sigma of 4 + rho^2."""
    w = config0()
    inj = w.injections[0]
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [DetectorData(d.lat, d.lon, d.az, d.t_start, b) for d, b in zip(w.detectors, bins)]
    twoF = O.compute_fstat(dets, w.T, w.k_lo, w.dterms, inj.alpha, inj.delta,
                           np.array([inj.f]), np.array([0.0]), w.bank.t_ref)[0]
    rho2 = inj.rho ** 2
    assert abs(twoF - 4 - rho2) < 4 * math.sqrt(8 + 4 * rho2)


def _independent_noise_draws(D, n_seeds, nb, spacing, n_sft=6):
    """2F at templates whose Dirichlet windows use disjoint bins: independent draws."""
    t_start = gapped_timestamps(5, 2, T_REF, T, n_sft)
    k_lo = 180000
    alpha, delta = 2.1, -0.5
    out = []
    preds = []
    for seed in range(n_seeds):
        bins = cn_noise(900 + seed, 3, (n_sft, nb))
        det = DetectorData(DET_L["lat"], 0.0, DET_L["az"], t_start, bins)
        kk = np.arange(k_lo + D + 40, k_lo + nb - D - 40, spacing)
        f = (kk + 0.5) / T
        twoF, parts = O.compute_fstat([det], T, k_lo, D, alpha, delta, f, np.zeros_like(f), T_REF,
                                      return_parts=True)
        out.append(twoF)
        if seed == 0:
            dtau, tdot, a, b = O.sft_timing_antenna(det, T, alpha, delta, T_REF)
            for fi in f[:3]:
                _, kh = O.phase_and_kappa(fi, 0.0, dtau, tdot, T)
                kap = kh - np.floor(kh)
                t = sum(np.sin(math.pi * kap) ** 2 / (math.pi ** 2 * (kap - n) ** 2)
                        for n in range(-D + 1, D + 1))
                A, B, C, Dd = parts["A"], parts["B"], parts["C"], parts["D"]
                preds.append(2 * (B * np.sum(a * a * t) + A * np.sum(b * b * t)
                                  - 2 * C * np.sum(a * b * t)) / Dd)
    return np.concatenate(out), np.array(preds)


def test_noise_mean_matches_finite_dterms_prediction():
    """O3: on pure noise E[2F] = 2 (B sum a^2 t + A sum b^2 t - 2 C sum ab t) / D
    with t the window's kernel mass (-> 4 as D -> infinity)."""
    x, preds = _independent_noise_draws(8, 6, 16000, 20)
    assert x.shape[0] > 4000
    se = math.sqrt(8.0 / x.shape[0])
    assert np.all(np.abs(preds - 4.0) < 0.1)
    assert abs(x.mean() - preds.mean()) < 4 * se
    assert np.all(x >= 0)


def test_noise_is_chi2_4_for_large_dterms():
    """O3: with D = 256 the noise-only 2F follows chi^2 with 4 degrees of freedom."""
    from scipy import stats
    x, _ = _independent_noise_draws(256, 12, 60000, 520, n_sft=4)
    assert x.shape[0] > 1000
    assert stats.kstest(x, "chi2", args=(4,)).pvalue > 1e-3
    assert abs(x.mean() - 4.0) < 4 * math.sqrt(8.0 / x.shape[0])


# ---------------------------------------------------------------- invariants

def _small_two_det(seed=21):
    dets = []
    for i, g in enumerate((DET_H, DET_L)):
        t = gapped_timestamps(seed, i, T_REF, T, 25)
        dets.append(DetectorData(g["lat"], g["lon"], g["az"], t, cn_noise(seed, 10 + i, (25, 90))))
    return dets


def test_permutation_and_independence_invariants():
    dets = _small_two_det()
    k_lo = 180000
    f = 100.0 + (30 + np.arange(25) * 1.3) / T
    fd = np.full_like(f, -4e-10)
    ref = O.compute_fstat(dets, T, k_lo, 8, 1.1, 0.4, f, fd, T_REF)
    # permute SFTs within each detector and the detector order
    rng = np.random.default_rng(2)
    pd = []
    for d in dets[::-1]:
        p = rng.permutation(d.n_sft)
        pd.append(DetectorData(d.lat, d.lon, d.az, d.t_start[p], d.bins[p]))
    perm = O.compute_fstat(pd, T, k_lo, 8, 1.1, 0.4, f, fd, T_REF)
    np.testing.assert_allclose(perm, ref, rtol=1e-11)
    # templates are independent: one template alone equals it inside the batch
    for i in (0, 7, 24):
        one = O.compute_fstat(dets, T, k_lo, 8, 1.1, 0.4, f[i:i + 1], fd[i:i + 1], T_REF)
        assert one[0] == ref[i]
    assert np.all(ref >= 0)
    # D = AB - C^2 > 0 (Cauchy-Schwarz, a and b not proportional)
    _, parts = O.compute_fstat(dets, T, k_lo, 8, 1.1, 0.4, f, fd, T_REF, return_parts=True)
    assert parts["D"] > 0


def test_template_indexing_round_trip():
    from workload import template_index, template_params
    bank = TemplateBank(np.zeros((7, 2)), 100.0, 1 / T, 13, np.zeros(5), T_REF)
    for s, d, f in [(0, 0, 0), (6, 4, 12), (3, 2, 7)]:
        i = template_index(bank, s, d, f)
        assert tuple(int(x) for x in template_params(bank, i)) == (s, d, f)


# ---------------------------------------------------------------- toplist

def test_toplist_exhaustive_with_ties():
    rng = np.random.default_rng(9)
    v = rng.integers(0, 30, 500).astype(np.float64) / 4.0     # many exact ties
    for k in (1, 10, 77, 500):
        idx, val = O.toplist(v, k)
        ref = sorted(range(v.shape[0]), key=lambda i: (-v[i], i))[:k]
        assert list(idx) == ref
        assert list(val) == [v[i] for i in ref]
