"""Pins of the plain-C FP64 oracle (oracle/fstat_oracle.c).

It restates the numpy oracle's arithmetic as plain loops (Listing 1's nest:
templates, then detectors, then SFTs).  Pinned by:
  * equality with the numpy oracle -- itself pinned by brute-force
    demodulation, closed forms and the chi^2_4 law -- on the tiny case and on
    a gapped two-detector case whose windows leave the stored band;
  * the noise-free closed form of a model-exact injection (Fa, Fb at the true
    template) and its D -> infinity limit rho^2;
  * planted mistakes (compiled from edited copies of the C source) that these
    pins must catch.
"""
import dataclasses
import math
import os

import numpy as np
import pytest

from oracle import c_oracle as CO
from oracle import fstat_oracle as O
from workload import (DET_H, DET_L, DetectorData, Injection, config0, config_mid, gapped_timestamps,
                      T_SFT)

T = T_SFT


def _with_signals(w):
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    return [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]


@pytest.fixture(scope="module")
def cases():
    out = []
    for w in (config0(), config_mid(n_sky=3, n_f=90)):
        dets = _with_signals(w)
        ref = O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank)
        out.append((w, dets, ref))
    return out


def _close(got, ref):
    return np.all(np.abs(got - ref) <= 1e-7 * np.abs(ref) + 1e-9)


def test_c_oracle_equals_numpy_oracle(cases):
    for w, dets, ref in cases:
        got = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank, threads=2)
        assert got.shape == ref.shape
        assert _close(got, ref), np.max(np.abs(got - ref) / (np.abs(ref) + 1e-9))


def test_c_oracle_template_indices_in_any_order(cases):
    w, dets, ref = cases[1]
    rng = np.random.default_rng(3)
    idx = rng.permutation(ref.size)[:200]
    got = CO.compute_fstat_templates(dets, w.T, w.k_lo, w.dterms, w.bank, idx, threads=3)
    assert _close(got, ref.ravel()[idx])


def test_c_oracle_noise_free_closed_form():
    """O1: Fa, Fb at the true template of a model-exact signal equal
    (T/2) sum a t (a c_a + b c_b); the C oracle returns 2F, compared with the
    closed form's combine (FP32 storage of the bins: 1e-6)."""
    w = config0()
    inj = w.injections[0]
    h0 = O.injection_h0(w.detectors, w.T, inj, w.bank.t_ref)
    dets = [DetectorData(d.lat, d.lon, d.az, d.t_start,
                         O.signal_bins(d, w.T, w.k_lo, w.n_bins, inj, h0, w.bank.t_ref).astype(np.complex64))
            for d in w.detectors]
    Fa, Fb = O.closed_form_fa_fb(dets, w.T, w.dterms, inj, h0, w.bank.t_ref)
    a_all, b_all = [], []
    for d in dets:
        _, _, a, b = O.sft_timing_antenna(d, w.T, inj.alpha, inj.delta, w.bank.t_ref)
        a_all.append(a)
        b_all.append(b)
    A, B, C, D = O.abcd(a_all, b_all)
    want = float(O.normalized(np.array([Fa]), np.array([Fb]), A, B, C, D)[0])
    bank = dataclasses.replace(w.bank, sky=np.array([[inj.alpha, inj.delta]]), f0=inj.f, n_f=1,
                               fdot=np.array([inj.fdot]))
    got = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, bank)[0, 0, 0]
    assert abs(got - want) <= 1e-6 * want
    assert 0.9 * inj.rho ** 2 < got < inj.rho ** 2


def test_c_oracle_large_dterms_recovers_rho2():
    """O1 as D -> infinity: 2F at the true template tends to rho^2."""
    rng = np.random.default_rng(11)
    n_sft, nb, D, t_ref = 30, 6000, 2900, 8.0e8
    t_start = gapped_timestamps(77, 1, t_ref, T, n_sft)
    k_lo = 180000 - nb // 2
    for geom in (DET_H, DET_L):
        inj = Injection(rng.uniform(0, 6.28), math.asin(rng.uniform(-1, 1)), rng.uniform(-0.7, 0.7),
                        rng.uniform(-1, 1), rng.uniform(0, 6.28), 100.0 + 0.37 / T, -3e-10, 12.0)
        det = DetectorData(geom["lat"], 0.0, geom["az"], t_start, np.zeros((n_sft, nb), np.complex64))
        h0 = O.injection_h0([det], T, inj, t_ref)
        det.bins = O.signal_bins(det, T, k_lo, nb, inj, h0, t_ref).astype(np.complex64)
        from workload import TemplateBank
        bank = TemplateBank(np.array([[inj.alpha, inj.delta]]), inj.f, 1.0, 1, np.array([inj.fdot]), t_ref)
        got = CO.compute_fstat_freq_band([det], T, k_lo, D, bank)[0, 0, 0]
        np.testing.assert_allclose(got, inj.rho ** 2, rtol=2e-4)


# ---------------------------------------------------------------- planted mistakes

MUTANTS = {
    "no_k0_sign": ("double sgn = (k0 & 1) ? -1.0 : 1.0;", "double sgn = 1.0;"),
    "conjugate_phase": ("ri = -sgn * sin(2.0 * PI * frac);", "ri = sgn * sin(2.0 * PI * frac);"),
    "window_shift": ("for (int n = -dterms + 1; n <= dterms; n++) {", "for (int n = -dterms + 2; n <= dterms + 1; n++) {"),
    "drop_kernel_factor": ("double s = sin(PI * kappa) / PI;", "double s = 1.0;"),
    "roemer_sign": ("out[s].dtau = (tm - t_ref) + ", "out[s].dtau = (tm - t_ref) - "),
    "swap_a_b_weights": ("double q = B * (far * far + fai * fai) + A * (fbr * fbr + fbi * fbi)",
                         "double q = A * (far * far + fai * fai) + B * (fbr * fbr + fbi * fbi)"),
    "y_arm_sign": ("w[i] = -sin(d->az) * north[i] + cos(d->az) * east[i];",
                   "w[i] = sin(d->az) * north[i] + cos(d->az) * east[i];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(tmp_path, cases, name):
    old, new = MUTANTS[name]
    with open(CO.SRC) as fh:
        src = fh.read()
    assert src.count(old) == 1, name
    path = os.path.join(tmp_path, f"{name}.c")
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    lib = CO.open_library(CO.compile_c(path, os.path.join(tmp_path, f"lib{name}.so")))
    caught = False
    for w, dets, ref in cases:
        got = CO.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank, threads=2, lib=lib)
        caught = caught or not _close(got, ref)
    assert caught, f"mutant {name} passed the equality pin"
