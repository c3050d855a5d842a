"""Planted mistakes in the oracle (on the CPU) must be caught by its pins.

Each mutant wraps one oracle function with a plausible error -- a dropped
sign, a conjugated phase, a window off by one bin, swapped A/B, a flipped
Roemer delay, a dropped kernel factor -- and the test asserts that the
matching pin no longer holds.
"""
import math

import numpy as np
import pytest

from oracle import fstat_oracle as O
import tests.test_oracle_pins as P

T = P.T


def _brute_force_error(monkeypatch, doppler, df_off):
    Fa, Fb, Fa_bf, Fb_bf, scale = P._brute_force_case(monkeypatch, doppler, 10.0, df_off,
                                                      fdot=-1e-9 if doppler else 0.0)
    return max(abs(Fa - Fa_bf), abs(Fb - Fb_bf)) / scale


def _mutant_no_k0_sign(orig):
    def f(bins_row, k_lo, kh, phase, D):
        z = orig(bins_row, k_lo, kh, phase, D)
        return z * (1.0 - 2.0 * (np.floor(kh).astype(np.int64) & 1))
    return f


def _mutant_conj_phase(orig):
    def f(bins_row, k_lo, kh, phase, D):
        return orig(bins_row, k_lo, kh, -np.asarray(phase), D)
    return f


def _mutant_window_shift(orig):
    def f(bins_row, k_lo, kh, phase, D):
        return orig(bins_row, k_lo + 1, kh, phase, D)
    return f


def _mutant_drop_kernel_factor(orig):
    def f(bins_row, k_lo, kh, phase, D):
        kap = np.asarray(kh) - np.floor(kh)
        z = orig(bins_row, k_lo, kh, phase, D)
        return np.where(kap < O.KAPPA_LIMIT, z, z / (np.sin(math.pi * kap) / math.pi))
    return f


@pytest.mark.parametrize("mutant", [_mutant_no_k0_sign, _mutant_conj_phase, _mutant_window_shift,
                                    _mutant_drop_kernel_factor])
def test_brute_force_pin_catches_sft_term_mutants(monkeypatch, mutant):
    assert _brute_force_error(monkeypatch, False, 0.3 / T) < 1e-3
    monkeypatch.setattr(O, "some_calculations", mutant(O.some_calculations))
    worst = max(_brute_force_error(monkeypatch, False, off) for off in (0.3 / T, 1.37 / T))
    assert worst > 1e-2


def test_doppler_pin_catches_flipped_roemer_delay(monkeypatch):
    orig = O.sft_timing_antenna

    def flipped(det, T_, alpha, delta, t_ref):
        dtau, tdot, a, b = orig(det, T_, alpha, delta, t_ref)
        tm = np.asarray(det.t_start) + 0.5 * T_
        return 2 * (tm - t_ref) - dtau, 2.0 - tdot, a, b

    monkeypatch.setattr(O, "sft_timing_antenna", flipped)
    assert _brute_force_error(monkeypatch, True, 0.3 / T) > 1e-1


def test_rho2_pin_catches_swapped_combine(monkeypatch):
    orig = O.normalized

    def swapped(Fa, Fb, A, B, C, D, sigma2=1.0):
        return orig(Fa, Fb, B, A, C, D, sigma2)

    monkeypatch.setattr(O, "normalized", swapped)
    with pytest.raises(AssertionError):
        P.test_large_dterms_recovers_rho2()


def test_rho2_pin_catches_dropped_cross_term(monkeypatch):
    orig = O.normalized

    def dropped(Fa, Fb, A, B, C, D, sigma2=1.0):
        return orig(Fa, Fb, A, B, 0.0, D, sigma2)

    monkeypatch.setattr(O, "normalized", dropped)
    with pytest.raises(AssertionError):
        P.test_large_dterms_recovers_rho2()


def test_noise_pin_catches_wrong_normalisation(monkeypatch):
    orig = O.normalized
    monkeypatch.setattr(O, "normalized", lambda Fa, Fb, A, B, C, D, s=1.0: orig(Fa, Fb, A, B, C, D, 2.0))
    with pytest.raises(AssertionError):
        P.test_noise_mean_matches_finite_dterms_prediction()


# ------------------------------------------------------------ stack-slide

def _slide_mutant(kind):
    from oracle import semicoherent_oracle as S
    orig = S.slide_constants

    def f(f0, df, fdot, t_ref, f0_s, df_s, t_s):
        if kind == "sign":          # slide the wrong way
            return orig(f0, df, fdot, t_s, f0_s, df_s, t_ref)
        if kind == "no_slide":      # forget the spindown term
            return orig(f0, df, np.zeros_like(np.asarray(fdot, dtype=np.float64)), t_ref, f0_s, df_s, t_s)
        A_fx, B_fx = orig(f0, df, fdot, t_ref, f0_s, df_s, t_s)
        if kind == "truncate":      # nearest bin taken as floor
            return A_fx - (1 << 31), B_fx
        if kind == "inverse_ratio":  # df_s / df instead of df / df_s
            return A_fx, int(round(2.0 ** 64 / B_fx))
        raise ValueError(kind)
    return f


@pytest.mark.parametrize("kind", ["sign", "no_slide", "truncate", "inverse_ratio"])
def test_stack_slide_pins_catch_mutants(monkeypatch, kind):
    from oracle import semicoherent_oracle as S
    import tests.test_oracle_semicoherent as SP
    pins = [SP.test_exactly_representable_slides_move_by_whole_bins, SP.test_half_bin_slides_round_up,
            SP.test_finer_semicoherent_grid_maps_four_to_one,
            SP.test_signal_with_spindown_peaks_at_its_template_only_when_slid]
    for pin in pins:
        pin()
    monkeypatch.setattr(S, "slide_constants", _slide_mutant(kind))
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, kind


# ------------------------------------------------------------ frequency coverage

def _coverage_mutant(kind):
    from oracle import coverage_oracle as CO
    orig = CO.compute_fstat_coverage

    def f(dets, T, k_lo, dterms, bank, j_lo, j_hi, sky_indices=None):
        j_lo, j_hi = np.asarray(j_lo), np.asarray(j_hi)
        if kind == "inclusive_end":       # [j_lo, j_hi] instead of [j_lo, j_hi)
            return orig(dets, T, k_lo, dterms, bank, j_lo, j_hi + 1, sky_indices)
        if kind == "ignored":             # coverage dropped
            return orig(dets, T, k_lo, dterms, bank, np.zeros_like(j_lo), np.full_like(j_hi, bank.n_f), sky_indices)
        if kind == "off_by_one_start":    # (j_lo, j_hi)
            return orig(dets, T, k_lo, dterms, bank, j_lo + 1, j_hi, sky_indices)
        raise ValueError(kind)
    return f


@pytest.mark.parametrize("kind", ["inclusive_end", "ignored", "off_by_one_start"])
def test_coverage_pins_catch_mutants(monkeypatch, kind):
    from oracle import coverage_oracle as CO
    import tests.test_oracle_coverage as CP
    pins = [CP.test_detector_split_gives_each_detector_alone,
            CP.test_sft_covering_nothing_is_absent_and_uncovered_frequency_is_zero]
    for pin in pins:
        pin()
    monkeypatch.setattr(CO, "compute_fstat_coverage", _coverage_mutant(kind))
    failed = 0
    for pin in pins:
        try:
            pin()
        except AssertionError:
            failed += 1
    assert failed >= 1, kind
