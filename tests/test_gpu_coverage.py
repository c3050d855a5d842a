"""Per-SFT frequency coverage through the C ABI against the coverage oracle.

Ragged coverage (SFTs covering everything, nothing, or random sub-ranges
whose edges fall inside thread tiles) must match the FP64 oracle element by
element in every form; switching it off must restore the plain result.
"""
import dataclasses

import numpy as np
import pytest

from oracle import coverage_oracle as CO
from oracle import fstat_oracle as O
from workload import config_mid

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3


def _ragged(n_sft, n_f, seed):
    rng = np.random.default_rng(seed)
    lo = np.zeros(n_sft, np.int32)
    hi = np.full(n_sft, n_f, np.int32)
    kind = rng.random(n_sft)
    none = kind < 0.15
    part = kind >= 0.55
    lo[none] = hi[none] = rng.integers(0, n_f, none.sum())
    lo[part] = rng.integers(-10, n_f, part.sum())
    hi[part] = np.minimum(lo[part] + rng.integers(1, n_f, part.sum()), n_f + 10)
    return lo, hi


@pytest.fixture(scope="module")
def case():
    w = config_mid(n_sky=4, n_f=150, n_fdot=3)
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    dets = [dataclasses.replace(d, bins=b) for d, b in zip(w.detectors, bins)]
    lo, hi = _ragged(w.n_sft_total, w.bank.n_f, 11)
    ref = CO.compute_fstat_coverage(dets, w.T, w.k_lo, w.dterms, w.bank, lo, hi).ravel()
    return w, bins, lo, hi, ref


FORMS = [("c64", False, "auto"), ("c64", False, "farpoly"), ("c64", False, "direct"), ("c64", True, "direct"),
         ("f16", False, "auto")]


@pytest.mark.parametrize("form,kahan,algo", FORMS)
def test_coverage_matches_oracle(lib, case, form, kahan, algo):
    w, bins, lo, hi, ref = case
    g = lib.FStat(0, topk=10, bins_form=form, kahan=kahan, algo=algo)
    try:
        g.load_workload(w, bins_override=bins)
        lib.fstat_set_coverage(g.ctx, lo, hi)
        g.compute()
        got = g.twoF().astype(np.float64)
        assert g.error_flags() == 0
        if algo == "farpoly":
            assert g.plan()["variant"] >= 100   # the ring form took the coverage
        if form == "c64":
            assert np.all(np.abs(got - ref) <= REL * ref + ABS), np.max(np.abs(got - ref))
        else:                                    # 16-bit storage: its format's level
            assert np.max(np.abs(got - ref) / (ref + 1.0)) < 5e-3
    finally:
        g.close()


def test_coverage_uncovered_frequencies_are_zero_and_off_restores_plain(lib, case):
    w, bins, _, _, _ = case
    n = w.n_sft_total
    lo = np.zeros(n, np.int32)
    hi = np.full(n, w.bank.n_f - 7, np.int32)    # the last seven frequencies: no SFT
    g = lib.FStat(0, topk=10)
    try:
        g.load_workload(w, bins_override=bins)
        g.compute()
        plain = g.twoF().reshape(w.bank.n_sky, w.bank.n_fdot, w.bank.n_f).copy()
        lib.fstat_set_coverage(g.ctx, lo, hi)
        g.compute()
        got = g.twoF().reshape(plain.shape)
        assert g.error_flags() == 0
        assert np.all(got[..., -7:] == 0.0)
        np.testing.assert_array_equal(got[..., :-7], plain[..., :-7])   # full coverage there: same sums
        lib.fstat_set_coverage(g.ctx, None, None)
        g.compute()
        np.testing.assert_array_equal(g.twoF().reshape(plain.shape), plain)
    finally:
        g.close()


def test_coverage_detector_split_matches_single_detectors(lib, case):
    w, bins, _, _, _ = case
    n0, n1 = (d.n_sft for d in w.detectors)
    J = 61
    lo = np.r_[np.zeros(n0), np.full(n1, J)].astype(np.int32)
    hi = np.r_[np.full(n0, J), np.full(n1, w.bank.n_f)].astype(np.int32)
    ref = [O.compute_fstat_freq_band([dataclasses.replace(w.detectors[i], bins=bins[i])], w.T, w.k_lo, w.dterms,
                                     w.bank) for i in range(2)]
    g = lib.FStat(0, topk=10)
    try:
        g.load_workload(w, bins_override=bins)
        lib.fstat_set_coverage(g.ctx, lo, hi)
        g.compute()
        got = g.twoF().reshape(w.bank.n_sky, w.bank.n_fdot, w.bank.n_f).astype(np.float64)
        for part, r in ((slice(0, J), ref[0]), (slice(J, None), ref[1])):
            assert np.all(np.abs(got[..., part] - r[..., part]) <= REL * r[..., part] + ABS)
    finally:
        g.close()


def test_coverage_errors(lib, case):
    w, bins, lo, hi, _ = case
    g = lib.FStat(0, topk=10)
    try:
        with pytest.raises(lib.FstatError) as e:   # before any SFT
            lib.fstat_set_coverage(g.ctx, lo, hi)
        assert e.value.code == lib.FSTAT_ESTATE
        g.load_workload(w, bins_override=bins)
        with pytest.raises(lib.FstatError) as e:   # wrong SFT count
            lib.fstat_set_coverage(g.ctx, lo[:-1], hi[:-1])
        assert e.value.code == lib.FSTAT_EINVAL
        bad = hi.copy()
        bad[3] = lo[3] - 1
        with pytest.raises(lib.FstatError) as e:   # j_lo > j_hi
            lib.fstat_set_coverage(g.ctx, lo, bad)
        assert e.value.code == lib.FSTAT_EINVAL
        lib.fstat_set_coverage(g.ctx, lo, hi)      # and the context still computes
        g.compute()
        assert g.error_flags() == 0
    finally:
        g.close()


def test_coverage_with_noise_floor_and_weights(lib):
    from oracle import noise_oracle as N
    import tests.test_gpu_noise as TN
    w, scaled, dets = TN._case(seed=33)
    lo, hi = _ragged(w.n_sft_total, w.bank.n_f, 12)
    ref = CO.compute_fstat_coverage(N.weighted_detectors(dets, TN.W), w.T, w.k_lo, w.dterms, w.bank, lo, hi).ravel()
    g = lib.FStat(0, dterms=w.dterms, topk=10)
    try:
        g.load_workload(w, bins_override=scaled)
        lib.fstat_set_noise_floor(g.ctx, TN.W)
        lib.fstat_set_coverage(g.ctx, lo, hi)
        g.compute()
        got = g.twoF().astype(np.float64)
        assert g.error_flags() == 0
    finally:
        g.close()
    assert np.all(np.abs(got - ref) <= REL * ref + ABS)


def test_coverage_rejects_bands_wider_than_its_limit(lib, case):
    w, bins, _, _, _ = case
    wide = dataclasses.replace(w.bank, n_f=8193, df=w.bank.df / 64)
    g = lib.FStat(0, topk=10)
    try:
        g.load_workload(dataclasses.replace(w, bank=wide), bins_override=bins)
        lib.fstat_set_coverage(g.ctx, np.zeros(w.n_sft_total, np.int32), np.full(w.n_sft_total, 10, np.int32))
        with pytest.raises(lib.FstatError) as e:
            g.compute()
        assert e.value.code == lib.FSTAT_EINVAL
        lib.fstat_set_coverage(g.ctx, None, None)   # without coverage the same bank computes
        g.compute()
    finally:
        g.close()
