"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerance of the FP32 path: |d2F| <= 1e-4 * 2F + 1e-3, element by element.
Inputs are the seeded workloads of `workload`; signals are added by the
oracle (never by the GPU) before both sides compute.
"""
import dataclasses
import math

import numpy as np
import pytest

from oracle import fstat_oracle as O
from oracle import quantize as Q
from workload import (DET_H, DET_L, DetectorData, TemplateBank, Injection, config0, config_mid,
                      cn_noise, gapped_timestamps, random_sky, T0, T_SFT)

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3


def _dets(w, bins):
    return [DetectorData(d.lat, d.lon, d.az, d.t_start, b) for d, b in zip(w.detectors, bins)]


def _oracle_bins(w):
    return O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)


def _gpu(lib, w, bins, **opts):
    opts.setdefault("dterms", w.dterms)
    opts.setdefault("topk", min(w.topk, w.n_templates))
    g = lib.FStat(0, **opts)
    try:
        g.load_workload(w, bins_override=bins)
        g.compute()
        out = dict(twoF=g.twoF(), flags=g.error_flags(), plan=g.plan(), abcd=g.abcd())
        k = opts["topk"]
        out["top"] = g.toplist(k) if k > 0 else None
    finally:
        g.close()
    return out


def _assert_parity(got, ref, what=""):
    got = np.asarray(got, dtype=np.float64).ravel()
    ref = np.asarray(ref, dtype=np.float64).ravel()
    assert got.shape == ref.shape
    err = np.abs(got - ref)
    tol = REL * np.abs(ref) + ABS
    bad = np.nonzero(err > tol)[0]
    assert bad.size == 0, (f"{what}: {bad.size}/{ref.size} over tolerance; worst at {bad[np.argmax(err[bad])]}"
                           f" got {got[bad[np.argmax(err[bad])]]} ref {ref[bad[np.argmax(err[bad])]]}")


def _check_toplist(top, gpu_all, ref_all, k):
    idx, val = top
    # exact selection on the GPU's own values: (2F desc, index asc)
    order = np.lexsort((np.arange(gpu_all.size), -gpu_all.astype(np.float64)))[:k]
    np.testing.assert_array_equal(idx, order)
    np.testing.assert_array_equal(val, gpu_all[order])
    # against the oracle: entries clearly above the K-th oracle value must be present,
    # and every selected entry must be within tolerance of the oracle's K-th value
    ridx, rval = O.toplist(ref_all, k)
    vk = rval[-1]
    tol_k = REL * vk + ABS
    sure = set(ridx[rval > vk + 2 * tol_k].tolist())
    assert sure <= set(idx.tolist())
    assert np.all(ref_all[idx] >= vk - 2 * tol_k)
    return int(np.sum(np.isin(idx, ridx)))


# ---------------------------------------------------------------- kernel (a): timing, antenna, A/B/C/D

def test_sft_timing_and_abcd_match_oracle(lib):
    w = config_mid()
    g = lib.FStat(0, dterms=8, topk=10)
    try:
        g.load_workload(w)
        g.compute()
        abcd = g.abcd()
        for s in range(w.bank.n_sky):
            dtau, tdot, a, b = g.sft_timing(s)
            alpha, delta = w.bank.sky[s]
            ref = [O.sft_timing_antenna(d, w.T, alpha, delta, w.bank.t_ref) for d in w.detectors]
            r_dtau = np.concatenate([r[0] for r in ref])
            r_tdot = np.concatenate([r[1] for r in ref])
            r_a = np.concatenate([r[2] for r in ref])
            r_b = np.concatenate([r[3] for r in ref])
            np.testing.assert_allclose(dtau, r_dtau, rtol=0, atol=1e-9)
            np.testing.assert_allclose(tdot, r_tdot, rtol=0, atol=1e-14)
            np.testing.assert_allclose(a, r_a, rtol=0, atol=1e-10)
            np.testing.assert_allclose(b, r_b, rtol=0, atol=1e-10)
            A, B, C, D = O.abcd([r[2] for r in ref], [r[3] for r in ref])
            np.testing.assert_allclose(abcd[s], [A, B, C, D], rtol=1e-9)
    finally:
        g.close()


# ---------------------------------------------------------------- kernels (b)-(d): 2F and toplist

ALGOS = ["farpoly", "direct", "sincpoly", "sincrows", "sincpairs"]


@pytest.mark.parametrize("algo", ALGOS)
def test_config0_parity_and_recovery(lib, algo):
    w = config0()
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, algo=algo)
    assert (out["plan"]["variant"] >= 100) == (algo != "direct")
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, "config0")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)
    inj = w.injections[0]
    assert abs(out["twoF"].max() - 4 - inj.rho ** 2) < 4 * math.sqrt(8 + 4 * inj.rho ** 2)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("df_bins,expect", [(1.0, (2, 2)), (0.125, (8, 1)), (2.0, (1, 2)),
                                            (0.5, (4, 2)), (0.37, (1, 1))])
def test_mid_parity_grids(lib, df_bins, expect, algo):
    """Workunit-shaped data: 2 gapped detectors, band edges inside the Doppler
    excursion (zero-filled windows), several columns and ragged tails, and
    frequency spacings that select each thread layout (P, L), in both
    evaluations of the kernel sum."""
    w = config_mid(df_bins=df_bins)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, algo=algo)
    assert (out["plan"]["P"], out["plan"]["L"]) == expect
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, f"mid df={df_bins}/T")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("tile", [dict(tile_m=7), dict(tile_m=5, tile_warps=4), dict(tile_warps=2, sft_chunk=3),
                                  dict(tile_m=1), dict(sft_chunk=1), dict(tile_m=9, sft_chunk=2)])
def test_tile_overrides_keep_parity(lib, tile, algo):
    w = config_mid(n_f=97, n_fdot=4, n_sky=3)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, algo=algo, **tile)
    _assert_parity(out["twoF"], ref, str(tile))


@pytest.mark.parametrize("algo,ids", [("sincrows", range(120, 127)), ("sincpairs", range(127, 129))])
@pytest.mark.parametrize("n_fdot,df_bins", [(4, 1.0), (5, 1.0), (7, 0.5), (10, 1.0), (13, 2.0)])
def test_row_tiled_forms_on_ragged_row_counts(lib, algo, ids, n_fdot, df_bins):
    """The two forms that tile spindown rows inside a thread: row counts that
    leave a partial last row chunk (or an odd last row pair), several columns
    with a ragged tail, element-wise parity and the toplist."""
    w = config_mid(n_f=130, n_fdot=n_fdot, n_sky=3, df_bins=df_bins)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, algo=algo)
    assert out["plan"]["variant"] in ids
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, f"{algo} n_fdot={n_fdot}")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)


@pytest.mark.parametrize("tile_warps,variant", [(3, 130), (5, 129), (0, None)])
@pytest.mark.parametrize("n_fdot", [1, 2, 3])
def test_small_block_rings_on_few_spindowns(lib, tile_warps, variant, n_fdot):
    """The one-row sinc ring with 2 and 4 compute warps (tile_warps = 3 / 5)
    and the planner's own choice (the 10-warp sinc ring; for one or two
    spindowns possibly the far-field ring): parity and the toplist on a wide
    band with a ragged last column."""
    w = config_mid(n_f=410, n_fdot=n_fdot, n_sky=3, n_bins=520)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, tile_warps=tile_warps)
    if variant is not None:
        assert out["plan"]["variant"] == variant
    else:   # one or two spindowns: the sinc or the far-field ring by the planner's copy model
        assert out["plan"]["variant"] in ((110, 112) if n_fdot <= 2 else (112,))
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, f"tile_warps={tile_warps} n_fdot={n_fdot}")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)


@pytest.mark.parametrize("D", [1, 2, 3, 5, 16])
def test_runtime_dterms(lib, D):
    w = config_mid(n_f=40, n_fdot=2, n_sky=2, n_bins=160)
    w.dterms = D
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, D, w.bank).ravel()
    out = _gpu(lib, w, bins)
    _assert_parity(out["twoF"], ref, f"D={D}")


@pytest.mark.parametrize("kahan", [False, True])
@pytest.mark.parametrize("form", ["f16", "bf16"])
def test_precision_forms(lib, form, kahan):
    """16-bit storage: parity with the oracle fed the same dequantised values,
    and the error against the unquantised data stays at the format's level."""
    w = config_mid(n_f=120, n_fdot=3, n_sky=3)
    bins = _oracle_bins(w)
    deq = []
    for b in bins:
        br, bi, sc = Q.quantize(b, form)
        deq.append(Q.dequantize(br, bi, sc, form))
    ref_q = O.compute_fstat_freq_band(_dets(w, deq), w.T, w.k_lo, w.dterms, w.bank).ravel()
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, bins_form=form, kahan=kahan)
    _assert_parity(out["twoF"], ref_q, f"{form} vs dequantised")
    rel = np.abs(out["twoF"] - ref) / (ref + 1.0)
    assert np.max(rel) < (5e-3 if form == "f16" else 4e-2)


def test_kahan_fp32_parity(lib):
    w = config_mid(n_f=60, n_fdot=2, n_sky=2)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, kahan=True)
    _assert_parity(out["twoF"], ref, "kahan c64")


def test_toplist_ties_take_lowest_indices(lib):
    """Templates whose windows miss the stored band have 2F = 0 exactly; a
    toplist longer than the nonzero set must take the zero ties in index order."""
    w = config_mid(n_f=60, n_fdot=2, n_sky=2, n_bins=40)
    w.bank.f0 = (w.k_lo - 5) / w.T   # first templates' windows are inside, later ones far outside
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    n_zero = int(np.sum(ref == 0))
    assert n_zero > 20
    k = int(np.sum(ref > 0)) + 15
    out = _gpu(lib, w, bins, topk=k)
    assert np.sum(out["twoF"] == 0) == n_zero
    _assert_parity(out["twoF"], ref, "ties")
    idx, val = out["top"]
    zeros = np.nonzero(out["twoF"] == 0)[0][:15]
    np.testing.assert_array_equal(idx[-15:], zeros)
    assert np.all(val[-15:] == 0)


def test_injection_kernel_matches_oracle(lib):
    w = config_mid(n_sft=60)
    ref = _oracle_bins(w)
    g = lib.FStat(0)
    try:
        g.load_workload(w)
        g.inject(w.injections, w.bank.t_ref)
        for i, d in enumerate(w.detectors):
            got = lib.fstat_get_bins(g.ctx, i, d.n_sft, w.n_bins)
            scale = np.max(np.abs(ref[i]))
            assert np.max(np.abs(got - ref[i])) <= 4 * 2.0 ** -24 * scale
    finally:
        g.close()


# ---------------------------------------------------------------- edge cases and errors

def test_edge_single_template_single_sky(lib):
    w = config_mid(n_f=1, n_fdot=1, n_sky=1)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, topk=1)
    _assert_parity(out["twoF"], ref, "1 template")
    assert out["top"][0][0] == 0


def test_edge_degenerate_sky_flags_and_zero(lib):
    """One SFT: a, b are proportional, D = AB - C^2 = 0; 2F is set to 0 and flagged."""
    T = T_SFT
    det = DetectorData(DET_H["lat"], 0.0, DET_H["az"], np.array([T0]), cn_noise(3, 1, (1, 64)))
    g = lib.FStat(0, topk=4)
    try:
        lib.fstat_set_sfts(g.ctx, 0, det.lat, det.lon, det.az, T, 180000, det.t_start, det.bins)
        g.set_bank(TemplateBank(np.array([[1.0, 0.2]]), (180000 + 20) / T, 1 / T, 10, np.zeros(1), T0))
        g.compute()
        assert g.error_flags() & 2
        assert np.all(g.twoF() == 0)
    finally:
        g.close()


def test_errors_are_reported_not_raised_on_device(lib):
    g = lib.FStat(0)
    try:
        with pytest.raises(lib.FstatError) as e:
            g.compute()
        assert e.value.code == lib.FSTAT_ESTATE
        bad = cn_noise(1, 1, (4, 32))
        bad[1, 3] = np.nan
        with pytest.raises(lib.FstatError) as e:
            lib.fstat_set_sfts(g.ctx, 0, 0.5, 0.0, 0.3, T_SFT, 180000, T0 + T_SFT * np.arange(4), bad)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError) as e:
            lib.fstat_set_sfts(g.ctx, 0, 0.5, 0.0, 0.3, -1.0, 180000, T0 + T_SFT * np.arange(4), bad * 0)
        assert e.value.code == lib.FSTAT_EINVAL
        ok = cn_noise(1, 1, (4, 32))
        lib.fstat_set_sfts(g.ctx, 0, 0.5, 0.0, 0.3, T_SFT, 180000, T0 + T_SFT * np.arange(4), ok)
        with pytest.raises(lib.FstatError) as e:   # second detector with another band
            lib.fstat_set_sfts(g.ctx, 1, 0.5, 0.0, 0.3, T_SFT, 180001, T0 + T_SFT * np.arange(4), ok)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError) as e:
            lib.fstat_set_templates(g.ctx, np.zeros((1, 2)), 100.0, -1.0, 10, np.zeros(1), T0)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError):
            lib.fstat_create(0, dterms=0)
        for bad_opts in (dict(algo=6), dict(algo="farpoly", dterms=5), dict(algo="farpoly", kahan=True),
                         dict(algo="sincpoly", dterms=5)):
            with pytest.raises(lib.FstatError) as e:
                lib.fstat_create(0, **bad_opts)
            assert e.value.code == lib.FSTAT_EINVAL
    finally:
        g.close()


def test_device_pointer_input_matches_host(lib):
    torch = pytest.importorskip("torch")
    w = config_mid(n_f=50, n_fdot=2, n_sky=2)
    host = _gpu(lib, w, None)
    g = lib.FStat(0, topk=10)
    try:
        for i, d in enumerate(w.detectors):
            dev = torch.from_numpy(d.bins.view(np.float32).reshape(d.n_sft, w.n_bins, 2).copy()).cuda()
            lib.fstat_set_sfts(g.ctx, i, d.lat, d.lon, d.az, w.T, w.k_lo, d.t_start, dev)
        g.set_bank(w.bank)
        s = torch.cuda.Stream()
        g.compute(s)
        out = torch.empty(g.n_templates, dtype=torch.float32, device="cuda")
        lib.fstat_get_2f(g.ctx, 0, g.n_templates, out)
        np.testing.assert_array_equal(out.cpu().numpy(), host["twoF"])
    finally:
        g.close()


def test_nonuniform_unsorted_spindowns(lib):
    """A spindown list that is not an arithmetic grid (and not sorted) takes the
    per-(sky, spindown, SFT) bases; a uniform one the compact per-(sky, SFT) bases."""
    w = config_mid(n_f=80, n_fdot=3, n_sky=3)
    w.bank.fdot = np.array([-7e-10, 0.0, -2e-10])
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins)
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, "non-uniform fdot")


def test_ring_wait_timeout_is_reported_and_context_survives(lib):
    """Failure detection without a fault: the ring's copy warp stops after 3
    SFTs, the compute warps' bounded waits expire (about 2 s), the compute
    returns with error flag bit 2, and the next compute on the same context
    is correct again."""
    w = config_mid(n_sky=1, n_f=40, n_fdot=1)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    g = lib.FStat(0, dterms=w.dterms, topk=5)
    try:
        g.load_workload(w, bins_override=bins)
        assert g.plan()["variant"] >= 107          # the TMA-ring form
        lib.fstat_test_ring_stall(g.ctx, 3)
        g.compute()
        assert g.error_flags() & 4
        with pytest.raises(lib.FstatError) as e:   # reading the results reports it too
            g.twoF()
        assert e.value.code == lib.FSTAT_ETIMEOUT
        lib.fstat_test_ring_stall(g.ctx, -1)
        g.compute()
        assert g.error_flags() == 0
        _assert_parity(g.twoF(), ref, "after a give-up")
    finally:
        g.close()


@pytest.mark.parametrize("n_sft,n_f", [(3, 37), (1, 23), (5, 203)])
def test_ring_form_edges(lib, n_sft, n_f):
    """TMA-ring form with fewer SFTs than ring stages, one SFT per detector,
    and frequency counts that leave ragged lane-groups and columns."""
    w = config_mid(n_sft=n_sft, n_sky=2, n_f=n_f, n_fdot=3, n_bins=260)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins)
    assert out["plan"]["variant"] >= 107
    assert out["flags"] & 1 == 0
    _assert_parity(out["twoF"], ref, f"ring n_sft={n_sft} n_f={n_f}")


@pytest.mark.parametrize("algo", ["sincpoly", "farpoly"])
def test_ring_with_four_threads_per_lane_group_on_a_wide_bank(lib, algo):
    """df = 1/(2T) gives P = 4 threads per lane-group; with enough lane-groups
    per block every one of them must have all four threads (warps divisible
    by P), else templates would go uncomputed."""
    w = config_mid(df_bins=0.5, n_f=600, n_fdot=10, n_sky=2, n_bins=360)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, algo=algo)
    assert (out["plan"]["P"], out["plan"]["L"]) == (4, 2)
    assert out["plan"]["variant"] >= 107 and (out["plan"]["warps"] - 1) % 4 == 0   # ring, 8 compute warps
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, "P=4 wide bank")


def test_sinc_ring_for_l1_banks(lib):
    """df = 1/(8T): P = 8, L = 1; the sinc form runs in the TMA ring on plain
    (not parity-split) tables, with M = 1 or 5 per the planner, across
    several blocks per column and a ragged tail."""
    w = config_mid(df_bins=0.125, n_f=700, n_fdot=3, n_sky=2, n_bins=160)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    for tile in (dict(), dict(tile_m=5), dict(tile_m=1)):
        out = _gpu(lib, w, bins, algo="sincpoly", **tile)
        assert (out["plan"]["P"], out["plan"]["L"]) == (8, 1)
        assert out["plan"]["variant"] in (118, 119), out["plan"]
        assert out["flags"] == 0
        _assert_parity(out["twoF"], ref, f"L=1 ring {tile}")


def test_size_limits_are_errors_not_allocations(lib):
    """Banks past the documented limits are refused before any device
    allocation: more than 2^40 templates, more than 64 spindowns."""
    w = config_mid(n_sky=2, n_f=20, n_fdot=2)
    g = lib.FStat(0, topk=10)
    try:
        g.load_workload(w)
        sky = np.zeros((1 << 21, 2))
        with pytest.raises(lib.FstatError) as e:      # 2^21 x 2^20 x 1 = 2^41 templates
            lib.fstat_set_templates(g.ctx, sky, w.bank.f0, w.bank.df, 1 << 20, np.zeros(1), w.bank.t_ref)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError) as e:      # 65 spindowns
            lib.fstat_set_templates(g.ctx, w.bank.sky, w.bank.f0, w.bank.df, 20, np.zeros(65), w.bank.t_ref)
        assert e.value.code == lib.FSTAT_EINVAL
        g.compute()                                    # the earlier bank still computes
        assert g.error_flags() == 0
    finally:
        g.close()


def _close_sky(w, n_a, n_d, step):
    """The bank's sky replaced by a small regular grid around its first
    point (the signal's), delta fastest: consecutive points are neighbours,
    as in the learned proposal's maps."""
    a0, d0 = w.bank.sky[0]
    a = a0 + step * (np.arange(n_a) - n_a // 2)
    d = d0 + step * (np.arange(n_d) - n_d // 2)
    A, Dd = np.meshgrid(a, d, indexing="ij")
    sky = np.stack([A.ravel(), Dd.ravel()], axis=1)
    return dataclasses.replace(w, bank=dataclasses.replace(w.bank, sky=sky))


@pytest.mark.parametrize("n_fdot,df_bins,ids,tile_m,algo", [(1, 1.0, (131, 132), 0, "auto"),
                                                             (2, 1.0, (131, 132), 0, "auto"),
                                                             (1, 1.0, (132,), 0, "farpoly"),
                                                             (1, 0.125, (133, 134), 0, "auto"),
                                                             (1, 0.125, (134,), 1, "auto")])
def test_blocks_of_four_sky_points(lib, n_fdot, df_bins, ids, tile_m, algo):
    """The one-row ring with blocks of 4 consecutive sky points (one window for
    the four, meta and bases SFT-major), chosen by the planner for a bank of
    few spindowns on a grid of close sky points (18 points: a ragged last
    block of 2): parity, the toplist, and bit-identical 2F against the
    one-sky-point block of the same form where one exists (8 compute warps)."""
    n_f = 210 if df_bins == 1.0 else (256 if tile_m != 1 else 64)   # M = 1: a band of 8 lane-groups a row
    w = _close_sky(config_mid(n_f=n_f, n_fdot=n_fdot, n_sky=3, df_bins=df_bins, n_bins=300), 3, 6, 0.01)
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins, tile_m=tile_m, algo=algo)
    assert out["plan"]["variant"] in ids, out["plan"]
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, f"sky blocks n_fdot={n_fdot} df={df_bins}")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)
    if df_bins == 1.0:
        algo = "sincpoly" if out["plan"]["variant"] == 131 else "farpoly"
        one = _gpu(lib, w, bins, tile_warps=9, algo=algo)
        assert one["plan"]["variant"] in (114, 107), one["plan"]
        np.testing.assert_array_equal(out["twoF"], one["twoF"])


@pytest.mark.parametrize("n_fdot", [1, 2])
def test_blocks_of_four_sky_points_in_neighbour_order(lib, n_fdot):
    """A sky list whose consecutive points are far apart (Fibonacci lattice):
    the blocks group 4 neighbours of a neighbour order instead (meta and bases
    written in that order); parity, and 2F bit-identical to blocks of one sky
    point of the same form."""
    from workload import fibonacci_sky
    w = config_mid(n_f=210, n_fdot=n_fdot, n_sky=3, n_bins=300)
    w = dataclasses.replace(w, bank=dataclasses.replace(w.bank, sky=fibonacci_sky(150)))
    bins = _oracle_bins(w)
    ref = O.compute_fstat_freq_band(_dets(w, bins), w.T, w.k_lo, w.dterms, w.bank).ravel()
    out = _gpu(lib, w, bins)
    assert out["plan"]["variant"] in (131, 132), out["plan"]
    assert out["flags"] == 0
    _assert_parity(out["twoF"], ref, f"neighbour-order sky blocks n_fdot={n_fdot}")
    _check_toplist(out["top"], out["twoF"], ref, w.topk)
    algo = "sincpoly" if out["plan"]["variant"] == 131 else "farpoly"
    one = _gpu(lib, w, bins, tile_warps=9, algo=algo)
    np.testing.assert_array_equal(out["twoF"], one["twoF"])


@pytest.mark.parametrize("form", ["f16", "bf16"])
def test_sky_blocks_with_16_bit_storage_and_noise_weights(lib, form):
    """Blocks of 4 sky points (neighbour order) with 16-bit SFT storage and
    noise weights (a and b scaled per SFT before the SFT-major write): 2F
    bit-identical to blocks of one sky point of the same form."""
    from workload import fibonacci_sky
    w = config_mid(n_f=210, n_fdot=1, n_sky=3, n_bins=300)
    w = dataclasses.replace(w, bank=dataclasses.replace(w.bank, sky=fibonacci_sky(150)))
    bins = _oracle_bins(w)
    outs = []
    for tw in (0, 9):
        g = lib.FStat(0, dterms=w.dterms, topk=10, bins_form=form, tile_warps=tw, algo="sincpoly")
        try:
            g.load_workload(w, bins_override=bins)
            lib.fstat_set_noise_floor(g.ctx, 9)
            g.compute()
            outs.append((g.twoF(), g.plan()["variant"], g.error_flags()))
        finally:
            g.close()
    assert outs[0][1] == 131 and outs[1][1] == 114, (outs[0][1], outs[1][1])
    assert outs[0][2] == 0 and outs[1][2] == 0
    np.testing.assert_array_equal(outs[0][0], outs[1][0])
