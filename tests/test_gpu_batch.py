"""Batched persistent form and the measured tile autotuner, through the C ABI.

The batch runs many heterogeneous workunits (detectors, SFT counts, bands,
sky grids, spindown counts) through one persistent Dirichlet launch per
kernel variant, captured in a CUDA graph; each workunit's results must equal
the ordinary one-launch path on the same inputs and match the FP64 oracle.
"""
import numpy as np
import pytest

from oracle import fstat_oracle as O
from workload import DetectorData, config3_specs, config3_workunit, config_mid

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3


def _small_wus():
    specs = config3_specs(6, seed=3100)
    shapes = [dict(n_sky=7, n_sft_total=90, band=0.06), dict(n_sky=3, n_sft_total=150, band=0.11),
              dict(n_sky=11, n_sft_total=60, band=0.04), dict(n_sky=5, n_sft_total=120, band=0.09),
              dict(n_sky=2, n_sft_total=200, band=0.03), dict(n_sky=4, n_sft_total=75, band=0.07)]
    wus = [config3_workunit(sp, **sh) for sp, sh in zip(specs, shapes)]
    for w in wus:
        w.topk = 25
    return wus


def _with_signals(w):
    return O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)


def test_batch_matches_single_launches_and_oracle(lib):
    wus = _small_wus()
    bins = [_with_signals(w) for w in wus]
    g = lib.FStat(0, topk=25)
    single = []
    try:
        for w, b in zip(wus, bins):
            lib.fstat_batch_add(g.ctx, w, b)
        assert lib.fstat_batch_size(g.ctx) == len(wus)
        for i in range(len(wus)):
            lib.fstat_batch_compute_one(g.ctx, i)
            single.append((lib.fstat_batch_get_2f(g.ctx, i, 0, wus[i].n_templates),
                           lib.fstat_batch_get_toplist(g.ctx, i, 25)))
        for rep in range(2):   # first call runs and captures, second replays the graph
            lib.fstat_batch_compute(g.ctx)
            for i, w in enumerate(wus):
                got = lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates)
                np.testing.assert_array_equal(got, single[i][0])
                idx, val = lib.fstat_batch_get_toplist(g.ctx, i, 25)
                np.testing.assert_array_equal(idx, single[i][1][0])
        done, total = lib.fstat_batch_get_times(g.ctx, len(wus))
        assert total > 0 and np.all(done > 0) and np.all(done <= total * 1.001)
        for i in (0, 3):
            w = wus[i]
            dets = [DetectorData(d.lat, d.lon, d.az, d.t_start, b) for d, b in zip(w.detectors, bins[i])]
            ref = O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank).ravel()
            got = single[i][0].astype(np.float64)
            assert np.all(np.abs(got - ref) <= REL * ref + ABS)
    finally:
        g.close()


def test_batch_with_two_kernel_variants(lib):
    """A workunit whose frequency spacing needs the generic variant forms a
    second group (second persistent launch) in the same graph."""
    wus = _small_wus()[:3]
    odd = config_mid(n_f=40, n_fdot=2, n_sky=3, df_bins=0.37)
    odd.topk = 25
    wus.append(odd)
    g = lib.FStat(0, topk=25)
    try:
        for w in wus:
            lib.fstat_batch_add(g.ctx, w)
        ref = []
        for i, w in enumerate(wus):
            lib.fstat_batch_compute_one(g.ctx, i)
            ref.append(lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates))
        lib.fstat_batch_compute(g.ctx)
        lib.fstat_batch_compute(g.ctx)
        for i, w in enumerate(wus):
            np.testing.assert_array_equal(lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates), ref[i])
    finally:
        g.close()


@pytest.mark.parametrize("algo,chunks", [("direct", (6, 8, 10)), ("farpoly", (2, 3, 4, 6, 8)),
                                         ("sincpoly", (2, 3, 4, 6, 8)), ("auto", (2, 3, 4, 6, 8))])
def test_autotune_picks_a_valid_tiling_and_keeps_parity(lib, algo, chunks):
    w = config_mid(n_sky=40, n_f=150, n_fdot=3)
    b = _with_signals(w)
    dets = [DetectorData(d.lat, d.lon, d.az, d.t_start, x) for d, x in zip(w.detectors, b)]
    ref = O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, w.bank, range(5)).ravel()
    g = lib.FStat(0, topk=10, algo=algo)
    try:
        g.load_workload(w, bins_override=b)
        t = g.autotune()
        assert t["M"] in (5, 7, 9) and t["sft_chunk"] in chunks and t["slice_us"] > 0
        g.compute()
        assert g.plan()["M"] == t["M"] and g.error_flags() == 0
        got = g.twoF(0, ref.size).astype(np.float64)
        assert np.all(np.abs(got - ref) <= REL * ref + ABS)
    finally:
        g.close()


def test_batch_autotune_gives_m_and_keeps_each_plans_stages(lib):
    """A batch context tunes on its largest workunit and gives every workunit
    that M; each keeps the stage count its own plan chooses (the count a
    single context with the same M plans for it), and results stay those of
    the single launches."""
    specs = config3_specs(3, seed=3300)
    shapes = [dict(n_sky=40, n_sft_total=160, band=0.05), dict(n_sky=60, n_sft_total=200, band=0.12),
              dict(n_sky=30, n_sft_total=120, band=0.08)]
    wus = [config3_workunit(sp, **sh) for sp, sh in zip(specs, shapes)]
    g = lib.FStat(0, topk=10)
    try:
        for w in wus:
            lib.fstat_batch_add(g.ctx, w)
        t = lib.fstat_autotune(g.ctx)
        assert t["M"] in (5, 7, 9)
        for i, w in enumerate(wus):
            lib.fstat_batch_compute_one(g.ctx, i)
            pl = lib.fstat_batch_get_plan(g.ctx, i)
            got = lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates)
            s = lib.FStat(0, topk=10, tile_m=t["M"])
            try:
                s.load_workload(w)
                s.compute()
                ps = s.plan()
                ref = s.twoF()
            finally:
                s.close()
            assert pl["M"] == ps["M"] and pl["sft_chunk"] == ps["sft_chunk"] and pl["variant"] == ps["variant"], (pl, ps)
            np.testing.assert_array_equal(got, ref)
    finally:
        g.close()


def test_batch_with_blocks_of_sky_points(lib):
    """Workunits of one and two spindowns on Fibonacci skies run the ring with
    blocks of 4 neighbouring sky points in the persistent kernel: bit-exact
    against their single launches."""
    specs = config3_specs(2, seed=3400)
    wus = []
    for sp, nfd in zip(specs, (1, 2)):
        sp = dict(sp, n_fdot=nfd)
        wus.append(config3_workunit(sp, n_sky=3000, n_sft_total=160, band=0.1))
    g = lib.FStat(0, topk=10)
    try:
        for w in wus:
            lib.fstat_batch_add(g.ctx, w)
        ref = []
        for i, w in enumerate(wus):
            lib.fstat_batch_compute_one(g.ctx, i)
            assert lib.fstat_batch_get_plan(g.ctx, i)["variant"] in (131, 132)
            ref.append(lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates))
        for rep in range(2):
            lib.fstat_batch_compute(g.ctx)
            for i, w in enumerate(wus):
                np.testing.assert_array_equal(lib.fstat_batch_get_2f(g.ctx, i, 0, w.n_templates), ref[i])
    finally:
        g.close()
