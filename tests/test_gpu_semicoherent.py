"""Semicoherent stack-slide through the C ABI (include/fstat_semi.h) against
the stack-slide oracle.

Segments are time slices of a workload's SFTs, each computed on the GPU with
its bank at the segment's midpoint.  The slid lookups are decided in the same
32.32 fixed point on both sides, so the out-of-band counts must agree exactly
and the sums within FP32 rounding of the segment-ordered sum; against the
FP64 coherent oracle per segment, the sums agree within the per-segment 2F
tolerance.
"""
import numpy as np
import pytest

from oracle import fstat_oracle as O
from oracle import semicoherent_oracle as S
from workload import DetectorData, TemplateBank, config_mid

pytestmark = pytest.mark.gpu

REL, ABS = 1e-4, 1e-3


def _split(w, n_seg, bins=None):
    """Per segment: its detectors (time slice of every detector) and midpoint."""
    t_all = np.concatenate([d.t_start for d in w.detectors])
    t0, t1 = float(t_all.min()), float(t_all.max()) + w.T
    edges = t0 + (t1 - t0) * np.arange(n_seg + 1) / n_seg
    edges[-1] += 1.0
    out = []
    for s in range(n_seg):
        dets = []
        for i, d in enumerate(w.detectors):
            b = d.bins if bins is None else bins[i]
            sel = (d.t_start >= edges[s]) & (d.t_start < edges[s + 1])
            assert sel.any()
            dets.append(DetectorData(d.lat, d.lon, d.az, d.t_start[sel], b[sel]))
        out.append((dets, 0.5 * (edges[s] + edges[s + 1])))
    return out


def _compute_segments(lib, w, n_seg, pad, df_s, algo="auto", bins=None):
    ctxs, grids, tws, segs = [], [], [], []
    for dets, t_s in _split(w, n_seg, bins):
        bank = TemplateBank(sky=w.bank.sky, f0=w.bank.f0 - pad * df_s, df=df_s,
                            n_f=int(round(w.bank.n_f * w.bank.df / df_s)) + 2 * pad, fdot=w.bank.fdot, t_ref=t_s)
        g = lib.FStat(0, topk=10, algo=algo)
        ws = type(w)(w.name, w.T, w.k_lo, w.n_bins, w.dterms, 10, dets, bank)
        g.load_workload(ws)
        g.compute()
        assert g.error_flags() == 0
        ctxs.append(g)
        grids.append((bank.f0, bank.df, t_s))
        tws.append(g.twoF().reshape(bank.n_sky, bank.n_fdot, bank.n_f))
        segs.append((dets, bank))
    return ctxs, grids, tws, segs


def _run(lib, ctxs, w, f0, df, n_f, t_ref):
    import torch
    out = torch.empty(w.bank.n_sky * w.bank.n_fdot * n_f, dtype=torch.float32, device="cuda")
    n_out = lib.fstat_stackslide([c.ctx for c in ctxs], f0, df, n_f, t_ref, out)
    return out.cpu().numpy().reshape(w.bank.n_sky, w.bank.n_fdot, n_f).astype(np.float64), n_out


def _close(ctxs):
    for c in ctxs:
        c.close()


@pytest.mark.parametrize("algo", ["auto", "direct"])
def test_stackslide_matches_oracle_on_gpu_segments(lib, algo):
    w = config_mid(n_sky=5, n_f=120, n_fdot=4)
    w.bank.fdot[:] = np.array([-3e-9, -1.5e-9, 0.0, 1.5e-9])
    ctxs, grids, tws, _ = _compute_segments(lib, w, 3, 3, w.bank.df, algo)
    try:
        got, n_out = _run(lib, ctxs, w, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.t_ref)
        want, want_out = S.stack_slide(tws, grids, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.fdot, w.bank.t_ref)
        assert n_out == want_out
        np.testing.assert_allclose(got, want, rtol=4 * 3 * 2.0 ** -24, atol=0)
    finally:
        _close(ctxs)


def test_stackslide_finer_grid_and_counted_band_edges(lib):
    # semicoherent grid twice as fine as the segments', band wider than theirs
    w = config_mid(n_sky=3, n_f=100, n_fdot=3)
    ctxs, grids, tws, _ = _compute_segments(lib, w, 4, 0, w.bank.df)
    try:
        f0, df, n_f = w.bank.f0 - 4 * w.bank.df, w.bank.df / 2, 2 * w.bank.n_f + 16
        got, n_out = _run(lib, ctxs, w, f0, df, n_f, w.bank.t_ref + 1e5)
        want, want_out = S.stack_slide(tws, grids, f0, df, n_f, w.bank.fdot, w.bank.t_ref + 1e5)
        assert n_out == want_out and n_out > 0
        np.testing.assert_allclose(got, want, rtol=4 * 4 * 2.0 ** -24, atol=0)
    finally:
        _close(ctxs)


def test_stackslide_against_fp64_coherent_oracle_with_signal(lib):
    w = config_mid(n_sky=3, n_f=60, n_fdot=3)
    bins = O.inject(w.detectors, w.T, w.k_lo, w.injections, w.bank.t_ref)
    ctxs, grids, tws, segs = _compute_segments(lib, w, 3, 2, w.bank.df, bins=bins)
    try:
        got, n_out = _run(lib, ctxs, w, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.t_ref)
        ref = [O.compute_fstat_freq_band(dets, w.T, w.k_lo, w.dterms, bank) for dets, bank in segs]
        want, want_out = S.stack_slide(ref, grids, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.fdot, w.bank.t_ref)
        assert n_out == want_out == 0
        assert np.all(np.abs(got - want) <= REL * want + 3 * ABS)   # per-segment 2F tolerance, summed
        assert want.max() > 20     # the injected signal stands out in the sum
    finally:
        _close(ctxs)


def test_stackslide_full_band_sampled(lib):
    # 8 segments, 1800 semicoherent frequencies x 10 spindowns x 32 sky points
    w = config_mid(n_sky=32, n_f=1800, n_fdot=10, n_bins=1900, n_sft=96)
    ctxs, grids, tws, _ = _compute_segments(lib, w, 8, 4, w.bank.df)
    try:
        got, n_out = _run(lib, ctxs, w, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.t_ref)
        want, want_out = S.stack_slide(tws, grids, w.bank.f0, w.bank.df, w.bank.n_f, w.bank.fdot, w.bank.t_ref)
        assert n_out == want_out
        np.testing.assert_allclose(got, want, rtol=4 * 8 * 2.0 ** -24, atol=0)
    finally:
        _close(ctxs)


def test_stackslide_errors(lib):
    import torch
    w = config_mid(n_sky=3, n_f=40, n_fdot=2)
    ctxs, grids, tws, segs = _compute_segments(lib, w, 2, 2, w.bank.df)
    out = torch.empty(3 * 2 * 40, dtype=torch.float32, device="cuda")
    other = lib.FStat(0, topk=10)
    try:
        dets, bank = segs[1]
        other.load_workload(type(w)(w.name, w.T, w.k_lo, w.n_bins, w.dterms, 10, dets, bank))
        with pytest.raises(lib.FstatError) as e:   # not computed yet
            lib.fstat_stackslide([ctxs[0].ctx, other.ctx], w.bank.f0, w.bank.df, 40, w.bank.t_ref, out)
        assert e.value.code == lib.FSTAT_ESTATE
        sky2 = w.bank.sky.copy()
        sky2[0, 0] += 1e-3
        other.set_bank(TemplateBank(sky=sky2, f0=bank.f0, df=bank.df, n_f=bank.n_f, fdot=bank.fdot,
                                    t_ref=bank.t_ref))
        other.compute()
        with pytest.raises(lib.FstatError) as e:   # another sky list
            lib.fstat_stackslide([ctxs[0].ctx, other.ctx], w.bank.f0, w.bank.df, 40, w.bank.t_ref, out)
        assert e.value.code == lib.FSTAT_EINVAL
        with pytest.raises(lib.FstatError) as e:   # grid ratio out of range
            lib.fstat_stackslide([c.ctx for c in ctxs], w.bank.f0, w.bank.df * 2.0 ** 21, 40, w.bank.t_ref, out)
        assert e.value.code == lib.FSTAT_EINVAL
        # the context stays usable
        got, _ = _run(lib, ctxs, w, w.bank.f0, w.bank.df, 40, w.bank.t_ref)
        want, _ = S.stack_slide(tws, grids, w.bank.f0, w.bank.df, 40, w.bank.fdot, w.bank.t_ref)
        np.testing.assert_allclose(got, want, rtol=8 * 2.0 ** -24, atol=0)
    finally:
        other.close()
        _close(ctxs)
