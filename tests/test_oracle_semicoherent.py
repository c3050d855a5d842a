"""Pins of the stack-slide oracle (CPU only).

Exact cases whose coarse indices follow from the grids by construction
(identity, plain shifts, exactly representable slides, ties, a finer
semicoherent grid), and a physics case: a signal with a spindown, searched
coherently per segment by the pinned FP64 F-statistic oracle, must peak in
the semicoherent sum at its own template, and only because of the slide.
"""
import numpy as np

from oracle import fstat_oracle as O
from oracle import semicoherent_oracle as S
from workload import DET_H, DetectorData, Injection, TemplateBank, cn_noise, contiguous_timestamps


def _rand(shape, seed):
    return np.random.default_rng(seed).random(shape).astype(np.float32) * 20


def test_single_segment_on_the_same_grid_is_the_identity():
    tw = _rand((3, 4, 50), 1)
    fdot = np.array([-2e-9, -1e-9, 0.0, 1e-9])
    out, n_out = S.stack_slide([tw], [(100.0, 1 / 1800, 8e8)], 100.0, 1 / 1800, 50, fdot, 8e8)
    np.testing.assert_array_equal(out, tw.astype(np.float64))
    assert n_out == 0


def test_zero_spindown_is_a_shifted_sum_with_counted_edges():
    df = 1 / 1800
    segs = [_rand((2, 3, 40), s) for s in range(4)]
    grids = [(100.0 - 3 * df, df, 8e8 + 1e5 * s) for s in range(4)]   # coarse grid starts 3 bins lower
    out, n_out = S.stack_slide(segs, grids, 100.0, df, 40, np.zeros(3), 8e8)
    want = np.zeros((2, 3, 40))
    for tw in segs:
        want[:, :, :37] += tw[:, :, 3:].astype(np.float64)
    np.testing.assert_array_equal(out, want)
    assert n_out == 3 * 2 * 3 * 4   # the last three frequencies of every (sky, fdot, segment)


def test_exactly_representable_slides_move_by_whole_bins():
    # df = 2^-4 Hz, t_s - t_ref = k 2^10 s, fdot_m = m 2^-14 Hz/s: slide = m k bins exactly
    df = 2.0 ** -4
    fdot = np.array([-2, -1, 0, 1, 2]) * 2.0 ** -14
    n_f, pad = 30, 12
    segs, grids = [], []
    for k in (-2, -1, 0, 1, 2):
        segs.append(_rand((1, 5, n_f + 2 * pad), 10 + k))
        grids.append((64.0 - pad * df, df, 4096.0 + k * 1024.0))
    out, n_out = S.stack_slide(segs, grids, 64.0, df, n_f, fdot, 4096.0)
    assert n_out == 0
    want = np.zeros((1, 5, n_f))
    j = np.arange(n_f)
    for tw, k in zip(segs, (-2, -1, 0, 1, 2)):
        for m in range(5):
            want[0, m] += tw[0, m, j + pad + (m - 2) * k]
    np.testing.assert_array_equal(out, want)


def test_half_bin_slides_round_up():
    # slide of exactly +1/2 and -1/2 bin: floor(x + 1/2) takes j+1 and j
    df = 2.0 ** -4
    tw = np.arange(20, dtype=np.float32)[None, None, :].repeat(2, 1)
    fdot = np.array([-1, 1]) * 2.0 ** -15      # x 2^10 s = -+1/32 Hz = -+1/2 bin
    out, _ = S.stack_slide([tw], [(64.0 - 5 * df, df, 5120.0)], 64.0, df, 10, fdot, 4096.0)
    np.testing.assert_array_equal(out[0, 0], np.arange(10) + 5)        # -1/2 bin -> j + 5
    np.testing.assert_array_equal(out[0, 1], np.arange(10) + 6)        # +1/2 bin -> j + 6


def test_finer_semicoherent_grid_maps_four_to_one():
    df_s = 2.0 ** -4
    tw = np.arange(40, dtype=np.float32)[None, None, :]
    out, n_out = S.stack_slide([tw], [(64.0, df_s, 0.0)], 64.0, df_s / 4, 16, [0.0], 0.0)
    # nearest coarse bin of j/4 (ties up): 0 0 1 1 1 1 2 2 2 2 3 3 3 3 4 4
    np.testing.assert_array_equal(out[0, 0], [0, 0, 1, 1, 1, 1, 2, 2, 2, 2, 3, 3, 3, 3, 4, 4])
    assert n_out == 0


def test_signal_with_spindown_peaks_at_its_template_only_when_slid():
    T, n_seg, per = 1800.0, 3, 20
    t0 = 8.0e8
    t_start = contiguous_timestamps(t0, T, n_seg * per)
    T_seg = per * T
    df = 1.0 / (2 * T_seg)                 # same frequency step on every grid
    u_fd = df / T_seg                      # spindown that slides one bin per segment step
    t_ref = t0 + 1.5 * T_seg               # midpoint of the middle segment
    f_sig = 100.0 + 137 * df
    fdot = u_fd * np.array([-6.0, -4.0, -2.0, 0.0, 2.0])
    k_lo, n_bins = int(round(100.0 * T)) - 40, 100
    noise = cn_noise(77, 0, (n_seg * per, n_bins))
    det = DetectorData(DET_H["lat"], DET_H["lon"], DET_H["az"], t_start, noise)
    inj = Injection(alpha=1.1, delta=0.4, psi=0.3, cosi=0.2, phi0=0.5, f=f_sig, fdot=fdot[1], rho=40.0)
    bins = O.inject([det], T, k_lo, [inj], t_ref)[0]
    sky = np.array([[inj.alpha, inj.delta]])
    n_f, pad = 9, 8
    f0 = f_sig - 4 * df
    segs, grids = [], []
    for s in range(n_seg):
        sl = slice(s * per, (s + 1) * per)
        d = DetectorData(det.lat, det.lon, det.az, t_start[sl], bins[sl])
        t_s = t0 + (s + 0.5) * T_seg
        bank = TemplateBank(sky=sky, f0=f0 - pad * df, df=df, n_f=n_f + 2 * pad, fdot=fdot, t_ref=t_s)
        segs.append(O.compute_fstat_freq_band([d], T, k_lo, 8, bank, [0]))
        grids.append((bank.f0, df, t_s))
    out, n_out = S.stack_slide(segs, grids, f0, df, n_f, fdot, t_ref)
    assert n_out == 0
    m, j = np.unravel_index(np.argmax(out[0]), out[0].shape)
    assert (m, j) == (1, 4), (m, j)
    # each segment's own peak sits at the slid frequency ...
    for s, tw in enumerate(segs):
        assert np.argmax(tw[0, 1]) == pad + 4 - 4 * (s - 1)
    # ... and the sum over segments at the true template without the slide is far lower
    no_slide = sum(tw[0, 1, pad + 4] for tw in segs)
    assert out[0, 1, 4] > 1.5 * no_slide


# ---------------------------------------------------------------- fixed point vs the plain nearest bin

def _nearest_exact(f0, df, fdot, t_ref, f0_s, df_s, t_s, n_f):
    """The plain definition, nearest coarse bin floor(x + 1/2) of
    x = (f0 + j df + fdot (t_s - t_ref) - f0_s) / df_s, in exact rational
    arithmetic on the FP64 inputs; also the distance of frac(x) from 1/2."""
    from fractions import Fraction as F
    a = (F(f0) - F(f0_s) + F(fdot) * (F(t_s) - F(t_ref))) / F(df_s)
    b = F(df) / F(df_s)
    den = a.denominator * b.denominator
    an, bn = a.numerator * b.denominator, b.numerator * a.denominator
    idx = np.empty(n_f, dtype=np.int64)
    tie = np.empty(n_f, dtype=np.float64)
    for j in range(n_f):
        num = an + j * bn
        q = (2 * num + den) // (2 * den)           # floor(x + 1/2)
        idx[j] = q
        r = F(num, den) - q + F(1, 2)               # in [0, 1): 0 means an exact tie
        tie[j] = float(min(r, 1 - r))
    return idx, tie


def _grids():
    """Workunit-shaped stack-slide grids (1/T steps, 8 segments over ~3.1e6 s,
    spindowns to -1e-9 Hz/s, bands padded by 8 bins) and finer and shifted
    semicoherent grids with random offsets."""
    rng = np.random.default_rng(17)
    T = 1800.0
    out = []
    t_ref = 8.0e8
    for s in range(8):
        t_s = t_ref + (s + 0.5) * 3.1e6 / 8
        out.append((100.0, 1 / T, t_ref, 100.0 - 8 / T, 1 / T, t_s, 1800))
    for k in (1, 2, 3, 4, 8):
        f0 = 100.0 + rng.integers(0, 1000) / T + rng.uniform(0, 1) / (k * T)
        t_s = t_ref + rng.uniform(-5e6, 5e6)
        f0_s = f0 - rng.integers(10, 30) / T + rng.uniform(-0.5, 0.5) / T
        out.append((f0, 1 / (k * T), t_ref, f0_s, 1 / T, t_s, 600))
    return out


def test_fixed_point_index_is_the_plain_nearest_bin():
    """Wherever frac(x) is not within 1e-6 of 1/2, the 32.32 fixed-point
    index equals the nearest bin of the plain definition, and the plain FP64
    evaluation round((f - f0_s) / df_s) agrees with both."""
    fdots = np.concatenate([-1e-9 * np.arange(10) / 9, [3e-10, -2.7e-9]])
    n_cmp = n_near = 0
    for f0, df, t_ref, f0_s, df_s, t_s, n_f in _grids():
        A_fx, B_fx = S.slide_constants(f0, df, fdots, t_ref, f0_s, df_s, t_s)
        j = np.arange(n_f)
        for m, fd in enumerate(fdots):
            got = S.slide_index(A_fx[m], B_fx, j)
            want, tie = _nearest_exact(f0, df, float(fd), t_ref, f0_s, df_s, t_s, n_f)
            plain = np.floor((f0 + j * df + fd * (t_s - t_ref) - f0_s) / df_s + 0.5).astype(np.int64)
            ok = tie > 1e-6
            np.testing.assert_array_equal(got[ok], want[ok])
            np.testing.assert_array_equal(plain[ok], want[ok])
            n_cmp += int(ok.sum())
            n_near += int((~ok).sum())
    assert n_cmp > 100_000
    assert n_near <= 1e-4 * n_cmp


def test_nearest_bin_pin_catches_truncation_and_inverse_ratio():
    f0, df, t_ref, f0_s, df_s, t_s, n_f = _grids()[9]
    want, tie = _nearest_exact(f0, df, -4e-10, t_ref, f0_s, df_s, t_s, n_f)
    A_fx, B_fx = S.slide_constants(f0, df, [-4e-10], t_ref, f0_s, df_s, t_s)
    j = np.arange(n_f)
    trunc = (np.int64(A_fx[0]) + j * np.int64(B_fx)) >> np.int64(32)
    assert np.any(trunc[tie > 1e-6] != want[tie > 1e-6])
    A2, B2 = S.slide_constants(f0, df_s, [-4e-10], t_ref, f0_s, df, t_s)
    assert np.any(S.slide_index(A2[0], B2, j)[tie > 1e-6] != want[tie > 1e-6])
