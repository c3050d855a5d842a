"""Host-side geometry of the learned proposal (CPU only): frequency patches,
patch indexing, the fine grids' alignment with the coarse templates, signal
cells and the training windows."""
import math
from types import SimpleNamespace

import numpy as np

import paper_0904_1826_gb300.proposal as P

T = 1800.0


def _bank(n_f=900):
    return SimpleNamespace(f0=120.0, df=1.0 / T, n_f=n_f)


def test_frequency_patches_cover_the_band_and_count_232():
    fs = P.f_starts(900)
    assert len(fs) == 29 and fs[0] == 0 and fs[-1] + P.N_FP == 900
    assert np.all(np.diff(fs[:-1]) == P.N_FP)        # all but the last are disjoint
    assert P.patch_count(900) == 232                 # 4 x 2 sky patches x 29
    assert len(P.f_starts(896)) == 28                # an exact multiple has no overlap


def test_patch_index_is_a_bijection():
    n_q = len(P.f_starts(900))
    seen = set()
    for ia in range(0, P.N_A, P.S_A):
        for id_ in range(0, P.N_D, P.S_D):
            for q in range(n_q):
                seen.add(P.patch_of(ia, id_, q, n_q))
    assert seen == set(range(P.patch_count(900)))


def test_fine_grid_holds_every_coarse_template_of_its_patch():
    bank = _bank()
    da, ds = 2 * math.pi / P.N_A, 2.0 / P.N_D
    fs = P.f_starts(bank.n_f)
    for p in (0, 37, 231):
        sky, f0, df, n_f = P.fine_bank(p, bank)
        q, r = p % len(fs), p // len(fs)
        pa, pd = r // (P.N_D // P.S_D), r % (P.N_D // P.S_D)
        assert sky.shape == (P.S_A * P.FINE_A * P.S_D * P.FINE_D, 2)
        assert df == bank.df / P.FINE_F and n_f == P.N_FP * P.FINE_F
        assert f0 == bank.f0 + fs[q] * bank.df
        # coarse frequencies f0 + k df sit on the fine grid at index 8 k
        for k in (0, 5, P.N_FP - 1):
            coarse = bank.f0 + (fs[q] + k) * bank.df
            assert abs((coarse - f0) / df - P.FINE_F * k) < 1e-6
        # coarse cell centres are fine sky points
        alpha, sind = sky[:, 0], np.sin(sky[:, 1])
        for ia in (pa * P.S_A, pa * P.S_A + P.S_A - 1):
            for id_ in (pd * P.S_D, pd * P.S_D + P.S_D - 1):
                ca, cs = (ia + 0.5) * da, -1.0 + (id_ + 0.5) * ds
                assert np.min(np.hypot(alpha - ca, sind - cs)) < 1e-12


def test_signal_cell_and_patches():
    bank = _bank()
    da, ds = 2 * math.pi / P.N_A, 2.0 / P.N_D
    for ia, id_, m in ((0, 0, 0), (40, 17, 500), (63, 31, 899), (12, 5, 880)):
        inj = SimpleNamespace(alpha=(ia + 0.5) * da, delta=math.asin(-1.0 + (id_ + 0.5) * ds),
                              f=bank.f0 + m * bank.df)
        assert P.signal_cell(inj, bank) == (ia, id_, m)
        fs = P.f_starts(bank.n_f)
        pats = P.signal_patches(inj, bank)
        want = [P.patch_of(ia, id_, q, len(fs)) for q, s in enumerate(fs) if s <= m < s + P.N_FP]
        assert pats == want and 1 <= len(pats) <= 2   # two where the last patch overlaps


def test_training_windows_hold_their_cell_and_negatives_hold_none():
    rng = np.random.default_rng(3)
    cells = [(0, 3, 10), (63, 31, 899), (30, 16, 450)]
    org, lab = P.window_origins(cells, 900, rng, n_pos=16, n_neg=200)
    assert org.shape == (len(cells) * 16 + 200, 3) and lab.sum() == len(cells) * 16

    def holds(o, c):
        return ((c[0] - o[0]) % P.N_A) < P.S_A and o[1] <= c[1] < o[1] + P.S_D and o[2] <= c[2] < o[2] + P.N_FP

    for o, y in zip(org, lab):
        assert 0 <= o[0] < P.N_A and 0 <= o[1] <= P.N_D - P.S_D and 0 <= o[2] <= 900 - P.N_FP
        if y == 1.0:
            assert any(holds(o, c) for c in cells)
        else:
            assert not any(holds(o, c) for c in cells)
    # positives of each cell hold that cell, wrapping in alpha
    for k, c in enumerate(cells):
        for o in org[k * 16:(k + 1) * 16]:
            assert holds(o, c)
