"""Coherent F-statistic with a per-SFT frequency coverage (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; it shares no code with the CUDA library.

The paper's version-3 CUDA client meets data sets in which the number of SFTs
differs from frequency to frequency (Section "CUDA", version 3: the thread
block's x extent is padded to the largest SFT count of the band).  The
design's reading: every SFT alpha carries a half-open range [j_lo, j_hi) of
template frequency indices f_j = f0 + j df of the bank that it contributes
to.  A template at frequency index j then uses only the SFTs whose range
holds j, for its Fa, Fb and for its own A, B, C, D:

    Fa(j) = sum_{alpha covers j} a_alpha z_alpha(j)      (likewise Fb)
    A(j)  = sum_{alpha covers j} a_alpha^2               (likewise B, C)
    2F(j) = 2 (B|Fa|^2 + A|Fb|^2 - 2 C Re(Fa Fb*)) / D,  D = AB - C^2

with 2F = 0 where D is degenerate (no SFT, or D <= 1e-13 AB), as for a
degenerate sky.  Everything else (z, a, b, the window) is the plain oracle's.
"""
from __future__ import annotations

import numpy as np

from oracle import fstat_oracle as O


def compute_fstat_coverage(dets, T: float, k_lo: int, dterms: int, bank, j_lo, j_hi, sky_indices=None):
    """2F [n_sky_sel, n_fdot, n_f] (FP64).  j_lo, j_hi: per SFT in detector
    order (all SFTs of detector 0, then detector 1, ...)."""
    j_lo = np.asarray(j_lo, dtype=np.int64)
    j_hi = np.asarray(j_hi, dtype=np.int64)
    if sky_indices is None:
        sky_indices = range(bank.sky.shape[0])
    jj = np.arange(bank.n_f, dtype=np.int64)
    f = bank.f0 + jj.astype(np.float64) * bank.df
    F, FD = np.meshgrid(f, np.asarray(bank.fdot, dtype=np.float64), indexing="xy")
    J = np.broadcast_to(jj[None, :], F.shape)
    out = []
    for s in sky_indices:
        alpha, delta = bank.sky[s]
        Fa = np.zeros(F.shape, dtype=np.complex128)
        Fb = np.zeros(F.shape, dtype=np.complex128)
        A = np.zeros(F.shape)
        B = np.zeros(F.shape)
        C = np.zeros(F.shape)
        base = 0
        for det in dets:
            dtau, tdot, a, b = O.sft_timing_antenna(det, T, alpha, delta, bank.t_ref)
            w = getattr(det, "weights", None)
            if w is not None:
                sw = np.sqrt(np.asarray(w, dtype=np.float64))
                a, b = a * sw, b * sw
            for k in range(len(det.t_start)):
                cov = (J >= j_lo[base + k]) & (J < j_hi[base + k])
                if not cov.any():
                    continue
                frac, kh = O.phase_and_kappa(F, FD, dtau[k], tdot[k], T)
                z = O.some_calculations(det.bins[k], k_lo, kh, frac, dterms)
                Fa += np.where(cov, a[k] * z, 0.0)
                Fb += np.where(cov, b[k] * z, 0.0)
                A += np.where(cov, a[k] * a[k], 0.0)
                B += np.where(cov, b[k] * b[k], 0.0)
                C += np.where(cov, a[k] * b[k], 0.0)
            base += len(det.t_start)
        D = A * B - C * C
        ok = (D > 1e-300) & (D > 1e-13 * A * B)
        q = B * np.abs(Fa) ** 2 + A * np.abs(Fb) ** 2 - 2.0 * C * np.real(Fa * np.conj(Fb))
        out.append(np.where(ok, 2.0 * q / np.where(ok, D, 1.0), 0.0))
    return np.stack(out, 0)
