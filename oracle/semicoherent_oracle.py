"""Semicoherent stack-slide of coherent 2F over time segments (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; it shares no code with the CUDA library.

The paper's Einstein@Home client follows the F-statistic with a second,
semicoherent stage (a Hough transform over the coherent results of several
data segments, Section "Einstein@Home"); it gives no algorithm for it.  This
is the generic stack-slide form of that stage, the design's reading:

* the data are split into segments s; segment s has its own coherent bank
  (same sky list, same spindown list) with frequencies f0_s + i df_s,
  i < n_f_s, at its own reference time t_s;
* a semicoherent template (sky, f, fdot) with f = f0 + j df at t_ref has the
  frequency f + fdot (t_s - t_ref) at t_s ("slide");
* its statistic is the sum over segments, in segment order, of the segment's
  coherent 2F at (sky, fdot, nearest coarse frequency); a slid frequency
  outside the segment's band contributes nothing and is counted.

The nearest coarse frequency is decided in 32.32 fixed point, the same
precision on both sides: with FP64 (round to nearest, no fused operations,
in this order)

    A = ((f0 - f0_s) + fdot * (t_s - t_ref)) / df_s,    B = df / df_s,

A_fx = rint(A 2^32) and B_fx = rint(B 2^32) (half to even), and the index is
i = floor((A_fx + j B_fx + 2^31) / 2^32) in exact integer arithmetic.  The sum
itself is FP64 here.  Wherever x = (f0 + j df + fdot (t_s - t_ref) - f0_s) / df_s
is not within 1e-6 of a half-integer, this index is the plain nearest bin
floor(x + 1/2) of the exact x (pinned on workunit-shaped and finer grids in
tests/test_oracle_semicoherent.py).
"""
from __future__ import annotations

import numpy as np

TWO32 = float(2 ** 32)


def slide_constants(f0: float, df: float, fdot, t_ref: float, f0_s: float, df_s: float, t_s: float):
    """(A_fx [n_fdot] int64, B_fx int) of one segment, by the FP64 steps above."""
    fdot = np.asarray(fdot, dtype=np.float64)
    d1 = np.float64(f0) - np.float64(f0_s)
    d2 = np.float64(t_s) - np.float64(t_ref)
    A = (d1 + fdot * d2) / np.float64(df_s)
    B = np.float64(df) / np.float64(df_s)
    A_fx = np.rint(A * TWO32).astype(np.int64)
    B_fx = int(np.rint(B * TWO32))
    return A_fx, B_fx


def slide_index(A_fx: int, B_fx: int, j):
    """Coarse index of semicoherent frequency index j (exact integer arithmetic)."""
    j = np.asarray(j, dtype=np.int64)
    return (np.int64(A_fx) + j * np.int64(B_fx) + np.int64(1 << 31)) >> np.int64(32)


def stack_slide(seg_twoF, seg_grids, f0: float, df: float, n_f: int, fdot, t_ref: float):
    """Semicoherent sum.

    seg_twoF  list of arrays [n_sky][n_fdot][n_f_s] (any float type)
    seg_grids list of (f0_s, df_s, t_s) per segment
    returns (out [n_sky][n_fdot][n_f] FP64, n_outside)
    """
    fdot = np.asarray(fdot, dtype=np.float64)
    n_sky, n_fdot = seg_twoF[0].shape[0], seg_twoF[0].shape[1]
    out = np.zeros((n_sky, n_fdot, n_f), dtype=np.float64)
    n_outside = 0
    j = np.arange(n_f, dtype=np.int64)
    for tw, (f0_s, df_s, t_s) in zip(seg_twoF, seg_grids):
        tw = np.asarray(tw, dtype=np.float64)
        n_f_s = tw.shape[2]
        A_fx, B_fx = slide_constants(f0, df, fdot, t_ref, f0_s, df_s, t_s)
        for m in range(n_fdot):
            i = slide_index(A_fx[m], B_fx, j)
            ok = (i >= 0) & (i < n_f_s)
            n_outside += int(np.count_nonzero(~ok)) * n_sky
            out[:, m, ok] += tw[:, m, i[ok]]
    return out, n_outside
