"""Noise-floor normalisation and noise weights (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
may import this module; it shares no code with the CUDA path.

The paper's client works on white, stationary SFTs; this is the step before
its path for coloured, non-stationary noise (the design's reading, applied
identically on both sides):

* power P_k = Re^2 + Im^2 of each stored bin, in FP32 (the two squares
  rounded, then their sum);
* noise floor S(k) = median{P_j : |j - k| <= W, j in the stored band} / ln 2
  (the median of an exponential variable of mean S is S ln 2); an even count,
  at the clipped band edges, averages its two middle values; FP32, in the
  order (m1 + m2) * 0.5 / ln 2;
* whitened bins X'_k = X_k / sqrt(S(k)) (0 where S(k) = 0);
* weight of SFT alpha: w = (1 / Sbar) / mean_beta(1 / Sbar_beta) over all SFTs
  of all detectors, Sbar = mean of S over the SFT's bins (0 where Sbar = 0,
  left out of the mean);
* the F-statistic then uses sqrt(w) a, sqrt(w) b in A, B, C, Fa and Fb.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LN2_F32 = np.float32(math.log(2.0))


@dataclass
class WeightedDetector:
    """A detector whose SFTs are whitened and carry per-SFT noise weights."""
    lat: float
    lon: float
    az: float
    t_start: np.ndarray
    bins: np.ndarray
    weights: np.ndarray

    @property
    def n_sft(self) -> int:
        return int(self.bins.shape[0])


def power_f32(bins: np.ndarray) -> np.ndarray:
    """|X|^2 in FP32: re*re and im*im each rounded, then their sum rounded."""
    re = np.ascontiguousarray(bins.real, dtype=np.float32)
    im = np.ascontiguousarray(bins.imag, dtype=np.float32)
    return (re * re) + (im * im)


def running_median_floor(bins: np.ndarray, half_window: int) -> np.ndarray:
    """S [n_sft, n_bins] (FP32) of complex bins [n_sft, n_bins]."""
    p = power_f32(np.asarray(bins))
    n_sft, n = p.shape
    out = np.empty((n_sft, n), dtype=np.float32)
    half = np.float32(0.5)
    for s in range(n_sft):
        row = p[s]
        for k in range(n):
            w = np.sort(row[max(0, k - half_window):min(n, k + half_window + 1)])
            c = w.shape[0]
            m1, m2 = w[(c - 1) // 2], w[c // 2]
            out[s, k] = np.float32(np.float32(m1 + m2) * half) / LN2_F32
    return out


def whiten(bins: np.ndarray, floor: np.ndarray) -> np.ndarray:
    """X / sqrt(S) in FP64 (0 where S = 0)."""
    f = np.asarray(floor, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(f > 0, np.asarray(bins, dtype=np.complex128) / np.sqrt(np.where(f > 0, f, 1.0)), 0.0)


def noise_weights(floors) -> list:
    """Per-detector weight arrays from the detectors' floors (a list of
    [n_sft, n_bins] arrays), normalised over all SFTs of all detectors."""
    inv = []
    for f in floors:
        sbar = np.asarray(f, dtype=np.float64).mean(axis=1)
        inv.append(np.where(sbar > 0, 1.0 / np.where(sbar > 0, sbar, 1.0), 0.0))
    allv = np.concatenate(inv)
    pos = allv[allv > 0]
    norm = pos.mean() if pos.size else 1.0
    return [v / norm for v in inv]


def weighted_detectors(dets, half_window: int) -> list:
    """Whitened, weighted copies of detectors (lat, lon, az, t_start, bins)."""
    floors = [running_median_floor(d.bins, half_window) for d in dets]
    ws = noise_weights(floors)
    return [WeightedDetector(d.lat, d.lon, d.az, np.asarray(d.t_start), whiten(d.bins, f), w)
            for d, f, w in zip(dets, floors, ws)]
