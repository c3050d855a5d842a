"""Seeded synthetic Einstein@Home-shaped workunits.

Every random number comes from a counter-based Philox stream keyed by
(seed, stream id), so a workload is reproducible bit for bit on any machine.
The paper measures on real LIGO/GEO SFT files (Section "Test cases"), which are
not available; these generators stand in for them with the shapes of its
"small test case" and "full work unit" data: one or two detectors, 1800 s SFTs,
a narrow band of complex bins, white Gaussian noise and a few continuous-wave
signals.  Signal parameters are drawn here; the signal itself is added by
whoever owns the method's arithmetic (the oracle in tests, the library's
injection call elsewhere), because computing it needs the timing and antenna
model.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "T_SFT", "T0", "DET_H", "DET_L", "DetectorData", "TemplateBank", "Injection",
    "Workload", "Line", "add_lines", "philox", "cn_noise", "contiguous_timestamps", "gapped_timestamps",
    "fibonacci_sky", "random_sky", "draw_injections", "config0", "config1",
    "config_mid", "config3_workunit", "config3_specs", "config4_workunit",
    "n_templates", "template_index", "template_params",
]

T_SFT = 1800.0          # SFT length in seconds
T0 = 8.0e8              # first SFT start (GPS-like seconds)

# Detector geometry: latitude, longitude of the vertex, x-arm azimuth measured
# from local North, clockwise (y-arm at azimuth + 90 degrees).
DET_H = dict(lat=math.radians(46.45), lon=0.0, az=math.radians(36.0))
DET_L = dict(lat=math.radians(30.56), lon=0.0, az=math.radians(72.0))

# Philox stream ids
_S_NOISE = 1
_S_TIME = 20
_S_SKY = 40
_S_INJ = 60
_S_WU = 80


def philox(seed: int, stream: int) -> np.random.Generator:
    """Counter-based generator keyed by (seed, stream)."""
    key = np.array([seed & 0xFFFFFFFFFFFFFFFF, stream & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return np.random.Generator(np.random.Philox(key=key))


def cn_noise(seed: int, stream: int, shape) -> np.ndarray:
    """Circular complex Gaussian noise with E|X|^2 = 1 (Re, Im ~ N(0, 1/2)), complex64."""
    g = philox(seed, stream)
    x = g.standard_normal(tuple(shape) + (2,), dtype=np.float64) * math.sqrt(0.5)
    return (x[..., 0] + 1j * x[..., 1]).astype(np.complex64)


def contiguous_timestamps(t0: float, T: float, n: int) -> np.ndarray:
    return t0 + T * np.arange(n, dtype=np.float64)


def gapped_timestamps(seed: int, stream: int, t0: float, T: float, n: int,
                      duty: float = 0.7) -> np.ndarray:
    """Walk a grid of spacing T and keep each slot with probability `duty`
    until n slots are kept (random gaps, like a detector's duty cycle)."""
    g = philox(seed, stream)
    out = []
    slot = 0
    while len(out) < n:
        u = g.random(4096)
        for ui in u:
            if ui < duty:
                out.append(t0 + T * slot)
                if len(out) == n:
                    break
            slot += 1
    return np.asarray(out, dtype=np.float64)


def fibonacci_sky(n: int) -> np.ndarray:
    """Golden-spiral lattice: n nearly isotropic sky points, [n, 2] (alpha, delta)."""
    i = np.arange(n, dtype=np.float64)
    golden = (1.0 + math.sqrt(5.0)) / 2.0
    z = 1.0 - (2.0 * i + 1.0) / n
    delta = np.arcsin(z)
    alpha = np.mod(2.0 * math.pi * i / golden, 2.0 * math.pi)
    return np.stack([alpha, delta], axis=1)


def random_sky(seed: int, stream: int, n: int) -> np.ndarray:
    g = philox(seed, stream)
    alpha = g.uniform(0.0, 2.0 * math.pi, n)
    delta = np.arcsin(g.uniform(-1.0, 1.0, n))
    return np.stack([alpha, delta], axis=1)


@dataclass
class DetectorData:
    lat: float
    lon: float
    az: float
    t_start: np.ndarray        # float64 [n_sft], SFT start times
    bins: np.ndarray           # complex64 [n_sft, n_bins], bins k_lo .. k_lo+n_bins-1

    @property
    def n_sft(self) -> int:
        return int(self.t_start.shape[0])


@dataclass
class TemplateBank:
    sky: np.ndarray            # float64 [n_sky, 2] (alpha, delta) equatorial, radians
    f0: float                  # first frequency, Hz
    df: float                  # frequency spacing, Hz
    n_f: int
    fdot: np.ndarray           # float64 [n_fdot], Hz/s
    t_ref: float               # reference time of f, fdot

    @property
    def n_sky(self) -> int:
        return int(self.sky.shape[0])

    @property
    def n_fdot(self) -> int:
        return int(self.fdot.shape[0])


@dataclass
class Injection:
    """Random parameters of one continuous-wave signal; the amplitude is fixed
    through its target optimal SNR `rho` by whoever synthesises it."""
    alpha: float
    delta: float
    psi: float
    cosi: float
    phi0: float
    f: float
    fdot: float
    rho: float


@dataclass
class Workload:
    name: str
    T: float
    k_lo: int
    n_bins: int
    dterms: int
    topk: int
    detectors: list
    bank: TemplateBank
    injections: list = field(default_factory=list)
    lines: list = field(default_factory=list)       # detector lines (Line) added to the bins

    @property
    def n_sft_total(self) -> int:
        return sum(d.n_sft for d in self.detectors)

    @property
    def n_templates(self) -> int:
        return n_templates(self.bank)

    @property
    def n_pairs(self) -> int:
        return self.n_templates * self.n_sft_total


def n_templates(bank: TemplateBank) -> int:
    return bank.n_sky * bank.n_fdot * bank.n_f


def template_index(bank: TemplateBank, sky: int, fdot: int, f: int) -> int:
    """Flat template index: ((sky * n_fdot) + fdot) * n_f + f."""
    return (sky * bank.n_fdot + fdot) * bank.n_f + f


def template_params(bank: TemplateBank, idx):
    """(sky index, fdot index, f index) of flat template indices."""
    idx = np.asarray(idx, dtype=np.int64)
    f = idx % bank.n_f
    r = idx // bank.n_f
    return r // bank.n_fdot, r % bank.n_fdot, f


def draw_injections(seed: int, stream: int, n: int, f_lo: float, f_hi: float,
                    fdot_lo: float, fdot_hi: float, rho_lo: float, rho_hi: float,
                    log_rho: bool = False) -> list:
    g = philox(seed, stream)
    out = []
    for _ in range(n):
        alpha = g.uniform(0.0, 2.0 * math.pi)
        delta = math.asin(g.uniform(-1.0, 1.0))
        psi = g.uniform(-math.pi / 4, math.pi / 4)
        cosi = g.uniform(-1.0, 1.0)
        phi0 = g.uniform(0.0, 2.0 * math.pi)
        f = g.uniform(f_lo, f_hi)
        fdot = g.uniform(fdot_lo, fdot_hi)
        if log_rho:
            rho = math.exp(g.uniform(math.log(rho_lo), math.log(rho_hi)))
        else:
            rho = g.uniform(rho_lo, rho_hi)
        out.append(Injection(alpha, delta, psi, cosi, phi0, f, fdot, rho))
    return out


def _det(geom: dict, t_start: np.ndarray, bins: np.ndarray) -> DetectorData:
    return DetectorData(lat=geom["lat"], lon=geom["lon"], az=geom["az"],
                        t_start=t_start, bins=bins)


def config0(seed: int = 0) -> Workload:
    """Tiny plain-method case: 1 detector, 60 contiguous SFTs, 64 bins around
    100 Hz, one signal at 100.01 Hz with rho = 20, 4 sky x 200 f x 1 fdot."""
    T = T_SFT
    n_sft = 60
    k_c = int(round(100.01 * T))
    k_lo, n_bins = k_c - 32, 64
    t = contiguous_timestamps(T0, T, n_sft)
    bins = cn_noise(seed, _S_NOISE, (n_sft, n_bins))
    g = philox(seed, _S_INJ)
    alpha = g.uniform(0.0, 2.0 * math.pi)
    delta = math.asin(g.uniform(-1.0, 1.0))
    inj = Injection(alpha, delta, g.uniform(-math.pi / 4, math.pi / 4), g.uniform(-1.0, 1.0),
                    g.uniform(0.0, 2.0 * math.pi), 100.01, 0.0, 20.0)
    sky = np.concatenate([np.array([[alpha, delta]]), random_sky(seed, _S_SKY, 3)], axis=0)
    T_obs = n_sft * T
    df = 1.0 / (2.0 * T_obs)
    bank = TemplateBank(sky=sky, f0=100.01 - 100 * df, df=df, n_f=200,
                        fdot=np.zeros(1), t_ref=T0)
    return Workload("plain-tiny 1det x 60 SFT, 4 sky x 200 f", T, k_lo, n_bins, 8, 20,
                    [_det(DET_H, t, bins)], bank, [inj])


def config1(seed: int = 1000, n_sky: int = 10000, n_sft: int = 1200, n_f: int = 1800,
            n_fdot: int = 10, n_inj: int = 8, sky: np.ndarray | None = None) -> Workload:
    """Workunit-sized plain case: 2 detectors x 1200 gapped SFTs, 1 Hz band at
    100 Hz (1800 bins + 2 x 8 margin), 8 signals with rho in [5, 30];
    templates 10 000 Fibonacci sky x 1800 f (1/T spacing) x 10 fdot in
    [-1e-9, 0]; top-1000.  Keyword arguments shrink it for tests."""
    T = T_SFT
    dterms = 8
    k_lo = int(round(100.0 * T)) - dterms
    n_bins = int(round(1.0 * T)) + 2 * dterms
    dets = []
    for i, geom in enumerate((DET_H, DET_L)):
        t = gapped_timestamps(seed, _S_TIME + i, T0, T, n_sft, 0.7)
        bins = cn_noise(seed, _S_NOISE + i, (n_sft, n_bins))
        dets.append(_det(geom, t, bins))
    margin = 40.0 / T
    injs = draw_injections(seed, _S_INJ, n_inj, 100.0 + margin, 101.0 - margin,
                           -1e-9, 0.0, 5.0, 30.0)
    if sky is None:
        sky = fibonacci_sky(n_sky)
    fdot = -1e-9 * np.arange(n_fdot, dtype=np.float64) / max(n_fdot - 1, 1)
    bank = TemplateBank(sky=sky, f0=100.0, df=1.0 / T, n_f=n_f, fdot=fdot, t_ref=T0)
    return Workload(f"plain-workunit 2det x {n_sft} SFT, {sky.shape[0]} sky x {n_f} f x {n_fdot} fdot",
                    T, k_lo, n_bins, dterms, 1000, dets, bank, injs)


def config_mid(seed: int = 500, n_sft: int = 150, n_bins: int = 120, n_sky: int = 6,
               n_f: int = 150, n_fdot: int = 3, df_bins: float = 1.0) -> Workload:
    """Mid-sized parity case shaped like the workunit: 2 gapped detectors, a
    band narrower than the Doppler excursion at its edges (so windows leave
    the stored band), several template tiles with ragged tails."""
    T = T_SFT
    k_lo = int(round(100.0 * T)) - 8
    dets = []
    for i, geom in enumerate((DET_H, DET_L)):
        t = gapped_timestamps(seed, _S_TIME + i, T0, T, n_sft, 0.7)
        bins = cn_noise(seed, _S_NOISE + i, (n_sft, n_bins))
        dets.append(_det(geom, t, bins))
    f_lo = (k_lo + 30) / T
    injs = draw_injections(seed, _S_INJ, 2, f_lo, f_lo + 40.0 / T, -1e-9, 0.0, 10.0, 20.0)
    sky = np.concatenate([np.array([[injs[0].alpha, injs[0].delta]]),
                          random_sky(seed, _S_SKY, n_sky - 1)], axis=0)
    fdot = -1e-9 * np.arange(n_fdot, dtype=np.float64) / max(n_fdot - 1, 1)
    bank = TemplateBank(sky=sky, f0=(k_lo + 2) / T, df=df_bins / T, n_f=n_f, fdot=fdot, t_ref=T0)
    return Workload(f"mid 2det x {n_sft} SFT", T, k_lo, n_bins, 8, 50, dets, bank, injs)


def config3_specs(n_wu: int = 64, seed: int = 3000) -> list:
    """Seed-drawn shapes of the heterogeneous batch: per workunit the SFT count
    (200-2400 over 1-2 detectors), band (0.1-2 Hz), sky-grid size (100-20 000),
    spindown count (1-20) and number of signals (0-4)."""
    specs = []
    for w in range(n_wu):
        g = philox(seed + w, _S_WU)
        n_sft_total = int(g.integers(200, 2401))
        n_det = int(g.integers(1, 3))
        band = float(g.uniform(0.1, 2.0))
        n_sky = int(g.integers(100, 20001))
        n_fdot = int(g.integers(1, 21))
        n_inj = int(g.integers(0, 5))
        f_base = float(np.round(g.uniform(50.0, 400.0) * T_SFT) / T_SFT)
        specs.append(dict(seed=seed + w, n_sft_total=n_sft_total, n_det=n_det, band=band,
                          n_sky=n_sky, n_fdot=n_fdot, n_inj=n_inj, f_base=f_base))
    return specs


def config3_workunit(spec: dict, n_sky: int | None = None, n_sft_total: int | None = None,
                     band: float | None = None) -> Workload:
    """One workunit of the heterogeneous batch from its spec (overrides shrink it)."""
    T = T_SFT
    dterms = 8
    seed = spec["seed"]
    n_sky = spec["n_sky"] if n_sky is None else n_sky
    n_sft_total = spec["n_sft_total"] if n_sft_total is None else n_sft_total
    band = spec["band"] if band is None else band
    n_f = max(1, int(round(band * T)))
    k0 = int(round(spec["f_base"] * T))
    k_lo = k0 - dterms
    n_bins = n_f + 2 * dterms
    n_det = spec["n_det"]
    counts = [n_sft_total // n_det + (1 if i < n_sft_total % n_det else 0) for i in range(n_det)]
    dets = []
    for i in range(n_det):
        geom = (DET_H, DET_L)[i]
        t = gapped_timestamps(seed, _S_TIME + i, T0, T, counts[i], 0.7)
        bins = cn_noise(seed, _S_NOISE + i, (counts[i], n_bins))
        dets.append(_det(geom, t, bins))
    margin = 40.0 / T
    f_lo = k0 / T
    f_hi = (k0 + n_f) / T
    n_inj = spec["n_inj"] if f_hi - f_lo > 2 * margin else 0
    injs = draw_injections(seed, _S_INJ, n_inj, f_lo + margin, f_hi - margin, -1e-9, 0.0, 8.0, 30.0)
    n_fdot = spec["n_fdot"]
    fdot = -1e-9 * np.arange(n_fdot, dtype=np.float64) / max(n_fdot - 1, 1)
    bank = TemplateBank(sky=fibonacci_sky(n_sky), f0=f_lo, df=1.0 / T, n_f=n_f, fdot=fdot, t_ref=T0)
    return Workload(f"batch-wu seed {seed}", T, k_lo, n_bins, dterms, 100, dets, bank, injs)


_S_LINE = 100


@dataclass
class Line:
    """A detector line: a sinusoid fixed in the detector's frame at the centre
    of stored bin `k` (absolute), amplitude `amp` per SFT bin (noise bins have
    E|X|^2 = 1), phase `phi` at the SFT starts."""
    det: int
    k: int
    amp: float
    phi: float


def add_lines(dets, k_lo: int, lines) -> None:
    """Add each line to its detector's bins in place: a sinusoid at a bin
    centre, sampled at SFT starts on the SFT grid, is the same complex number
    amp e^{i phi} in that one bin of every SFT."""
    for ln in lines:
        b = dets[ln.det].bins
        b[:, ln.k - k_lo] += np.complex64(ln.amp * complex(math.cos(ln.phi), math.sin(ln.phi)))


def config4_workunit(index: int, train: bool = True, n_sft: int = 800, noise_only_frac: float = 0.25,
                     seed_base: int = 4000, n_signals: int = 1, n_lines: int = 0,
                     line_amp: tuple = (1.5, 15.0)) -> Workload:
    """Learned-proposal workunit: 2 detectors x 800 SFTs, 0.5 Hz band, coarse
    grid 64 x 32 sky (alpha, sin delta) x 900 f x 1 fdot.  A quarter of the
    workunits are noise only; the rest carry n_signals signals (one in the
    held-out set; training sets may take more) with log-uniform rho in
    [4, 40], each placed on a coarse template.  n_lines > 0 adds up to that
    many detector lines (uniform count 1..n_lines, random detector,
    log-uniform amplitude in line_amp), each at least 64 coarse frequencies
    from every signal; they are listed in the workload's `lines`."""
    T = T_SFT
    seed = seed_base + (0 if train else 100000) + index
    dterms = 8
    k0 = int(round(120.0 * T))
    n_f = 900
    k_lo = k0 - dterms - 24
    n_bins = n_f + 2 * (dterms + 24)
    dets = []
    for i, geom in enumerate((DET_H, DET_L)):
        t = gapped_timestamps(seed, _S_TIME + i, T0, T, n_sft, 0.7)
        bins = cn_noise(seed, _S_NOISE + i, (n_sft, n_bins))
        dets.append(_det(geom, t, bins))
    g = philox(seed, _S_WU)
    noise_only = g.random() < noise_only_frac
    margin = 40.0 / T
    injs = [] if noise_only else draw_injections(seed, _S_INJ, n_signals, k0 / T + margin,
                                                 (k0 + n_f) / T - margin, 0.0, 0.0, 4.0, 40.0,
                                                 log_rho=True)
    n_a, n_d = 64, 32
    # Neither grid resolves a coherent signal over this span (a template off by
    # 1/8 of a coarse step in f or sky keeps < 0.1 % of 2F), so each signal is
    # moved onto the nearest coarse template: a sky cell centre and a coarse
    # frequency, both of which the 8x finer grid also contains.
    for inj in injs:
        ia = min(n_a - 1, int((inj.alpha % (2 * math.pi)) / (2 * math.pi / n_a)))
        id_ = min(n_d - 1, int((math.sin(inj.delta) + 1.0) / (2.0 / n_d)))
        inj.alpha = (ia + 0.5) * (2 * math.pi / n_a)
        inj.delta = math.asin(-1.0 + (id_ + 0.5) * (2.0 / n_d))
        inj.f = (k0 + round((inj.f - k0 / T) * T)) / T
    a = (np.arange(n_a) + 0.5) * (2 * math.pi / n_a)
    sd = -1.0 + (np.arange(n_d) + 0.5) * (2.0 / n_d)
    A, SD = np.meshgrid(a, sd, indexing="ij")
    sky = np.stack([A.ravel(), np.arcsin(SD.ravel())], axis=1)
    bank = TemplateBank(sky=sky, f0=k0 / T, df=1.0 / T, n_f=n_f, fdot=np.zeros(1), t_ref=T0)
    w = Workload(f"proposal-wu {'train' if train else 'test'} {index}", T, k_lo, n_bins, dterms,
                 100, dets, bank, injs)
    if n_lines > 0:
        gl = philox(seed, _S_LINE)
        sig_f = [int(round((inj.f - k0 / T) * T)) for inj in injs]
        n_here = int(gl.integers(1, n_lines + 1))
        tries = 0
        while len(w.lines) < n_here and tries < 1000:
            tries += 1
            fj = int(gl.integers(20, n_f - 20))
            if any(abs(fj - q) < 64 for q in sig_f) or any(abs(fj + k0 - ln.k) < 8 for ln in w.lines):
                continue
            amp = math.exp(gl.uniform(math.log(line_amp[0]), math.log(line_amp[1])))
            w.lines.append(Line(int(gl.integers(0, 2)), k0 + fj, amp, gl.uniform(0.0, 2.0 * math.pi)))
        add_lines(dets, k_lo, w.lines)
    return w
