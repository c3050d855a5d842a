"""Plain FP64 CPU oracle of the coherent multi-detector F-statistic over SFTs.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import or run this module.
It shares no code with the CUDA library: no kernels, headers, helpers or
constants; the seeded inputs it reads come from the separate ``workload``
generator.

What it computes follows the loop structure of the paper's F-statistic
pseudo-code (Listing 1, Section "Einstein@Home"):

    ComputeFStatFreqBand   for each frequency (template) of the band
      ComputeFStat         sum over detectors
        ComputeFaFb        sum over the SFTs of one detector of
                           some_calculations(SFT), then normalized(...)

The paper does not print the body of ``some_calculations`` or ``normalized``.
The oracle takes the standard SFT demodulation of the F-statistic literature
that the Einstein@Home client implements: the phase is linearised about each
SFT's midpoint, the data are matched against the Dirichlet kernel over 2*Dterms
bins around the instantaneous frequency, weighted by the antenna-pattern
coefficients a, b, and combined with A = sum a^2, B = sum b^2, C = sum ab,
D = AB - C^2 into 2F.  Every formula is written out directly in FP64 with
numpy, vectorised over templates only; nothing is blocked or reordered.

Readings where the paper is silent, taken here:
  * synthetic Sun-centred ephemeris (circular orbit in the ecliptic plane,
    spherical rotating Earth), no Einstein or Shapiro delays;
  * x-arm azimuth from local North clockwise, y-arm at +90 degrees;
  * phase expansion about the SFT midpoint, window k0-D+1 .. k0+D with
    k0 = floor(kappa_hat);
  * noise with E|X|^2 = 1 (sigma^2 = 1); 2F normalised so E[2F] = 4 on noise
    as D -> infinity;
  * kappa < 2^-24 uses the exact limit z = (-1)^k0 e^{-i Phi} X_k0;
  * window bins outside the stored band count as zero;
  * one global combine over all detectors (not one per detector).
"""
from __future__ import annotations

import math

import numpy as np

# Physical constants of the synthetic ephemeris.
C_LIGHT = 299792458.0                 # m/s
AU_M = 1.495978707e11                 # m, orbital radius
OBLIQUITY = math.radians(23.4393)     # ecliptic obliquity
YEAR_S = 3.15581498e7                 # s, orbital period
EARTH_R = 6.371e6                     # m, Earth radius
SIDEREAL_W = 2.0 * math.pi / 86164.0905   # rad/s, Earth rotation rate
T_EQUINOX = 0.0                       # orbital phase origin

KAPPA_LIMIT = 2.0 ** -24              # below this kappa uses the exact limit


# ---------------------------------------------------------------------------
# Detector kinematics and response
# ---------------------------------------------------------------------------

def detector_position_velocity(lat: float, lon: float, t):
    """Position (m) and velocity (m/s) of a detector vertex, equatorial frame
    centred on the Sun.  r = r_orbit + r_rotation; v = dr/dt analytically."""
    t = np.asarray(t, dtype=np.float64)
    th = 2.0 * math.pi * (t - T_EQUINOX) / YEAR_S
    w_orb = 2.0 * math.pi / YEAR_S
    ce, se = math.cos(OBLIQUITY), math.sin(OBLIQUITY)
    r_orb = np.stack([AU_M * np.cos(th), AU_M * ce * np.sin(th), AU_M * se * np.sin(th)], -1)
    v_orb = np.stack([-AU_M * w_orb * np.sin(th), AU_M * w_orb * ce * np.cos(th),
                      AU_M * w_orb * se * np.cos(th)], -1)
    phi = lon + SIDEREAL_W * t
    cl, sl = math.cos(lat), math.sin(lat)
    r_rot = np.stack([EARTH_R * cl * np.cos(phi), EARTH_R * cl * np.sin(phi),
                      EARTH_R * sl * np.ones_like(phi)], -1)
    v_rot = np.stack([-EARTH_R * SIDEREAL_W * cl * np.sin(phi),
                      EARTH_R * SIDEREAL_W * cl * np.cos(phi), np.zeros_like(phi)], -1)
    return r_orb + r_rot, v_orb + v_rot


def detector_tensor(lat: float, lon: float, az: float, t):
    """Long-wavelength response tensor D = (u u - v v)/2 of an L-shaped
    detector, equatorial components, [..., 3, 3].  u is the x-arm (azimuth az
    from local North, clockwise), v the y-arm (azimuth az + 90 degrees)."""
    t = np.asarray(t, dtype=np.float64)
    phi = lon + SIDEREAL_W * t
    east = np.stack([-np.sin(phi), np.cos(phi), np.zeros_like(phi)], -1)
    north = np.stack([-math.sin(lat) * np.cos(phi), -math.sin(lat) * np.sin(phi),
                      math.cos(lat) * np.ones_like(phi)], -1)
    u = math.cos(az) * north + math.sin(az) * east
    v = -math.sin(az) * north + math.cos(az) * east
    return 0.5 * (u[..., :, None] * u[..., None, :] - v[..., :, None] * v[..., None, :])


def sky_unit_vector(alpha, delta):
    alpha = np.asarray(alpha, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    return np.stack([np.cos(delta) * np.cos(alpha), np.cos(delta) * np.sin(alpha), np.sin(delta)], -1)


def wave_frame(alpha, delta):
    """Polarisation basis X = d n/d alpha normalised, Y = d n/d delta."""
    alpha = np.asarray(alpha, dtype=np.float64)
    delta = np.asarray(delta, dtype=np.float64)
    X = np.stack([-np.sin(alpha), np.cos(alpha), np.zeros_like(alpha)], -1)
    Y = np.stack([-np.sin(delta) * np.cos(alpha), -np.sin(delta) * np.sin(alpha), np.cos(delta)], -1)
    return X, Y


def antenna_ab(Dt, alpha, delta):
    """a = D:(XX - YY), b = D:(XY + YX); F+ = a cos 2psi + b sin 2psi,
    Fx = b cos 2psi - a sin 2psi."""
    X, Y = wave_frame(alpha, delta)
    DX = np.einsum("...ij,...j->...i", Dt, X)
    DY = np.einsum("...ij,...j->...i", Dt, Y)
    a = np.einsum("...i,...i->...", X, DX) - np.einsum("...i,...i->...", Y, DY)
    b = 2.0 * np.einsum("...i,...i->...", X, DY)
    return a, b


def sft_timing_antenna(det, T: float, alpha, delta, t_ref: float):
    """Per-SFT quantities at the SFT midpoints t_m = t_start + T/2 for one sky
    position (alpha, delta scalars) or broadcastable arrays:
      dtau  = (t_m - t_ref) + n.r(t_m)/c   source-frame time since t_ref
      tdot  = 1 + n.v(t_m)/c               d tau / d t
      a, b  = antenna-pattern coefficients at t_m
    """
    t_m = np.asarray(det.t_start, dtype=np.float64) + 0.5 * T
    r, v = detector_position_velocity(det.lat, det.lon, t_m)
    Dt = detector_tensor(det.lat, det.lon, det.az, t_m)
    n = sky_unit_vector(alpha, delta)
    dtau = (t_m - t_ref) + np.einsum("...i,...i->...", n, r) / C_LIGHT
    tdot = 1.0 + np.einsum("...i,...i->...", n, v) / C_LIGHT
    a, b = antenna_ab(Dt, alpha, delta)
    return dtau, tdot, a, b


def abcd(a_list, b_list):
    """A = sum a^2, B = sum b^2, C = sum ab over all SFTs of all detectors, D = AB - C^2."""
    A = sum(float(np.sum(a * a)) for a in a_list)
    B = sum(float(np.sum(b * b)) for b in b_list)
    C = sum(float(np.sum(a * b)) for a, b in zip(a_list, b_list))
    return A, B, C, A * B - C * C


# ---------------------------------------------------------------------------
# Per-SFT term (the body of the SFT loop) and the 2F combine
# ---------------------------------------------------------------------------

def phase_and_kappa(f, fdot, dtau, tdot, T: float):
    """Phase Phi(tau) = 2 pi (f dtau + fdot dtau^2 / 2) at the SFT midpoint, as
    a fraction of a cycle in [0, 1), and the instantaneous frequency in bins
    kappa_hat = (f + fdot dtau) tdot T."""
    cyc = f * dtau + 0.5 * fdot * dtau * dtau
    frac = cyc - np.floor(cyc)
    kappa_hat = (f + fdot * dtau) * tdot * T
    return frac, kappa_hat


def some_calculations(bins_row, k_lo: int, kappa_hat, phase_frac, dterms: int):
    """Contribution z of one SFT to the matched filter, for a vector of
    templates (kappa_hat, phase_frac arrays):

        z = (-1)^k0 e^{-i Phi} (sin pi kappa / pi) sum_{k=k0-D+1}^{k0+D} X_k / (kappa_hat - k)

    k0 = floor(kappa_hat), kappa = kappa_hat - k0; bins outside the stored band
    [k_lo, k_lo + n_bins) count as zero; kappa < 2^-24 takes the exact limit
    z = (-1)^k0 e^{-i Phi} X_k0."""
    n_bins = bins_row.shape[0]
    kappa_hat = np.asarray(kappa_hat, dtype=np.float64)
    k0 = np.floor(kappa_hat).astype(np.int64)
    kappa = kappa_hat - k0
    Q = np.zeros(kappa_hat.shape, dtype=np.complex128)
    x_k0 = np.zeros(kappa_hat.shape, dtype=np.complex128)
    for n in range(-dterms + 1, dterms + 1):
        j = k0 + n - k_lo
        inside = (j >= 0) & (j < n_bins)
        X = np.where(inside, bins_row[np.clip(j, 0, n_bins - 1)].astype(np.complex128), 0.0)
        denom = kappa - n
        with np.errstate(divide="ignore", invalid="ignore"):
            Q = Q + np.where(denom != 0.0, X / np.where(denom != 0.0, denom, 1.0), 0.0)
        if n == 0:
            x_k0 = X
    sign = 1.0 - 2.0 * (k0 & 1).astype(np.float64)
    rot = sign * np.exp(-2j * math.pi * phase_frac)
    z = rot * (np.sin(math.pi * kappa) / math.pi) * Q
    small = kappa < KAPPA_LIMIT
    return np.where(small, rot * x_k0, z)


def compute_fa_fb(det, T: float, k_lo: int, dterms: int, alpha, delta, f, fdot, t_ref: float):
    """Fa, Fb of one detector summed over its SFTs, and that detector's
    a, b arrays (for A, B, C).  alpha, delta are scalars (one sky position);
    f, fdot are equal-shape template arrays.  A detector with per-SFT noise
    weights w (attribute `weights`, whitened bins) uses sqrt(w) a, sqrt(w) b."""
    dtau, tdot, a, b = sft_timing_antenna(det, T, alpha, delta, t_ref)
    w = getattr(det, "weights", None)
    if w is not None:
        sw = np.sqrt(np.asarray(w, dtype=np.float64))
        a = a * sw
        b = b * sw
    f = np.asarray(f, dtype=np.float64)
    fdot = np.asarray(fdot, dtype=np.float64)
    Fa = np.zeros(f.shape, dtype=np.complex128)
    Fb = np.zeros(f.shape, dtype=np.complex128)
    for s in range(det.n_sft if hasattr(det, "n_sft") else len(det.t_start)):
        frac, kh = phase_and_kappa(f, fdot, dtau[s], tdot[s], T)
        z = some_calculations(det.bins[s], k_lo, kh, frac, dterms)
        Fa += a[s] * z
        Fb += b[s] * z
    return Fa, Fb, a, b


def normalized(Fa, Fb, A: float, B: float, C: float, D: float, sigma2: float = 1.0):
    """2F = (2 / sigma^2) (B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*)) / D."""
    q = B * np.abs(Fa) ** 2 + A * np.abs(Fb) ** 2 - 2.0 * C * np.real(Fa * np.conj(Fb))
    return 2.0 * q / (sigma2 * D)


def compute_fstat(dets, T: float, k_lo: int, dterms: int, alpha, delta, f, fdot, t_ref: float,
                  return_parts: bool = False):
    """2F at one sky position for template arrays f, fdot: Fa, Fb, A, B, C
    summed over all detectors, then one combine."""
    Fa = 0.0
    Fb = 0.0
    a_all, b_all = [], []
    for det in dets:
        fa, fb, a, b = compute_fa_fb(det, T, k_lo, dterms, alpha, delta, f, fdot, t_ref)
        Fa = Fa + fa
        Fb = Fb + fb
        a_all.append(a)
        b_all.append(b)
    A, B, C, D = abcd(a_all, b_all)
    twoF = normalized(Fa, Fb, A, B, C, D)
    if return_parts:
        return twoF, dict(Fa=Fa, Fb=Fb, A=A, B=B, C=C, D=D)
    return twoF


def compute_fstat_freq_band(dets, T: float, k_lo: int, dterms: int, bank, sky_indices=None):
    """2F over a template bank, [n_sky_sel, n_fdot, n_f] float64, for each
    frequency f_j = f0 + j df and spindown of the bank, at the selected sky
    points (all by default)."""
    if sky_indices is None:
        sky_indices = range(bank.sky.shape[0])
    j = np.arange(bank.n_f, dtype=np.float64)
    f = bank.f0 + j * bank.df
    F, FD = np.meshgrid(f, np.asarray(bank.fdot, dtype=np.float64), indexing="xy")
    out = []
    for s in sky_indices:
        alpha, delta = bank.sky[s]
        out.append(compute_fstat(dets, T, k_lo, dterms, alpha, delta, F, FD, bank.t_ref))
    return np.stack(out, 0)


def compute_fstat_templates(dets, T: float, k_lo: int, dterms: int, bank, indices):
    """2F of arbitrary flat template indices ((sky*n_fdot)+fdot)*n_f + f."""
    indices = np.asarray(indices, dtype=np.int64)
    f_idx = indices % bank.n_f
    r = indices // bank.n_f
    fd_idx = r % bank.n_fdot
    s_idx = r // bank.n_fdot
    out = np.empty(indices.shape[0], dtype=np.float64)
    for s in np.unique(s_idx):
        sel = np.nonzero(s_idx == s)[0]
        f = bank.f0 + f_idx[sel].astype(np.float64) * bank.df
        fd = np.asarray(bank.fdot, dtype=np.float64)[fd_idx[sel]]
        alpha, delta = bank.sky[s]
        out[sel] = compute_fstat(dets, T, k_lo, dterms, alpha, delta, f, fd, bank.t_ref)
    return out


def toplist(twoF_flat, k: int):
    """The k largest 2F, ordered by (2F descending, template index ascending)."""
    v = np.asarray(twoF_flat).ravel()
    idx = np.arange(v.shape[0], dtype=np.int64)
    order = np.lexsort((idx, -v))[:k]
    return idx[order], v[order]


# ---------------------------------------------------------------------------
# Model-exact signal in the SFT domain (for injections and closed forms)
# ---------------------------------------------------------------------------

def signal_amplitudes(psi: float, cosi: float, phi0: float, h0: float = 1.0):
    """Complex amplitudes of h = Re[(a c_a + b c_b) e^{i Phi}] for
    h = F+ A+ cos(Phi + phi0) + Fx Ax sin(Phi + phi0)."""
    ap = h0 * (1.0 + cosi * cosi) / 2.0
    ax = h0 * cosi
    e = complex(math.cos(phi0), math.sin(phi0))
    ca = (ap * math.cos(2 * psi) + 1j * ax * math.sin(2 * psi)) * e
    cb = (ap * math.sin(2 * psi) - 1j * ax * math.cos(2 * psi)) * e
    return ca, cb


def optimal_rho2(T: float, A: float, B: float, C: float, ca: complex, cb: complex, sigma2: float = 1.0):
    """rho^2 = (T^2 / (2 sigma^2)) (A |c_a|^2 + B |c_b|^2 + 2 C Re(c_a c_b*)),
    the noise-free 2F at the true template as Dterms -> infinity."""
    q = A * abs(ca) ** 2 + B * abs(cb) ** 2 + 2.0 * C * (ca * np.conj(cb)).real
    return (T * T / (2.0 * sigma2)) * q


def injection_h0(dets, T: float, inj, t_ref: float) -> float:
    """Amplitude h0 that gives the injection its target optimal SNR rho."""
    a_all, b_all = [], []
    for det in dets:
        _, _, a, b = sft_timing_antenna(det, T, inj.alpha, inj.delta, t_ref)
        a_all.append(a)
        b_all.append(b)
    A, B, C, _ = abcd(a_all, b_all)
    ca, cb = signal_amplitudes(inj.psi, inj.cosi, inj.phi0, 1.0)
    return inj.rho / math.sqrt(optimal_rho2(T, A, B, C, ca, cb))


def signal_bins(det, T: float, k_lo: int, n_bins: int, inj, h0: float, t_ref: float):
    """Noise-free SFT bins of a signal, [n_sft, n_bins] complex128:
    X_k = (T/2)(a c_a + b c_b) e^{i Phi_alpha} (-1)^k sinc(kappa_hat - k),
    the Fourier transform of the signal with its phase linearised about the
    SFT midpoint (the positive-frequency half of a real signal)."""
    dtau, tdot, a, b = sft_timing_antenna(det, T, inj.alpha, inj.delta, t_ref)
    ca, cb = signal_amplitudes(inj.psi, inj.cosi, inj.phi0, h0)
    frac, kh = phase_and_kappa(inj.f, inj.fdot, dtau, tdot, T)
    k = k_lo + np.arange(n_bins, dtype=np.int64)
    sign_k = 1.0 - 2.0 * (k & 1).astype(np.float64)
    amp = 0.5 * T * (a * ca + b * cb) * np.exp(2j * math.pi * frac)
    return amp[:, None] * sign_k[None, :] * np.sinc(kh[:, None] - k[None, :])


def inject(dets, T: float, k_lo: int, injections, t_ref: float):
    """Return copies of the detectors' bins with all signals added (sums in
    FP64, stored back as complex64 like the input)."""
    out = []
    for det in dets:
        n_bins = det.bins.shape[1]
        acc = det.bins.astype(np.complex128)
        for inj in injections:
            h0 = injection_h0(dets, T, inj, t_ref)
            acc = acc + signal_bins(det, T, k_lo, n_bins, inj, h0, t_ref)
        out.append(acc.astype(np.complex64))
    return out


def closed_form_fa_fb(dets, T: float, dterms: int, inj, h0: float, t_ref: float):
    """Noise-free Fa, Fb at the true template of a model-exact injection:
    Fa = (T/2) sum a t (a c_a + b c_b), Fb = (T/2) sum b t (a c_a + b c_b), with
    t = sum over the 2D window of sin^2(pi kappa) / (pi^2 (kappa - n)^2)."""
    ca, cb = signal_amplitudes(inj.psi, inj.cosi, inj.phi0, h0)
    Fa = 0.0
    Fb = 0.0
    for det in dets:
        dtau, tdot, a, b = sft_timing_antenna(det, T, inj.alpha, inj.delta, t_ref)
        _, kh = phase_and_kappa(inj.f, inj.fdot, dtau, tdot, T)
        kappa = kh - np.floor(kh)
        t = np.zeros_like(kappa)
        for n in range(-dterms + 1, dterms + 1):
            with np.errstate(divide="ignore", invalid="ignore"):
                t = t + np.where(kappa - n != 0.0,
                                 np.sin(math.pi * kappa) ** 2 / (math.pi ** 2 * (kappa - n) ** 2), 0.0)
        t = np.where(kappa < KAPPA_LIMIT, 1.0, t)
        s = a * ca + b * cb
        Fa = Fa + 0.5 * T * np.sum(a * t * s)
        Fb = Fb + 0.5 * T * np.sum(b * t * s)
    return Fa, Fb
