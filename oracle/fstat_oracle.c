/* Plain FP64 C restatement of the coherent multi-detector F-statistic.
 *
 * TEST INFRASTRUCTURE.  Only the tests, __graft_entry__.smoke() and the
 * CPU-baseline / reference legs of bench.py may load this library.  It shares
 * no code with the CUDA library (no headers, helpers or constants) and holds
 * the same arithmetic as oracle/fstat_oracle.py, written as plain loops in the
 * order of the paper's F-statistic pseudo-code (Listing 1, Section
 * "Einstein@Home"):
 *
 *   ComputeFStatFreqBand   for each template (frequency, spindown) of the band
 *     ComputeFStat         sum over detectors
 *       ComputeFaFb        sum over the SFTs of one detector of
 *                          some_calculations(SFT), then normalized(...)
 *
 * It exists because the numpy oracle vectorises over templates and runs at a
 * few million template.SFT pairs per second per core; whole-workunit toplists
 * (4.32e11 pairs) need the plain loop.  Its results are pinned against the
 * numpy oracle and against the noise-free closed form (tests/test_oracle_c.py).
 *
 * Readings where the paper is silent are the numpy oracle's:
 *   - Sun-centred equatorial ephemeris: circular orbit of 1 AU in the ecliptic
 *     (obliquity 23.4393 deg, period 3.15581498e7 s, phase origin t = 0) plus
 *     a spherical Earth of radius 6.371e6 m rotating at 2 pi / 86164.0905 s
 *     with the detector's longitude at t = 0; no Einstein or Shapiro delay;
 *   - x-arm azimuth from local North clockwise, y-arm at +90 degrees;
 *     long-wavelength tensor D = (u u - v v) / 2;
 *   - timing and antenna patterns at the SFT midpoint t_m = t_start + T/2;
 *   - window k = k0-D+1 .. k0+D with k0 = floor(kappa_hat); bins outside the
 *     stored band count as zero; kappa < 2^-24 takes the exact limit
 *     z = (-1)^k0 e^{-i Phi} X_k0;
 *   - noise E|X|^2 = 1, 2F = 2 (B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*)) / D with
 *     one combine over all detectors.
 *
 * Build: gcc -O2 -fPIC -shared (no fast-math: IEEE FP64 throughout).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

#define PI 3.14159265358979323846
#define C_LIGHT 299792458.0
#define AU_M 1.495978707e11
#define YEAR_S 3.15581498e7
#define EARTH_R 6.371e6
#define SIDEREAL_DAY_S 86164.0905
#define OBLIQUITY_DEG 23.4393
#define KAPPA_LIMIT (1.0 / 16777216.0) /* 2^-24 */

typedef struct {
    double lat, lon, az;    /* vertex latitude, longitude, x-arm azimuth (rad) */
    int n_sft;
    const double *t_start;  /* [n_sft] SFT start times (s) */
    const float *bins;      /* [n_sft][n_bins][2] complex bins k_lo .. k_lo+n_bins-1 */
} det_t;

/* Position r (m) and velocity v (m/s) of the detector vertex at time t. */
static void det_kinematics(const det_t *d, double t, double r[3], double v[3])
{
    double eps = OBLIQUITY_DEG * PI / 180.0;
    double w_orb = 2.0 * PI / YEAR_S;
    double w_rot = 2.0 * PI / SIDEREAL_DAY_S;
    double th = 2.0 * PI * t / YEAR_S;
    double phi = d->lon + w_rot * t;
    double cl = cos(d->lat), sl = sin(d->lat);
    r[0] = AU_M * cos(th) + EARTH_R * cl * cos(phi);
    r[1] = AU_M * cos(eps) * sin(th) + EARTH_R * cl * sin(phi);
    r[2] = AU_M * sin(eps) * sin(th) + EARTH_R * sl;
    v[0] = -AU_M * w_orb * sin(th) - EARTH_R * w_rot * cl * sin(phi);
    v[1] = AU_M * w_orb * cos(eps) * cos(th) + EARTH_R * w_rot * cl * cos(phi);
    v[2] = AU_M * w_orb * sin(eps) * cos(th);
}

/* Antenna-pattern coefficients a = D:(XX - YY), b = D:(XY + YX) at time t. */
static void det_antenna(const det_t *d, double t, double alpha, double delta, double *a, double *b)
{
    double phi = d->lon + (2.0 * PI / SIDEREAL_DAY_S) * t;
    double east[3] = {-sin(phi), cos(phi), 0.0};
    double north[3] = {-sin(d->lat) * cos(phi), -sin(d->lat) * sin(phi), cos(d->lat)};
    double u[3], w[3], X[3], Y[3], D[3][3];
    for (int i = 0; i < 3; i++) {
        u[i] = cos(d->az) * north[i] + sin(d->az) * east[i];
        w[i] = -sin(d->az) * north[i] + cos(d->az) * east[i];
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++)
            D[i][j] = 0.5 * (u[i] * u[j] - w[i] * w[j]);
    X[0] = -sin(alpha); X[1] = cos(alpha); X[2] = 0.0;
    Y[0] = -sin(delta) * cos(alpha); Y[1] = -sin(delta) * sin(alpha); Y[2] = cos(delta);
    double xdx = 0.0, ydy = 0.0, xdy = 0.0;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            xdx += X[i] * D[i][j] * X[j];
            ydy += Y[i] * D[i][j] * Y[j];
            xdy += X[i] * D[i][j] * Y[j];
        }
    *a = xdx - ydy;
    *b = 2.0 * xdy;
}

/* Per-SFT timing at the midpoint: dtau = (t_m - t_ref) + n.r/c, tdot = 1 + n.v/c. */
typedef struct { double dtau, tdot, a, b; } sft_state;

static void sky_state(const det_t *d, double T, double alpha, double delta, double t_ref, sft_state *out)
{
    double n[3] = {cos(delta) * cos(alpha), cos(delta) * sin(alpha), sin(delta)};
    for (int s = 0; s < d->n_sft; s++) {
        double tm = d->t_start[s] + 0.5 * T, r[3], v[3];
        det_kinematics(d, tm, r, v);
        out[s].dtau = (tm - t_ref) + (n[0] * r[0] + n[1] * r[1] + n[2] * r[2]) / C_LIGHT;
        out[s].tdot = 1.0 + (n[0] * v[0] + n[1] * v[1] + n[2] * v[2]) / C_LIGHT;
        det_antenna(d, tm, alpha, delta, &out[s].a, &out[s].b);
    }
}

/* some_calculations: the contribution z of one SFT to one template,
 *   z = (-1)^k0 e^{-i Phi} (sin pi kappa / pi) sum_{k=k0-D+1}^{k0+D} X_k / (kappa_hat - k). */
static void some_calculations(const float *row, int64_t k_lo, int n_bins, int dterms,
                              double f, double fdot, const sft_state *st, double T,
                              double *zr, double *zi)
{
    double cyc = f * st->dtau + 0.5 * fdot * st->dtau * st->dtau;
    double frac = cyc - floor(cyc);
    double kh = (f + fdot * st->dtau) * st->tdot * T;
    double k0f = floor(kh);
    int64_t k0 = (int64_t)k0f;
    double kappa = kh - k0f;
    double qr = 0.0, qi = 0.0, x0r = 0.0, x0i = 0.0;
    for (int n = -dterms + 1; n <= dterms; n++) {
        int64_t j = k0 + n - k_lo;
        double xr = 0.0, xi = 0.0;
        if (j >= 0 && j < n_bins) {
            xr = (double)row[2 * j];
            xi = (double)row[2 * j + 1];
        }
        if (n == 0) { x0r = xr; x0i = xi; }
        double den = kappa - n;
        if (den != 0.0) {
            double inv = 1.0 / den;
            qr += xr * inv;
            qi += xi * inv;
        }
    }
    double sgn = (k0 & 1) ? -1.0 : 1.0;
    double rr = sgn * cos(2.0 * PI * frac), ri = -sgn * sin(2.0 * PI * frac);  /* (-1)^k0 e^{-i Phi} */
    if (kappa < KAPPA_LIMIT) {
        *zr = rr * x0r - ri * x0i;
        *zi = rr * x0i + ri * x0r;
        return;
    }
    double s = sin(PI * kappa) / PI;
    *zr = s * (rr * qr - ri * qi);
    *zi = s * (rr * qi + ri * qr);
}

/* 2F of n_t templates (f[i], fdot[i]) at one sky position, over all detectors. */
static int fstat_sky(int n_det, const det_t *dets, double T, int64_t k_lo, int n_bins, int dterms,
                     double alpha, double delta, double t_ref,
                     int64_t n_t, const double *f, const double *fdot, double *twoF)
{
    sft_state *st[8];
    double A = 0.0, B = 0.0, C = 0.0;
    if (n_det > 8) return -1;
    for (int k = 0; k < n_det; k++) {
        st[k] = (sft_state *)malloc(sizeof(sft_state) * (size_t)(dets[k].n_sft > 0 ? dets[k].n_sft : 1));
        if (!st[k]) { for (int m = 0; m < k; m++) free(st[m]); return -2; }
        sky_state(&dets[k], T, alpha, delta, t_ref, st[k]);
        double a2 = 0.0, b2 = 0.0, ab = 0.0;
        for (int s = 0; s < dets[k].n_sft; s++) {
            a2 += st[k][s].a * st[k][s].a;
            b2 += st[k][s].b * st[k][s].b;
            ab += st[k][s].a * st[k][s].b;
        }
        A += a2; B += b2; C += ab;
    }
    double Dd = A * B - C * C;
    for (int64_t t = 0; t < n_t; t++) {                       /* ComputeFStatFreqBand */
        double far = 0.0, fai = 0.0, fbr = 0.0, fbi = 0.0;
        for (int k = 0; k < n_det; k++) {                     /* ComputeFStat */
            double dar = 0.0, dai = 0.0, dbr = 0.0, dbi = 0.0;
            for (int s = 0; s < dets[k].n_sft; s++) {         /* ComputeFaFb */
                double zr, zi;
                some_calculations(dets[k].bins + (size_t)s * (size_t)n_bins * 2, k_lo, n_bins, dterms,
                                  f[t], fdot[t], &st[k][s], T, &zr, &zi);
                dar += st[k][s].a * zr; dai += st[k][s].a * zi;
                dbr += st[k][s].b * zr; dbi += st[k][s].b * zi;
            }
            far += dar; fai += dai; fbr += dbr; fbi += dbi;
        }
        /* normalized: 2F = 2 (B |Fa|^2 + A |Fb|^2 - 2 C Re(Fa Fb*)) / D, sigma^2 = 1 */
        double q = B * (far * far + fai * fai) + A * (fbr * fbr + fbi * fbi) - 2.0 * C * (far * fbr + fai * fbi);
        twoF[t] = 2.0 * q / Dd;
    }
    for (int k = 0; k < n_det; k++) free(st[k]);
    return 0;
}

static int make_dets(int n_det, const int *n_sft, const double *geom, const double *t_start,
                     const float *bins, int n_bins, det_t *out)
{
    size_t off_t = 0, off_b = 0;
    if (n_det < 1 || n_det > 8 || n_bins < 1) return -1;
    for (int k = 0; k < n_det; k++) {
        out[k].lat = geom[3 * k];
        out[k].lon = geom[3 * k + 1];
        out[k].az = geom[3 * k + 2];
        out[k].n_sft = n_sft[k];
        out[k].t_start = t_start + off_t;
        out[k].bins = bins + off_b;
        off_t += (size_t)n_sft[k];
        off_b += (size_t)n_sft[k] * (size_t)n_bins * 2;
    }
    return 0;
}

/* 2F over the bank's band at sky points [sky_begin, sky_end):
 *   n_det detectors with n_sft[k] SFTs each, geometry geom[k] = (lat, lon, az) rad;
 *   t_start: all detectors' SFT start times concatenated in detector order;
 *   bins: all detectors' SFTs [n_sft_total][n_bins][2] (complex, FP32 storage);
 *   sky [n_sky][2] (alpha, delta); frequencies f0 + j df, j < n_f; fdot[n_fdot];
 *   out: [sky_end - sky_begin][n_fdot][n_f] FP64, caller-allocated.
 * Returns 0, or a negative value on bad sizes / allocation failure. */
int oracle_fstat_band(int n_det, const int *n_sft, const double *geom, const double *t_start,
                      const float *bins, double T, int64_t k_lo, int n_bins, int dterms,
                      const double *sky, int sky_begin, int sky_end,
                      double f0, double df, int n_f, const double *fdot, int n_fdot, double t_ref,
                      double *out)
{
    det_t dets[8];
    if (make_dets(n_det, n_sft, geom, t_start, bins, n_bins, dets) != 0) return -1;
    if (n_f < 1 || n_fdot < 1 || sky_end < sky_begin) return -1;
    int64_t n_t = (int64_t)n_f * n_fdot;
    double *f = (double *)malloc(sizeof(double) * (size_t)n_t);
    double *fd = (double *)malloc(sizeof(double) * (size_t)n_t);
    if (!f || !fd) { free(f); free(fd); return -2; }
    for (int m = 0; m < n_fdot; m++)
        for (int j = 0; j < n_f; j++) {
            f[(int64_t)m * n_f + j] = f0 + (double)j * df;
            fd[(int64_t)m * n_f + j] = fdot[m];
        }
    int rc = 0;
    for (int s = sky_begin; s < sky_end && rc == 0; s++)
        rc = fstat_sky(n_det, dets, T, k_lo, n_bins, dterms, sky[2 * s], sky[2 * s + 1], t_ref,
                       n_t, f, fd, out + (int64_t)(s - sky_begin) * n_t);
    free(f);
    free(fd);
    return rc;
}

/* 2F of arbitrary flat template indices ((sky * n_fdot) + fdot) * n_f + f of
 * the same bank; indices sharing a sky point are grouped by the caller or
 * not (each index is computed on its own; the per-SFT state is recomputed
 * whenever the sky point changes from one index to the next). */
int oracle_fstat_templates(int n_det, const int *n_sft, const double *geom, const double *t_start,
                           const float *bins, double T, int64_t k_lo, int n_bins, int dterms,
                           const double *sky, double f0, double df, int n_f, const double *fdot, int n_fdot,
                           double t_ref, const int64_t *idx, int64_t n_idx, double *out)
{
    det_t dets[8];
    if (make_dets(n_det, n_sft, geom, t_start, bins, n_bins, dets) != 0) return -1;
    if (n_f < 1 || n_fdot < 1) return -1;
    int64_t i = 0;
    while (i < n_idx) {
        int64_t s = idx[i] / ((int64_t)n_fdot * n_f);
        int64_t e = i;
        while (e < n_idx && idx[e] / ((int64_t)n_fdot * n_f) == s) e++;
        int64_t n = e - i;
        double *f = (double *)malloc(sizeof(double) * (size_t)n);
        double *fd = (double *)malloc(sizeof(double) * (size_t)n);
        if (!f || !fd) { free(f); free(fd); return -2; }
        for (int64_t q = 0; q < n; q++) {
            int64_t r = idx[i + q] % ((int64_t)n_fdot * n_f);
            f[q] = f0 + (double)(r % n_f) * df;
            fd[q] = fdot[r / n_f];
        }
        int rc = fstat_sky(n_det, dets, T, k_lo, n_bins, dterms, sky[2 * s], sky[2 * s + 1], t_ref,
                           n, f, fd, out + i);
        free(f);
        free(fd);
        if (rc) return rc;
        i = e;
    }
    return 0;
}
