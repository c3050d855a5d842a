// FP64 part of the path: detector state per SFT, and per (sky, SFT) timing,
// antenna patterns, A/B/C/D and the fixed-point bases of the bin offset
// kappa_hat and the phase Phi that the FP32 Dirichlet kernel steps through.
//
// The phase argument 2 pi f t at t ~ 1e7-1e8 s needs FP64 (the paper's
// CUDA port ran in FP32 only and notes its results were of no scientific
// value, Section "CUDA", final version); everything that touches absolute
// time stays here, and the hot kernel only sees fixed-point offsets.
#include "fstat_internal.cuh"

namespace fs {

namespace {

__device__ __forceinline__ void detector_state(double lat, double lon, double az, double t,
                                               SftState& s) {
    const double w_orb = kTwoPi / kYear;
    const double w_rot = kTwoPi / kSidereal;
    const double th = w_orb * t;
    double sth, cth;
    sincos(th, &sth, &cth);
    double se, ce;
    sincos(kObliquity, &se, &ce);
    const double phi = lon + w_rot * t;
    double sph, cph;
    sincos(phi, &sph, &cph);
    double sl, cl;
    sincos(lat, &sl, &cl);
    s.r[0] = kAU * cth + kEarthR * cl * cph;
    s.r[1] = kAU * ce * sth + kEarthR * cl * sph;
    s.r[2] = kAU * se * sth + kEarthR * sl;
    s.v[0] = -kAU * w_orb * sth - kEarthR * w_rot * cl * sph;
    s.v[1] = kAU * w_orb * ce * cth + kEarthR * w_rot * cl * cph;
    s.v[2] = kAU * w_orb * se * cth;
    // local East / North at the vertex, arms u (azimuth az) and v (az + 90 deg)
    const double e[3] = {-sph, cph, 0.0};
    const double n[3] = {-sl * cph, -sl * sph, cl};
    double sa, ca;
    sincos(az, &sa, &ca);
    double u[3], w[3];
    for (int i = 0; i < 3; ++i) {
        u[i] = ca * n[i] + sa * e[i];
        w[i] = -sa * n[i] + ca * e[i];
    }
    s.dt[0] = 0.5 * (u[0] * u[0] - w[0] * w[0]);
    s.dt[1] = 0.5 * (u[0] * u[1] - w[0] * w[1]);
    s.dt[2] = 0.5 * (u[0] * u[2] - w[0] * w[2]);
    s.dt[3] = 0.5 * (u[1] * u[1] - w[1] * w[1]);
    s.dt[4] = 0.5 * (u[1] * u[2] - w[1] * w[2]);
    s.dt[5] = 0.5 * (u[2] * u[2] - w[2] * w[2]);
}

__global__ void sft_state_kernel(const double* __restrict__ t_start, const int* __restrict__ det_of,
                                 fstat_detector d0, fstat_detector d1, fstat_detector d2,
                                 fstat_detector d3, fstat_detector d4, fstat_detector d5,
                                 fstat_detector d6, fstat_detector d7, int n_sft, double T,
                                 SftState* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sft) return;
    const fstat_detector dets[8] = {d0, d1, d2, d3, d4, d5, d6, d7};
    const fstat_detector g = dets[det_of[i] & 7];
    SftState s;
    s.t_mid = t_start[i] + 0.5 * T;
    detector_state(g.lat_rad, g.lon_rad, g.xarm_az_rad, s.t_mid, s);
    out[i] = s;
}

struct SkyFrame {
    double n[3], X[3], Y[3];
};

__device__ __forceinline__ SkyFrame sky_frame(double alpha, double delta) {
    double sa, ca, sd, cd;
    sincos(alpha, &sa, &ca);
    sincos(delta, &sd, &cd);
    SkyFrame f;
    f.n[0] = cd * ca;
    f.n[1] = cd * sa;
    f.n[2] = sd;
    f.X[0] = -sa;
    f.X[1] = ca;
    f.X[2] = 0.0;
    f.Y[0] = -sd * ca;
    f.Y[1] = -sd * sa;
    f.Y[2] = cd;
    return f;
}

// dtau, tdot, a, b of one SFT for one sky frame.
__device__ __forceinline__ void timing_antenna(const SftState& s, const SkyFrame& f, double t_ref,
                                               double& dtau, double& tdot, double& a, double& b) {
    const double nr = f.n[0] * s.r[0] + f.n[1] * s.r[1] + f.n[2] * s.r[2];
    const double nv = f.n[0] * s.v[0] + f.n[1] * s.v[1] + f.n[2] * s.v[2];
    dtau = (s.t_mid - t_ref) + nr / kC;
    tdot = 1.0 + nv / kC;
    const double* D = s.dt;
    const double DX[3] = {D[0] * f.X[0] + D[1] * f.X[1] + D[2] * f.X[2],
                          D[1] * f.X[0] + D[3] * f.X[1] + D[4] * f.X[2],
                          D[2] * f.X[0] + D[4] * f.X[1] + D[5] * f.X[2]};
    const double DY[3] = {D[0] * f.Y[0] + D[1] * f.Y[1] + D[2] * f.Y[2],
                          D[1] * f.Y[0] + D[3] * f.Y[1] + D[4] * f.Y[2],
                          D[2] * f.Y[0] + D[4] * f.Y[1] + D[5] * f.Y[2]};
    const double xdx = f.X[0] * DX[0] + f.X[1] * DX[1] + f.X[2] * DX[2];
    const double ydy = f.Y[0] * DY[0] + f.Y[1] * DY[1] + f.Y[2] * DY[2];
    const double xdy = f.X[0] * DY[0] + f.X[1] * DY[1] + f.X[2] * DY[2];
    a = xdx - ydy;
    b = 2.0 * xdy;
}

constexpr double kTwo32 = 4294967296.0;

// Fractional part of x in cycles as a 32-bit fixed-point number (wraps mod 1).
__device__ __forceinline__ unsigned int frac_fx32(double x) {
    const double fr = x - floor(x);
    const double s = rint(fr * kTwo32);
    return (unsigned int)(unsigned long long)(long long)s;   // 2^32 wraps to 0
}

// Absolute bin position as 32.32 fixed point.
__device__ __forceinline__ long long bin_fx(double khat) {
    const double hi = floor(khat);
    const double lo = rint((khat - hi) * kTwo32);
    return ((long long)hi << 32) + (long long)lo;
}

template <int BLOCK>
__device__ __forceinline__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (l < BLOCK / 32) ? red[l] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

constexpr int kTimingBlock = 256;

__global__ void __launch_bounds__(kTimingBlock) timing_kernel(const TimingParams p) {
    __shared__ double red[3][kTimingBlock / 32];
    const int sky = blockIdx.x;
    const SkyFrame fr = sky_frame(p.sky[2 * sky], p.sky[2 * sky + 1]);
    const double kconst = 2.0 / kPi;   // pair form of the Dirichlet sum and the 1/pi of sin(pi kappa)/pi
    double sAA = 0.0, sBB = 0.0, sAB = 0.0;
    for (int i = threadIdx.x; i < p.n_sft; i += kTimingBlock) {
        const SftState s = p.st[i];
        double dtau, tdot, a, b;
        timing_antenna(s, fr, p.t_ref, dtau, tdot, a, b);
        if (p.weight) {   // noise weights: sqrt(w) a, sqrt(w) b in A, B, C and in Fa, Fb
            const double sw = sqrt(p.weight[i]);
            a *= sw;
            b *= sw;
        }
        sAA += a * a;
        sBB += b * b;
        sAB += a * b;
        const double dk_real = p.df * tdot * p.T;
        const long long dk = llrint(dk_real * kTwo32);
        const long long pdk = (long long)p.P * dk;
        SkySftMeta m;
        m.dk = dk;
        m.span = (long long)(p.M - 1) * pdk;
        const unsigned int dphi = frac_fx32(p.df * dtau);
        m.dphi = dphi;
        m.eps = (float)((double)(pdk - ((long long)p.L << 32)) / kTwo32);
        // twiddle step e^{-2 pi i (P dphi + L/2)} from the same fixed-point step:
        // a reduced angle (the step in [-1/2, 1/2) cycle) whose sine and cosine
        // are stored in FP32, so they are taken in FP32 (error ~2e-7 rad from
        // rounding the 32-bit step to 24 bits; the kernels' own twiddles are
        // FP32 too)
        const unsigned int step = (unsigned int)p.P * dphi + ((unsigned int)p.L << 31);
        float sn, cs;
        sincospif((float)(int)step * 4.656612873077393e-10f, &sn, &cs);   // x 2^-31: half cycles
        m.rot_re = cs;
        m.rot_im = -sn;
        const double sc = (double)p.scale[i] * kconst;
        m.a = (float)(a * sc);
        m.b = (float)(b * sc);
        long long khmin = 0x7fffffffffffffffLL;
        if (p.uniform) {
            const double fd = p.fdot[0];
            SkySftBase bs;
            bs.kh0 = bin_fx((p.f0 + fd * dtau) * tdot * p.T);
            bs.dkh = llrint(p.dfdot * dtau * tdot * p.T * kTwo32);
            bs.ph0 = frac_fx32(p.f0 * dtau + 0.5 * fd * dtau * dtau);
            bs.dph = frac_fx32(0.5 * p.dfdot * dtau * dtau);
            // twiddle step from one spindown row to the next, e^{-2 pi i dph}
            // (read by the row-tiled forms only)
            float rs = 0.f, rc = 1.f;
            if (p.row_rot) sincospif((float)(int)bs.dph * 4.656612873077393e-10f, &rs, &rc);
            bs.rot_re = rc;
            bs.rot_im = -rs;
            p.base[p.sft_major ? (size_t)i * p.n_sky + (p.sky_rank ? p.sky_rank[sky] : sky)
                               : (size_t)sky * p.n_sft + i] = bs;
            const long long last = bs.kh0 + (long long)(p.n_fdot - 1) * bs.dkh;
            khmin = bs.kh0 < last ? bs.kh0 : last;
        } else {
            for (int d = 0; d < p.n_fdot; ++d) {
                const double fd = p.fdot[d];
                const double khat0 = (p.f0 + fd * dtau) * tdot * p.T;
                const double cyc0 = p.f0 * dtau + 0.5 * fd * dtau * dtau;
                const size_t o = ((size_t)sky * p.n_fdot + d) * p.n_sft + i;
                const long long kfx = bin_fx(khat0);
                p.kh0[o] = kfx;
                p.ph0[o] = frac_fx32(cyc0);
                khmin = kfx < khmin ? kfx : khmin;
            }
        }
        m.khmin = khmin;
        p.meta[p.sft_major ? (size_t)i * p.n_sky + (p.sky_rank ? p.sky_rank[sky] : sky)
                           : (size_t)sky * p.n_sft + i] = m;
    }
    const double A = block_sum<kTimingBlock>(sAA, red[0]);
    const double B = block_sum<kTimingBlock>(sBB, red[1]);
    const double C = block_sum<kTimingBlock>(sAB, red[2]);
    if (threadIdx.x == 0) {
        const double D = A * B - C * C;
        p.abcd[4 * sky + 0] = A;
        p.abcd[4 * sky + 1] = B;
        p.abcd[4 * sky + 2] = C;
        p.abcd[4 * sky + 3] = D;
        if (D > 1e-300 && D > 1e-13 * A * B) {
            p.comb[sky] = make_float4((float)(2.0 * B / D), (float)(2.0 * A / D), (float)(-4.0 * C / D), 1.f);
        } else {
            p.comb[sky] = make_float4(0.f, 0.f, 0.f, 0.f);
            atomicOr(p.err, 2);
        }
    }
}

// Per-frequency A, B, C of one sky point over the SFTs whose coverage
// [x, y) holds the frequency index: a^2, b^2, ab of each SFT (with its noise
// weight) in 2^-36 fixed point go into difference arrays at x and y (integer
// atomics: exact and order-free), a prefix over j gives A, B, C per j, and
// from them the combine weights.  A frequency no SFT covers gets zero weights
// (2F = 0) without a flag; any other degenerate D raises flag bit 1.
constexpr double kCovScale = 68719476736.0;   // 2^36

__global__ void __launch_bounds__(kTimingBlock) coverage_comb_kernel(const TimingParams p, const int2* __restrict__ cov,
                                                                     int n_f, float4* __restrict__ comb_j) {
    extern __shared__ unsigned long long cdiff[];   // [3][n_f + 1]
    __shared__ unsigned long long tot[3][kTimingBlock];
    const int sky = blockIdx.x;
    const int n1 = n_f + 1;
    for (int t = threadIdx.x; t < 3 * n1; t += kTimingBlock) cdiff[t] = 0ull;
    __syncthreads();
    const SkyFrame fr = sky_frame(p.sky[2 * sky], p.sky[2 * sky + 1]);
    for (int i = threadIdx.x; i < p.n_sft; i += kTimingBlock) {
        const int2 c = cov[i];
        const int lo = max(0, min(c.x, n_f)), hi = max(0, min(c.y, n_f));
        if (lo >= hi) continue;
        double dtau, tdot, a, b;
        timing_antenna(p.st[i], fr, p.t_ref, dtau, tdot, a, b);
        if (p.weight) {
            const double sw = sqrt(p.weight[i]);
            a *= sw;
            b *= sw;
        }
        const unsigned long long q[3] = {(unsigned long long)llrint(a * a * kCovScale),
                                         (unsigned long long)llrint(b * b * kCovScale),
                                         (unsigned long long)llrint(a * b * kCovScale)};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicAdd(&cdiff[k * n1 + lo], q[k]);
            atomicAdd(&cdiff[k * n1 + hi], 0ull - q[k]);
        }
    }
    __syncthreads();
    // inclusive prefix over j: each thread scans a contiguous run, then the
    // runs' totals are scanned by thread 0
    const int run = (n1 + kTimingBlock - 1) / kTimingBlock;
    const int j0 = threadIdx.x * run, j1 = min(n1, j0 + run);
    unsigned long long sum[3] = {0ull, 0ull, 0ull};
    for (int j = j0; j < j1; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) sum[k] += cdiff[k * n1 + j];
#pragma unroll
    for (int k = 0; k < 3; ++k) tot[k][threadIdx.x] = sum[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long acc[3] = {0ull, 0ull, 0ull};
        for (int t = 0; t < kTimingBlock; ++t)
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const unsigned long long v = tot[k][t];
                tot[k][t] = acc[k];
                acc[k] += v;
            }
    }
    __syncthreads();
    unsigned long long run_sum[3] = {tot[0][threadIdx.x], tot[1][threadIdx.x], tot[2][threadIdx.x]};
    bool degenerate = false;
    for (int j = j0; j < j1 && j < n_f; ++j) {
#pragma unroll
        for (int k = 0; k < 3; ++k) run_sum[k] += cdiff[k * n1 + j];
        const long long ia = (long long)run_sum[0], ib = (long long)run_sum[1], ic = (long long)run_sum[2];
        float4 w = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ia != 0 || ib != 0) {
            const double A = (double)ia / kCovScale, B = (double)ib / kCovScale, C = (double)ic / kCovScale;
            const double D = A * B - C * C;
            if (D > 1e-300 && D > 1e-13 * A * B)
                w = make_float4((float)(2.0 * B / D), (float)(2.0 * A / D), (float)(-4.0 * C / D), 1.f);
            else
                degenerate = true;
        }
        comb_j[(size_t)sky * n_f + j] = w;
    }
    if (degenerate) atomicOr(p.err, 2);
}

__global__ void sft_timing_one_kernel(const SftState* __restrict__ st, int n_sft, double alpha,
                                      double delta, double t_ref, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_sft) return;
    const SkyFrame fr = sky_frame(alpha, delta);
    double dtau, tdot, a, b;
    timing_antenna(st[i], fr, t_ref, dtau, tdot, a, b);
    out[i] = dtau;
    out[n_sft + i] = tdot;
    out[2 * n_sft + i] = a;
    out[3 * n_sft + i] = b;
}

// ---- injection -------------------------------------------------------------
// work layout per signal: [0..5] = (h0, Re ca, Im ca, Re cb, Im cb, unused),
// then per SFT 4 doubles: (Re amp, Im amp, khat, unused) with
// amp = (T/2) h0 (a ca + b cb) e^{i Phi}.
constexpr int kInjHead = 8;

__global__ void __launch_bounds__(kTimingBlock) inject_prep_kernel(const SftState* __restrict__ st, int n_sft,
                                                                   const fstat_signal* __restrict__ sig,
                                                                   double T, double t_ref,
                                                                   double* __restrict__ work) {
    __shared__ double red[3][kTimingBlock / 32];
    __shared__ double sh_h0;
    const fstat_signal g = sig[blockIdx.x];
    double* w = work + (size_t)blockIdx.x * (kInjHead + 4 * (size_t)n_sft);
    const SkyFrame fr = sky_frame(g.alpha, g.delta);
    // unit-amplitude complex amplitudes: h = Re[(a ca + b cb) e^{i Phi}]
    const double ap = (1.0 + g.cosi * g.cosi) / 2.0, ax = g.cosi;
    double s2p, c2p, sp0, cp0;
    sincos(2.0 * g.psi, &s2p, &c2p);
    sincos(g.phi0, &sp0, &cp0);
    const double ca_re = ap * c2p * cp0 - ax * s2p * sp0, ca_im = ap * c2p * sp0 + ax * s2p * cp0;
    const double cb_re = ap * s2p * cp0 + ax * c2p * sp0, cb_im = ap * s2p * sp0 - ax * c2p * cp0;
    double sAA = 0.0, sBB = 0.0, sAB = 0.0;
    for (int i = threadIdx.x; i < n_sft; i += kTimingBlock) {
        double dtau, tdot, a, b;
        timing_antenna(st[i], fr, t_ref, dtau, tdot, a, b);
        sAA += a * a;
        sBB += b * b;
        sAB += a * b;
    }
    const double A = block_sum<kTimingBlock>(sAA, red[0]);
    const double B = block_sum<kTimingBlock>(sBB, red[1]);
    const double C = block_sum<kTimingBlock>(sAB, red[2]);
    if (threadIdx.x == 0) {
        const double q = A * (ca_re * ca_re + ca_im * ca_im) + B * (cb_re * cb_re + cb_im * cb_im) +
                         2.0 * C * (ca_re * cb_re + ca_im * cb_im);
        const double rho2_unit = T * T / 2.0 * q;
        sh_h0 = g.rho / sqrt(rho2_unit);
        w[0] = sh_h0;
        w[1] = ca_re;
        w[2] = ca_im;
        w[3] = cb_re;
        w[4] = cb_im;
    }
    __syncthreads();
    const double h0 = sh_h0;
    for (int i = threadIdx.x; i < n_sft; i += kTimingBlock) {
        double dtau, tdot, a, b;
        timing_antenna(st[i], fr, t_ref, dtau, tdot, a, b);
        // phase in cycles: f dtau + (fdot/2) dtau^2, rounded step by step (no contraction)
        const double c1 = __dmul_rn(g.f, dtau);
        const double c2 = __dmul_rn(__dmul_rn(__dmul_rn(0.5, g.fdot), dtau), dtau);
        const double cyc = __dadd_rn(c1, c2);
        const double frac = cyc - floor(cyc);
        double sph, cph;
        sincospi(2.0 * frac, &sph, &cph);
        const double khat = __dmul_rn(__dmul_rn(__dadd_rn(g.f, __dmul_rn(g.fdot, dtau)), tdot), T);
        const double sr = a * ca_re + b * cb_re, si = a * ca_im + b * cb_im;
        const double amp = 0.5 * T * h0;
        double* o = w + kInjHead + 4 * (size_t)i;
        o[0] = amp * (sr * cph - si * sph);
        o[1] = amp * (sr * sph + si * cph);
        o[2] = khat;
        o[3] = 0.0;
    }
}

__global__ void inject_add_kernel(const double* __restrict__ work, int n_sig, int n_sft,
                                  long long k_lo, int n_bins, long long row, float2* __restrict__ bins) {
    const int i = blockIdx.y;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_bins) return;
    const long long k = k_lo + j;
    float2* x = bins + (size_t)i * row + j;
    double re = (double)x->x, im = (double)x->y;
    const double sgn = (k & 1) ? -1.0 : 1.0;
    for (int s = 0; s < n_sig; ++s) {
        const double* o = work + (size_t)s * (kInjHead + 4 * (size_t)n_sft) + kInjHead + 4 * (size_t)i;
        const double xk = o[2] - (double)k;
        double sc;
        if (xk == 0.0) {
            sc = 1.0;
        } else {
            const double y = kPi * xk;
            sc = sin(y) / y;
        }
        re += o[0] * sgn * sc;
        im += o[1] * sgn * sc;
    }
    *x = make_float2((float)re, (float)im);
}

// ---- 16-bit storage ----------------------------------------------------------
template <int FORM>
__global__ void __launch_bounds__(256) quantize_kernel(const float2* __restrict__ src, long long row, int n_bins,
                                                       void* __restrict__ dst, float* __restrict__ scale) {
    __shared__ float red[8];
    const int i = blockIdx.x;
    const float2* x = src + (size_t)i * row;
    float m = 0.f;
    for (int j = threadIdx.x; j < n_bins; j += 256) m = fmaxf(m, fmaxf(fabsf(x[j].x), fabsf(x[j].y)));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
        red[0] = t;
    }
    __syncthreads();
    const float mx = red[0];
    const float s = mx > 0.f ? mx * 6.103515625e-05f : 1.0f;   // m * 2^-14
    if (threadIdx.x == 0) scale[i] = s;
    for (int j = threadIdx.x; j < (int)row; j += 256) {
        float re = 0.f, im = 0.f;
        if (j < n_bins) {
            re = __fdiv_rn(x[j].x, s);
            im = __fdiv_rn(x[j].y, s);
        }
        if (FORM == FSTAT_BINS_F16) {
            ((__half2*)dst)[(size_t)i * row + j] = __halves2half2(__float2half_rn(re), __float2half_rn(im));
        } else {
            ((__nv_bfloat162*)dst)[(size_t)i * row + j] =
                __halves2bfloat162(__float2bfloat16_rn(re), __float2bfloat16_rn(im));
        }
    }
}

}  // namespace

cudaError_t launch_sft_state(const double* t_start, const int* det_of_sft, const fstat_detector* dets,
                             int n_sft, double T, SftState* out, cudaStream_t s) {
    const int b = 128;
    sft_state_kernel<<<(n_sft + b - 1) / b, b, 0, s>>>(t_start, det_of_sft, dets[0], dets[1], dets[2], dets[3],
                                                      dets[4], dets[5], dets[6], dets[7], n_sft, T, out);
    return cudaGetLastError();
}

cudaError_t launch_timing(const TimingParams& p, cudaStream_t s) {
    timing_kernel<<<p.n_sky, kTimingBlock, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sft_timing_one(const SftState* st, int n_sft, double alpha, double delta, double t_ref,
                                  double* out4, cudaStream_t s) {
    const int b = 128;
    sft_timing_one_kernel<<<(n_sft + b - 1) / b, b, 0, s>>>(st, n_sft, alpha, delta, t_ref, out4);
    return cudaGetLastError();
}

cudaError_t launch_inject(const SftState* st, int n_sft, const fstat_signal* sig_dev, int n_sig, double T,
                          double t_ref, long long k_lo, int n_bins, long long row, float2* bins, double* work,
                          cudaStream_t s) {
    inject_prep_kernel<<<n_sig, kTimingBlock, 0, s>>>(st, n_sft, sig_dev, T, t_ref, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 grid((n_bins + 127) / 128, n_sft);
    inject_add_kernel<<<grid, 128, 0, s>>>(work, n_sig, n_sft, k_lo, n_bins, row, bins);
    return cudaGetLastError();
}

cudaError_t launch_quantize(const float2* src, long long row, int n_sft, int n_bins, int form, void* dst,
                            float* scale, cudaStream_t s) {
    if (form == FSTAT_BINS_F16)
        quantize_kernel<FSTAT_BINS_F16><<<n_sft, 256, 0, s>>>(src, row, n_bins, dst, scale);
    else
        quantize_kernel<FSTAT_BINS_BF16><<<n_sft, 256, 0, s>>>(src, row, n_bins, dst, scale);
    return cudaGetLastError();
}

size_t inject_work_doubles(int n_sig, int n_sft) { return (size_t)n_sig * (kInjHead + 4 * (size_t)n_sft); }

cudaError_t launch_coverage_comb(const TimingParams& tp, const int2* cov, int n_f, float4* comb_j, cudaStream_t s) {
    const size_t smem = 3 * (size_t)(n_f + 1) * sizeof(unsigned long long);
    cudaError_t e = cudaFuncSetAttribute(coverage_comb_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    coverage_comb_kernel<<<tp.n_sky, kTimingBlock, smem, s>>>(tp, cov, n_f, comb_j);
    return cudaGetLastError();
}

}  // namespace fs
