// Far-field polynomial form of the Dirichlet accumulation (D = 8).
//
// The SFT term of the F-statistic (Section 2, the kernel sum of Listing 1)
// sums X_k / (kappa - k) over the 16 bins k0-7 .. k0+8 around khat.  Twelve of
// them (offsets -7..-2 and 3..8) never come closer than 2 bins to kappa in
// [0, 1): their sum is smooth in kappa and is replaced by its degree-5
// interpolant c_0 + c_1 kappa + ... + c_5 kappa^5 (error below 5e-6 of each
// term), with c_n = sum_k X_{k0+k} gamma[k][n] precomputed once per SFT and
// window position.  The four bins next to the poles (offsets -1..2) keep the
// exact pair form with product-form denominators, so a template.SFT pair
// costs one polynomial (5 packed multiply-adds) and two reciprocals instead of
// eight pair terms and eight reciprocals.
//
// Tables (built by far_tables_kernel from the stored bins, FP32), split by
// the parity of the position so that a block's entries of one parity are one
// contiguous run (half = n_pos / 2, position x at [x & 1][x >> 1]):
//   ptab [n_sft][2][half]      (X_b + X_{b+1}, X_{b+1} - X_b) for bin b
//   pcoef[n_sft][2][half][3]   record (c0, c1), (c2, c3), (c4, c5) for window k0 = b
// with position x <-> bin k_lo - xoff + x; bins outside the stored band are 0.
// A record is 3 x 16 bytes: an odd number of 16-byte slots, so lanes whose
// records sit an odd number of records apart read without bank conflicts,
// and a template's three loads share one address (immediate offsets).
//
// The block works like the direct kernel (one sky point, one column of
// frequencies, a run of spindown rows; M templates per thread at stride P
// whose windows sit L bins apart).  Two stagings:
//  * far_block: every thread stages rounds of C SFTs with cp.async into a
//    double buffer, one barrier per round (any L, any spindown list);
//  * far_ring_block (L = 2, uniform spindown grid): one producer warp copies
//    each SFT's rows with TMA bulk copies into a ring of S stages guarded by
//    mbarriers (full: copies landed; empty: all compute warps done), so
//    compute warps run up to S SFTs apart and never meet at a block barrier.
// Blocks are ordered sky-fastest inside a column: the blocks resident at one
// time read the same column slice of the tables, which stays in L2.
#include <type_traits>

#include "dirichlet.cuh"

namespace fs {
namespace {

template <int FORM>
__global__ void __launch_bounds__(256) far_tables_kernel(const typename RawT<FORM>::T* __restrict__ bins,
                                                         long long row, int n_sft, int n_bins, const FarGamma gam,
                                                         float4* __restrict__ ptab, float4* __restrict__ pcoef,
                                                         int n_pos, int xoff) {
    using RT = RawT<FORM>;
    const long long total = (long long)n_sft * n_pos;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / n_pos);
        const int x = (int)(t - (long long)s * n_pos);
        const int r = x - xoff;   // bin relative to k_lo
        const typename RT::T* rp = bins + (size_t)s * row;
        auto X = [&](int i) -> float2 {
            return (i >= 0 && i < n_bins) ? RT::f2(rp[i]) : make_float2(0.f, 0.f);
        };
        const size_t o = (size_t)s * n_pos + (size_t)(x & 1) * (n_pos >> 1) + (x >> 1);   // parity-split slot
        const float2 x0 = X(r), x1 = X(r + 1);
        ptab[o] = make_float4(x0.x + x1.x, x0.y + x1.y, x1.x - x0.x, x1.y - x0.y);
        float cr[kFarDeg + 1], ci[kFarDeg + 1];
#pragma unroll
        for (int n = 0; n <= kFarDeg; ++n) cr[n] = ci[n] = 0.f;
#pragma unroll
        for (int i = 0; i < kFarTerms; ++i) {
            const float2 v = X(r + far_offset(i));
#pragma unroll
            for (int n = 0; n <= kFarDeg; ++n) {
                cr[n] = fmaf(v.x, gam.g[i][n], cr[n]);
                ci[n] = fmaf(v.y, gam.g[i][n], ci[n]);
            }
        }
        float4* cp = pcoef + o * 3;
        cp[0] = make_float4(cr[0], ci[0], cr[1], ci[1]);
        cp[1] = make_float4(cr[2], ci[2], cr[3], ci[3]);
        cp[2] = make_float4(cr[4], ci[4], cr[5], ci[5]);
    }
}

// Window sum of one template: far polynomial plus the two exact near pairs.
// pn: pair entry of offsets (-1, 0); the pair of offsets (1, 2) is STRIDE
// entries further.  cp: the template's coefficient record.  Same scaling as
// the pair form of the direct kernel: Q = (1/2) sum_k X_k / (kappa - k).
template <int STRIDE>
__device__ __forceinline__ float2 far_window_sum(const float4* __restrict__ pn, const float4* __restrict__ cp,
                                                 float kap) {
    const float4 e0 = cp[0], e1 = cp[1], e2 = cp[2];
    const float2 kk = make_float2(kap, kap);
    float2 F = make_float2(e2.z, e2.w);
    F = __ffma2_rn(F, kk, make_float2(e2.x, e2.y));
    F = __ffma2_rn(F, kk, make_float2(e1.z, e1.w));
    F = __ffma2_rn(F, kk, make_float2(e1.x, e1.y));
    F = __ffma2_rn(F, kk, make_float2(e0.z, e0.w));
    F = __ffma2_rn(F, kk, make_float2(e0.x, e0.y));
    const float4 n3 = pn[0], n4 = pn[STRIDE];
    // offsets (-1, 0): Y = 2 kappa + 1, Y^2 - 1 = 4 kappa (kappa + 1)
    const float k4 = 4.0f * kap;
    const float r3 = rcp_approx(fmaf(k4, kap, k4));
    // offsets (1, 2): Y = 2 kappa - 3, Y^2 - 1 = 4 (kappa - 1)(kappa - 2)
    const float u = kap - 1.0f, u4 = 4.0f * u;
    const float r4 = rcp_approx(fmaf(u4, u, -u4));
    const float y3 = fmaf(2.0f, kap, 1.0f), y4 = fmaf(2.0f, kap, -3.0f);
    const float2 S3 = __ffma2_rn(make_float2(y3, y3), make_float2(n3.x, n3.y), make_float2(n3.z, n3.w));
    const float2 S4 = __ffma2_rn(make_float2(y4, y4), make_float2(n4.x, n4.y), make_float2(n4.z, n4.w));
    F = __ffma2_rn(S3, make_float2(r3, r3), F);
    return __ffma2_rn(S4, make_float2(r4, r4), F);
}

// Sinc-polynomial form of one SFT for one thread's M templates: cf is the
// staged row of 48-byte records c_{0..5} (FP32) of the half bin kappa < 1/2,
// cf + plane4 that of the half kappa >= 1/2, both parity-split for L = 2.
// P already carries sin(pi kappa)/2, so the template's term is the twiddle
// times P, with no reciprocal, sine or clamp.
template <int M, int L, bool COV>
__device__ __forceinline__ void sinc_sft(const DirichletParams& p, const SkySftMeta& m, long long kh_row,
                                         unsigned int ph0, int lo_rel, const float4* __restrict__ cf, int plane4,
                                         int half, int j_t, int clo, int chi, float2 (&fa)[M], float2 (&fb)[M]) {
    constexpr int D = 8;
    const bool part = COV && (j_t < clo || j_t + (M - 1) * p.P >= chi);   // coverage holds some templates only
    // template q counts for this SFT (always, without coverage)
    auto covered = [&](int q) { return !COV || !part || (j_t + q * p.P >= clo && j_t + q * p.P < chi); };
    const long long kh = kh_row + (long long)j_t * m.dk;
    const int k0 = (int)(kh >> 32);
    const int b = (k0 - (int)p.k_lo) - (D - 1) - lo_rel;
    const float2 a2 = make_float2(m.a, m.a), b2 = make_float2(m.b, m.b);
    // u = kappa - 1/2; the half bin is u >= 0, v = u -+ 1/4 its local variable
    auto horner = [&](const float4* __restrict__ r, float v) -> float2 {
        const float4 e0 = r[0], e1 = r[1], e2 = r[2];
        const float2 vv = make_float2(v, v);
        float2 P = __ffma2_rn(make_float2(e2.z, e2.w), vv, make_float2(e2.x, e2.y));
        P = __ffma2_rn(P, vv, make_float2(e1.z, e1.w));
        P = __ffma2_rn(P, vv, make_float2(e1.x, e1.y));
        P = __ffma2_rn(P, vv, make_float2(e0.z, e0.w));
        return __ffma2_rn(P, vv, make_float2(e0.x, e0.y));
    };
    auto poly = [&](int pos, float u) -> float2 {
        const bool up = u >= 0.f;
        return horner(cf + (up ? plane4 : 0) + 3 * pos, u + (up ? -0.25f : 0.25f));
    };
    // use = false (a template outside the SFT's coverage) adds zero: a select,
    // not a branch, so partially covered threads stay on the common path
    auto add = [&](float tw_re, float tw_im, float2 P, float2& fa_q, float2& fb_q, bool use) {
        float2 z = make_float2(fmaf(tw_re, P.x, -tw_im * P.y), fmaf(tw_re, P.y, tw_im * P.x));
        if (COV) z = use ? z : make_float2(0.f, 0.f);
        fa_q = __ffma2_rn(a2, z, fa_q);
        fb_q = __ffma2_rn(b2, z, fb_q);
    };
    const bool fast = ((int)((kh + m.span) >> 32) == k0 + (M - 1) * L);
    if (fast) {
        int bb = b;
        if (bb < 0 || bb + (M - 1) * L + 2 * (D - 1) >= p.w_pairs) {
            atomicOr(p.err, 1);
            bb = max(0, min(bb, p.w_pairs - 1 - (M - 1) * L - 2 * (D - 1)));
        }
        const int pos0 = tab_pos<L>(bb + 7, half);
        const unsigned int ph = ph0 + (unsigned int)j_t * m.dphi + ((unsigned int)k0 << 31);
        float sn, cs;
        __sincosf((float)(int)ph * kPhaseToRad, &sn, &cs);
        float tw_re = cs, tw_im = -sn;
        const float u0 = frac_to_float((unsigned int)kh) - 0.5f;
        // partially covered threads (coverage edges) take a copy of the loops
        // that zeroes the uncovered templates; everyone else runs them as is
        auto loops = [&](auto masked) {
            constexpr bool MK = decltype(masked)::value;
            float tr = tw_re, ti = tw_im;
            if (fabsf(m.eps) * (float)(M - 1) <= kSincSlack) {
                // kappa drifts by at most kSincSlack over the M templates: one half
                // bin, chosen at the middle template, serves all of them (at most
                // kSincSlack / 2 outside it, where the interpolant still holds)
                const bool up = fmaf(0.5f * (float)(M - 1), m.eps, u0) >= 0.f;
                const float4* cq = cf + (up ? plane4 : 0) + 3 * pos0;
                const float v0 = u0 + (up ? -0.25f : 0.25f);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    add(tr, ti, horner(cq + 3 * q, fmaf((float)q, m.eps, v0)), fa[q], fb[q], !MK || covered(q));
                    if (q + 1 < M) {
                        const float t = fmaf(tr, m.rot_re, -ti * m.rot_im);
                        ti = fmaf(tr, m.rot_im, ti * m.rot_re);
                        tr = t;
                    }
                }
            } else {
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    add(tr, ti, poly(pos0 + q, fmaf((float)q, m.eps, u0)), fa[q], fb[q], !MK || covered(q));
                    if (q + 1 < M) {
                        const float t = fmaf(tr, m.rot_re, -ti * m.rot_im);
                        ti = fmaf(tr, m.rot_im, ti * m.rot_re);
                        tr = t;
                    }
                }
            }
        };
        if (COV && part)
            loops(std::true_type{});
        else
            loops(std::false_type{});
    } else {
        const long long pdk = (long long)p.P * m.dk;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            if (!covered(q)) continue;
            const long long khq = kh + (long long)q * pdk;
            const int k0q = (int)(khq >> 32);
            const unsigned int phq = ph0 + (unsigned int)(j_t + q * p.P) * m.dphi + ((unsigned int)k0q << 31);
            float s2, c2;
            __sincosf((float)(int)phq * kPhaseToRad, &s2, &c2);
            int bq = b + (k0q - k0);
            if (bq < 0 || bq + 2 * (D - 1) >= p.w_pairs) {
                atomicOr(p.err, 1);
                bq = max(0, min(bq, p.w_pairs - 1 - 2 * (D - 1)));
            }
            add(c2, -s2, poly(tab_pos<L>(bq + 7, half), frac_to_float((unsigned int)khq) - 0.5f), fa[q], fb[q], true);
        }
    }
}

// Sinc tables: per (SFT, position x) and half bin h, the six complex
// coefficients c_{h,n} = sum_k X_{x - xoff + k} gamma[h][k + 7][n] (bins outside
// the band count as zero), stored at [SFT][h][position], positions split by
// parity for the L = 2 layouts.
template <int FORM>
__global__ void __launch_bounds__(256) sinc_tables_kernel(const typename RawT<FORM>::T* __restrict__ bins,
                                                          long long row, int n_sft, int n_bins, const SincGamma gam,
                                                          float4* __restrict__ pcoef, int n_pos, int xoff, bool split) {
    using RT = RawT<FORM>;
    const long long total = (long long)n_sft * n_pos;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
         t += (long long)gridDim.x * blockDim.x) {
        const int s = (int)(t / n_pos);
        const int x = (int)(t - (long long)s * n_pos);
        const int r = x - xoff;
        // parity-split position (L = 2) or plain (L = 1)
        const size_t slot = split ? (size_t)(x & 1) * (n_pos >> 1) + (x >> 1) : (size_t)x;
        const typename RT::T* rp = bins + (size_t)s * row;
        float2 v[kSincTerms];
#pragma unroll
        for (int i = 0; i < kSincTerms; ++i) {
            const int j = r + i - 7;
            v[i] = (j >= 0 && j < n_bins) ? RT::f2(rp[j]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float cr[kSincDeg + 1], ci[kSincDeg + 1];
#pragma unroll
            for (int n = 0; n <= kSincDeg; ++n) cr[n] = ci[n] = 0.f;
#pragma unroll
            for (int i = 0; i < kSincTerms; ++i)
#pragma unroll
                for (int n = 0; n <= kSincDeg; ++n) {
                    cr[n] = fmaf(v[i].x, gam.g[h][i][n], cr[n]);
                    ci[n] = fmaf(v[i].y, gam.g[h][i][n], ci[n]);
                }
            float4* cp = pcoef + 3 * (((size_t)s * 2 + h) * n_pos + slot);
#pragma unroll
            for (int e = 0; e < 3; ++e) cp[e] = make_float4(cr[2 * e], ci[2 * e], cr[2 * e + 1], ci[2 * e + 1]);
        }
    }
}

// One SFT of one thread's M templates: kh_row / ph0 are the fixed-point bin
// and phase bases of the thread's spindown row, lo_rel the bin of the staged
// rows' entry 0 relative to k_lo, tab / cf the staged pair and coefficient
// rows (parity-split for L = 2).
template <int M, int L, bool COV>
__device__ __forceinline__ void far_sft(const DirichletParams& p, const SkySftMeta& m, long long kh_row,
                                        unsigned int ph0, int lo_rel, const float4* __restrict__ tab,
                                        const float4* __restrict__ cf, int half, int j_t, int clo, int chi,
                                        float2 (&fa)[M], float2 (&fb)[M]) {
    constexpr int D = 8;
    constexpr int STRIDE = (L == 2) ? 1 : 2;
    const bool part = COV && (j_t < clo || j_t + (M - 1) * p.P >= chi);   // coverage holds some templates only
    // template q counts for this SFT (always, without coverage)
    auto covered = [&](int q) { return !COV || !part || (j_t + q * p.P >= clo && j_t + q * p.P < chi); };
    const long long kh = kh_row + (long long)j_t * m.dk;
    const int k0 = (int)(kh >> 32);
    const int b = (k0 - (int)p.k_lo) - (D - 1) - lo_rel;   // first pair of template 0
    const float2 a2 = make_float2(m.a, m.a), b2 = make_float2(m.b, m.b);
    const bool fast = ((int)((kh + m.span) >> 32) == k0 + (M - 1) * L);
    if (fast) {
        int bb = b;
        if (bb < 0 || bb + (M - 1) * L + 2 * (D - 1) >= p.w_pairs) {
            atomicOr(p.err, 1);   // outside the staged rows (clamped); rare, no register kept for it
            bb = max(0, min(bb, p.w_pairs - 1 - (M - 1) * L - 2 * (D - 1)));
        }
        const float4* pn = tab + tab_pos<L>(bb, half) + 3 * STRIDE;
        const float4* cp = cf + 3 * tab_pos<L>(bb + 7, half);
        const unsigned int ph = ph0 + (unsigned int)j_t * m.dphi + ((unsigned int)k0 << 31);
        float sn, cs;
        __sincosf((float)(int)ph * kPhaseToRad, &sn, &cs);
        float tw_re = cs, tw_im = -sn;
        const float kap0 = clamp_kappa(frac_to_float((unsigned int)kh));
#pragma unroll
        for (int q = 0; q < M; ++q) {
            const float kap = clamp_kappa(fmaf((float)q, m.eps, kap0));
            const float2 Q = far_window_sum<STRIDE>(pn + q, cp + 3 * q, kap);
            if (covered(q)) accumulate(tw_re, tw_im, sinpi_unit(kap), Q, a2, b2, fa[q], fb[q]);
            if (q + 1 < M) {
                const float t = fmaf(tw_re, m.rot_re, -tw_im * m.rot_im);
                tw_im = fmaf(tw_re, m.rot_im, tw_im * m.rot_re);
                tw_re = t;
            }
        }
    } else {
        const long long pdk = (long long)p.P * m.dk;
#pragma unroll
        for (int q = 0; q < M; ++q) {
            if (!covered(q)) continue;
            const long long khq = kh + (long long)q * pdk;
            const int k0q = (int)(khq >> 32);
            const float kap = clamp_kappa(frac_to_float((unsigned int)khq));
            const unsigned int phq = ph0 + (unsigned int)(j_t + q * p.P) * m.dphi + ((unsigned int)k0q << 31);
            float s2, c2;
            __sincosf((float)(int)phq * kPhaseToRad, &s2, &c2);
            int bq = b + (k0q - k0);
            if (bq < 0 || bq + 2 * (D - 1) >= p.w_pairs) {
                atomicOr(p.err, 1);
                bq = max(0, min(bq, p.w_pairs - 1 - 2 * (D - 1)));
            }
            const float2 Q = far_window_sum<STRIDE>(tab + tab_pos<L>(bq, half) + 3 * STRIDE,
                                                    cf + 3 * tab_pos<L>(bq + 7, half), kap);
            accumulate(c2, -s2, sinpi_unit(kap), Q, a2, b2, fa[q], fb[q]);
        }
    }
}

// 2F of a thread's M templates (fused combine, written once per template).
template <int M>
__device__ __forceinline__ void far_store(const DirichletParams& p, int sky, int drow, int j_t, int j_end,
                                          const float2 (&fa)[M], const float2 (&fb)[M]) {
    const float4 cm = p.comb[sky];
    float* out = p.twoF + ((size_t)sky * p.n_fdot + drow) * p.n_f;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const int j = j_t + q * p.P;
        if (j < j_end) {
            const float4 cw = p.comb_j ? p.comb_j[(size_t)sky * p.n_f + j] : cm;
            const float2 A_ = fa[q], B_ = fb[q];
            const float v = cw.x * fmaf(A_.x, A_.x, A_.y * A_.y) + cw.y * fmaf(B_.x, B_.x, B_.y * B_.y) +
                            cw.z * fmaf(A_.x, B_.x, A_.y * B_.y);
            out[j] = fmaxf(v, 0.0f);
        }
    }
}

template <int M, int L>
__device__ __forceinline__ void far_block(const DirichletParams& p, long long bid, unsigned char* smem) {
    constexpr int D = 8;
    const int NT = blockDim.x;
    const int C = p.sft_chunk;
    const PolySmem lay = farpoly_smem(C, p.w_tab, p.n_fdot);
    float4* s_pair = reinterpret_cast<float4*>(smem + lay.pairs);           // [2][C][w_tab]
    float4* s_coef = reinterpret_cast<float4*>(smem + lay.coef);            // [2][C][w_tab][3]
    SkySftMeta* s_meta = reinterpret_cast<SkySftMeta*>(smem + lay.meta);    // [3][C]
    SkySftBase* s_base = reinterpret_cast<SkySftBase*>(smem + lay.base);    // [3][C]
    long long* s_kh0 = reinterpret_cast<long long*>(smem + lay.kh0);        // [3][C][n_fdot]
    unsigned int* s_ph0 = reinterpret_cast<unsigned int*>(smem + lay.ph0);  // [3][C][n_fdot]

    const int chunk = (int)(bid % p.chunks_per_col);
    bid /= p.chunks_per_col;
    const int sky = (int)(bid % p.n_sky);
    const int col = (int)(bid / p.n_sky);
    const int PM = p.P * M;
    const int col_w = p.lg_row * PM;
    const int j_col0 = col * col_w;
    const int width = min(col_w, p.n_f - j_col0);
    const int Gc = (width + PM - 1) / PM;
    const int LG = p.n_fdot * Gc;
    const int u0 = chunk * p.lg_cta;
    if (u0 >= LG) return;
    const int u_end = min(u0 + p.lg_cta, LG);
    const int d_lo = u0 / Gc;
    const int d_hi = (u_end - 1) / Gc;
    const int n_rows = d_hi - d_lo + 1;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp % p.P;
    const int ul = (warp / p.P) * 32 + lane;
    const int u = u0 + ul;
    const bool active = (ul < p.lg_cta) && (u < u_end);
    const int uu = active ? u : u0;
    const int drow = uu / Gc;
    const int g = uu - drow * Gc;
    const int j_t = j_col0 + g * PM + r;
    const int row_i = drow - d_lo;
    const bool warp_live = __any_sync(0xffffffffu, active);
    const int half = p.w_tab >> 1;

    const size_t meta0 = (size_t)sky * p.n_sft;
    const size_t base0 = (size_t)sky * p.n_fdot * p.n_sft;
    const int n_rounds = (p.n_sft + C - 1) / C;

    auto issue_consts = [&](int rd) {
        const int a0 = rd * C, slot = rd % 3;
        const int nc = min(C, p.n_sft - a0);
        const char* msrc = reinterpret_cast<const char*>(p.meta + meta0 + a0);
        char* mdst = reinterpret_cast<char*>(s_meta + slot * C);
        for (int t = threadIdx.x; t < nc * 3; t += NT) cp_async16(mdst + 16 * t, msrc + 16 * t, 16);
        if (p.base) {
            const char* bsrc = reinterpret_cast<const char*>(p.base + meta0 + a0);
            char* bdst = reinterpret_cast<char*>(s_base + slot * C);
            for (int t = threadIdx.x; t < nc * 2; t += NT) cp_async16(bdst + 16 * t, bsrc + 16 * t, 16);
            return;
        }
        for (int t = threadIdx.x; t < nc * n_rows; t += NT) {
            const int c = t / n_rows, rr = t - c * n_rows;
            const size_t o = base0 + (size_t)(d_lo + rr) * p.n_sft + a0 + c;
            cp_async8(s_kh0 + (slot * C + c) * p.n_fdot + rr, p.kh0 + o);
            cp_async4(s_ph0 + (slot * C + c) * p.n_fdot + rr, p.ph0 + o);
        }
    };
    // table index 0 of an SFT row <-> bin k_lo + lo_of(m)
    auto lo_of = [&](const SkySftMeta& m) -> int {
        const long long kb = m.khmin + (long long)j_col0 * m.dk;
        return (int)((kb >> 32) - p.k_lo) - (D - 1);
    };
    auto issue_tabs = [&](int rd) {
        const int a0 = rd * C, slot = rd & 1, cslot = rd % 3;
        const int nc = min(C, p.n_sft - a0);
        for (int c = 0; c < nc; ++c) {
            const int x0 = lo_of(s_meta[cslot * C + c]) + p.xoff;
            const size_t row0 = (size_t)(a0 + c) * p.n_pos;
            const int nh = p.n_pos >> 1;
            float4* dpair = s_pair + ((size_t)slot * C + c) * p.w_tab;
            float4* dcoef = s_coef + ((size_t)slot * C + c) * 3 * p.w_tab;
            for (int i = threadIdx.x; i < p.w_pairs; i += NT) {
                const int x = x0 + i;
                const bool in = (x >= 0) && (x < p.n_pos);
                const size_t o = row0 + (in ? (size_t)(x & 1) * nh + (x >> 1) : 0);
                const int nb = in ? 16 : 0;
                const int tp = tab_pos<L>(i, half);
                cp_async16(dpair + tp, p.ptab + o, nb);
#pragma unroll
                for (int k = 0; k < 3; ++k) cp_async16(dcoef + 3 * tp + k, p.pcoef + 3 * o + k, nb);
            }
        }
    };

    float2 fa[M], fb[M];
#pragma unroll
    for (int q = 0; q < M; ++q) fa[q] = fb[q] = make_float2(0.f, 0.f);

    // prologue: constants of rounds 0 and 1, tables of round 0
    issue_consts(0);
    if (n_rounds > 1) issue_consts(1);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    issue_tabs(0);
    cp_async_commit();

    for (int rd = 0; rd < n_rounds; ++rd) {
        const int a0 = rd * C;
        const int nc = min(C, p.n_sft - a0);
        const int cslot = rd % 3, slot = rd & 1;
        cp_async_wait_all();
        __syncthreads();   // tables(rd), consts(rd+1) visible; everyone done with round rd-1
        if (rd + 1 < n_rounds) issue_tabs(rd + 1);
        if (rd + 2 < n_rounds) issue_consts(rd + 2);
        cp_async_commit();

        for (int c = 0; c < (warp_live ? nc : 0); ++c) {
            const SkySftMeta m = s_meta[cslot * C + c];
            long long kh_row;
            unsigned int ph0;
            if (p.base) {
                const SkySftBase bs = s_base[cslot * C + c];
                kh_row = bs.kh0 + (long long)drow * bs.dkh;
                ph0 = bs.ph0 + (unsigned int)drow * bs.dph;
            } else {
                kh_row = s_kh0[(cslot * C + c) * p.n_fdot + row_i];
                ph0 = s_ph0[(cslot * C + c) * p.n_fdot + row_i];
            }
            far_sft<M, L, false>(p, m, kh_row, ph0, lo_of(m), s_pair + ((size_t)slot * C + c) * p.w_tab,
                          s_coef + ((size_t)slot * C + c) * 3 * p.w_tab, half, j_t, 0, 0x7fffffff, fa, fb);
        }
    }
    if (active) far_store<M>(p, sky, drow, j_t, j_col0 + width, fa, fb);
}

template <int M, int L>
__global__ void __launch_bounds__(kMaxThreads, 2) dirichlet_far_kernel(const DirichletParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    far_block<M, L>(p, (long long)blockIdx.x, smem);
}


// ---- TMA ring form ------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_inval(uint32_t bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        " .reg .pred p;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of
// 16) that signals its bytes on the mbarrier at `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for the phase of parity `parity` of an mbarrier; gives up (false)
// after about two seconds or 2^30 polls, whichever comes first.  SLEEP_NS > 0
// backs off between polls (for a waiter that is ahead and must not take issue
// slots from the compute warps).
template <unsigned SLEEP_NS = 0>
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (unsigned int it = 1; it < (1u << 30); ++it) {
        if (SLEEP_NS) __nanosleep(SLEEP_NS);
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 0 && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// The ring's producer warp: fetches the window bases of 32 SFTs at a time
// (one per lane, so the loads overlap); lane 0 then waits for each SFT's
// stage to be free, writes its window base and coverage, and copies its
// constants and table rows into the stage with bulk copies under the stage's
// full barrier.  Returns (lane 0) the number of stages issued.
// SR > 1: the block holds n_in <= SR consecutive sky points starting at sky
// meta0 (meta and bases SFT-major, one copy of each for all of them); the
// window base is the lowest of theirs.
template <bool SINC, bool COV, int L, int SR = 1>
__device__ __forceinline__ int ring_produce(const DirichletParams& p, const RingSmem& lay, int S, unsigned char* smem,
                                            uint32_t sb, volatile int* ctrl, size_t meta0, int j_col0, int lane,
                                            int n_in = 1) {
    constexpr int D = 8;
    auto full_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s); };
    auto empty_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s + 8); };
    // the warp fetches the window bases of 32 SFTs at a time (one per lane,
    // so the loads overlap); lane 0 then waits, stages and copies each SFT
    const int nh = p.n_pos >> 1;
    const int half = p.w_tab >> 1;
    const int n0 = (p.w_pairs + 1) >> 1, n1 = p.w_pairs >> 1;
    // per position 16 + 48 bytes (far field) or 2 x 48 bytes (sinc)
    const uint32_t bytes = 80u * (uint32_t)n_in + (uint32_t)(n0 + n1) * (SINC ? 96u : 64u);
    int a = 0;
    bool stop = false;
    int pslot = 0;            // slot of SFT a
    uint32_t pparity = 0;     // parity of the empty phase the next reuse of pslot waits for
    const int n_issue = p.ring_stop >= 0 ? min(p.ring_stop, p.n_sft) : p.n_sft;
    for (int a0 = 0; a0 < n_issue && !stop; a0 += 32) {
        int x_lane = 0;
        int2 cv_lane = make_int2(0, 0x7fffffff);
        if (COV && a0 + lane < p.n_sft) cv_lane = p.cov[a0 + lane];
        if (a0 + lane < p.n_sft) {
            if (SR == 1) {
                const SkySftMeta* gm = p.meta + meta0 + a0 + lane;
                x_lane = (int)(((gm->khmin + (long long)j_col0 * gm->dk) >> 32) - p.k_lo) - (D - 1) + p.xoff;
            } else {
                const SkySftMeta* gm = p.meta + (size_t)(a0 + lane) * p.n_sky + meta0;
                long long kmin = gm->khmin + (long long)j_col0 * gm->dk;
                for (int q = 1; q < n_in; ++q) kmin = min(kmin, gm[q].khmin + (long long)j_col0 * gm[q].dk);
                x_lane = (int)((kmin >> 32) - p.k_lo) - (D - 1) + p.xoff;
            }
        }
        const int n_here = min(32, n_issue - a0);
        for (int j = 0; j < n_here; ++j) {
            int x0 = __shfl_sync(0xffffffffu, x_lane, j);
            const int clo = __shfl_sync(0xffffffffu, cv_lane.x, j);
            const int chi = __shfl_sync(0xffffffffu, cv_lane.y, j);
            if (lane == 0) {
                a = a0 + j;
                if (a >= S && !mbar_wait<128>(empty_bar(pslot), pparity)) {
                    ctrl[1] = 1;
                    atomicOr(p.err, 4);
                    stop = true;
                } else if (ctrl[1]) {
                    stop = true;
                } else {
                    if (x0 < 0 || x0 + p.w_pairs > p.n_pos) {   // outside the padded tables: clamp, flag
                        atomicOr(p.err, 1);
                        x0 = max(0, min(x0, p.n_pos - p.w_pairs));
                    }
                    unsigned char* st = smem + (size_t)pslot * lay.stage;
                    *reinterpret_cast<int4*>(st + lay.lo) = make_int4(x0 - p.xoff, 0, clo, chi);
                    const uint32_t ss = sb + (uint32_t)((size_t)pslot * lay.stage);
                    const uint32_t fb = full_bar(pslot);
                    mbar_expect_tx(fb, bytes);
                    if (SR == 1) {
                        bulk_g2s(ss + (uint32_t)lay.meta, p.meta + meta0 + a, 48, fb);
                        bulk_g2s(ss + (uint32_t)lay.base, p.base + meta0 + a, 32, fb);
                    } else {
                        bulk_g2s(ss + (uint32_t)lay.meta, p.meta + (size_t)a * p.n_sky + meta0, 48u * n_in, fb);
                        bulk_g2s(ss + (uint32_t)lay.base, p.base + (size_t)a * p.n_sky + meta0, 32u * n_in, fb);
                    }
                    if (L == 1) {   // plain tables: one run of w_pairs positions per plane
#pragma unroll
                        for (int hb = 0; hb < 2; ++hb)
                            bulk_g2s(ss + (uint32_t)(hb * lay.plane),
                                     p.pcoef + 3 * (((size_t)a * 2 + hb) * p.n_pos + x0),
                                     (uint32_t)p.w_pairs * 48u, fb);
                    }
#pragma unroll
                    for (int h = 0; h < (L == 2 ? 2 : 0); ++h) {
                        const int cnt = h ? n1 : n0;
                        const size_t go = (size_t)a * p.n_pos + (size_t)((x0 + h) & 1) * nh + ((x0 + h) >> 1);
                        if (SINC) {
                            const size_t gx = go - (size_t)a * p.n_pos;   // position within the SFT's row
#pragma unroll
                            for (int hb = 0; hb < 2; ++hb)
                                bulk_g2s(ss + (uint32_t)(hb * lay.plane + (size_t)h * half * 48),
                                         p.pcoef + 3 * (((size_t)a * 2 + hb) * p.n_pos + gx),
                                         (uint32_t)cnt * 48u, fb);
                        } else {
                            bulk_g2s(ss + (uint32_t)(lay.pairs + (size_t)h * half * 16), p.ptab + go,
                                     (uint32_t)cnt * 16u, fb);
                            bulk_g2s(ss + (uint32_t)(lay.coef + (size_t)h * half * 48), p.pcoef + 3 * go,
                                     (uint32_t)cnt * 48u, fb);
                        }
                    }
                    ++a;
                    if (++pslot == S) {   // the next use of slot 0 waits for the phase after this one
                        pslot = 0;
                        if (a > S) pparity ^= 1u;
                    }
                }
            }
            stop = __shfl_sync(0xffffffffu, stop, 0);
            if (stop) break;
        }
    }
    return a;
}

// Uniform spindown grid; L = 2 (tables split by position parity, two runs
// per table and SFT) or L = 1 (sinc form only: plain tables, one run).
// Warps 0..NW-1 compute, warp NW produces.
// SR > 1: a block holds SR consecutive sky points (the last block of a column
// fewer); its rows are (sky point, spindown), sky-major, and its window
// covers all of them (close sky points: their windows differ by a few bins).
// Error flag bit 2: a pipeline wait gave up (results of the block invalid).
template <int M, bool SINC, bool COV, int L, int SR = 1>
__device__ __forceinline__ void far_ring_block(const DirichletParams& p, long long bid, unsigned char* smem) {
    static_assert(L == 2 || (L == 1 && SINC), "the L = 1 ring is built for the sinc tables");
    static_assert(SR == 1 || !COV, "blocks of several sky points have no coverage path");
    constexpr int D = 8;
    const int S = p.sft_chunk;
    const RingSmem lay = ring_smem(S, p.w_tab, SINC, SR);
    const int NW = (int)(blockDim.x >> 5) - 1;

    const int chunk = (int)(bid % p.chunks_per_col);
    bid /= p.chunks_per_col;
    const int n_grp = SR == 1 ? p.n_sky : (p.n_sky + SR - 1) / SR;
    const int sky0 = (int)(bid % n_grp) * SR;
    const int col = (int)(bid / n_grp);
    const int n_in = SR == 1 ? 1 : min(SR, p.n_sky - sky0);
    const int PM = p.P * M;
    const int col_w = p.lg_row * PM;
    const int j_col0 = col * col_w;
    const int width = min(col_w, p.n_f - j_col0);
    const int Gc = (width + PM - 1) / PM;
    const int LG = n_in * p.n_fdot * Gc;
    const int u0 = chunk * p.lg_cta;
    if (u0 >= LG) return;   // block-uniform, before any barrier exists
    const int u_end = min(u0 + p.lg_cta, LG);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = (warp == NW);
    const int r = producer ? 0 : warp % p.P;
    const int ul = producer ? p.lg_cta : (warp / p.P) * 32 + lane;
    const int u = u0 + ul;
    const bool active = !producer && (ul < p.lg_cta) && (u < u_end);
    const int uu = active ? u : u0;
    const int row = uu / Gc;
    const int g = uu - row * Gc;
    const int sky_l = SR == 1 ? 0 : row / p.n_fdot;   // sky point of the block
    const int drow = SR == 1 ? row : row - sky_l * p.n_fdot;
    // SR > 1: the block's places in the grouping order, the sky point at each
    const int sky = SR == 1 || !p.sky_perm ? sky0 + sky_l : p.sky_perm[sky0 + sky_l];
    const int j_t = j_col0 + g * PM + r;
    const bool warp_live = __any_sync(0xffffffffu, active);

    const uint32_t sb = smem_u32(smem);
    volatile int* ctrl = reinterpret_cast<volatile int*>(smem + lay.ctrl);   // [0] issued, [1] abort
    auto full_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s); };
    auto empty_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s + 8); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), (uint32_t)NW);
        }
        ctrl[0] = 0;
        ctrl[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const size_t meta0 = SR == 1 ? (size_t)sky0 * p.n_sft : (size_t)sky0;
    if (producer) {
        const int issued = ring_produce<SINC, COV, L, SR>(p, lay, S, smem, sb, ctrl, meta0, j_col0, lane, n_in);
        if (lane == 0) ctrl[0] = issued;   // stages issued
    } else {
        float2 fa[M], fb[M];
#pragma unroll
        for (int q = 0; q < M; ++q) fa[q] = fb[q] = make_float2(0.f, 0.f);
        const int half = p.w_tab >> 1;
        // ring position kept incrementally (slot and phase parity); the stage's
        // data and barrier addresses follow from the slot
        int slot = 0;
        uint32_t parity = 0;
        for (int a = 0; a < p.n_sft; ++a) {
            const unsigned char* st = smem + (size_t)slot * lay.stage;
            if (!mbar_wait(full_bar(slot), parity)) {
                ctrl[1] = 1;
                atomicOr(p.err, 4);
                break;
            }
            if (warp_live) {
                // window base; with coverage, the SFT's frequency-index range
                const int4 lo4 = COV ? *reinterpret_cast<const int4*>(st + lay.lo)
                                     : make_int4(*reinterpret_cast<const int*>(st + lay.lo), 0, 0, 0x7fffffff);
                // skip an SFT whose coverage holds none of the thread's templates
                if (!COV || (j_t + (M - 1) * p.P >= lo4.z && j_t < lo4.w)) {
                    const SkySftMeta m = *reinterpret_cast<const SkySftMeta*>(st + lay.meta + 48 * sky_l);
                    const SkySftBase bs = *reinterpret_cast<const SkySftBase*>(st + lay.base + 32 * sky_l);
                    if (SINC)
                        sinc_sft<M, L, COV>(p, m, bs.kh0 + (long long)drow * bs.dkh,
                                            bs.ph0 + (unsigned int)drow * bs.dph, lo4.x,
                                            reinterpret_cast<const float4*>(st + lay.coef), (int)(lay.plane >> 4),
                                            half, j_t, lo4.z, lo4.w, fa, fb);
                    else
                        far_sft<M, L, COV>(p, m, bs.kh0 + (long long)drow * bs.dkh,
                                           bs.ph0 + (unsigned int)drow * bs.dph, lo4.x,
                                           reinterpret_cast<const float4*>(st + lay.pairs),
                                           reinterpret_cast<const float4*>(st + lay.coef), half, j_t, lo4.z, lo4.w, fa,
                                           fb);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_bar(slot));
            if (ctrl[1]) break;
            if (++slot == S) {
                slot = 0;
                parity ^= 1u;
            }
        }
        if (active) far_store<M>(p, sky, drow, j_t, j_col0 + width, fa, fb);
    }
    // after a give-up, wait for the copies still in flight into this block's
    // shared memory (each slot's latest phase) before the block retires; then
    // invalidate the barriers so that a persistent block can set them up again
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ctrl[1]) {
            const int issued = ctrl[0];
            for (int a = max(0, issued - S); a < issued; ++a) mbar_wait(full_bar(a % S), (uint32_t)((a / S) & 1));
        }
        for (int s = 0; s < S; ++s) {
            mbar_inval(full_bar(s));
            mbar_inval(empty_bar(s));
        }
    }
}

// NWC compute warps plus the producer; two resident blocks per SM; SR sky
// points per block.
template <int M, int NWC, bool SINC, bool COV, int L, int SR = 1>
__global__ void __launch_bounds__(32 * (NWC + 1), 2) dirichlet_far_ring_kernel(const DirichletParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    far_ring_block<M, SINC, COV, L, SR>(p, (long long)blockIdx.x, smem);
}

// Rows form of the sinc polynomial (uniform spindown grid, plain tables).
// A lane owns one frequency j and R consecutive spindown rows d0 .. d0+R-1;
// a warp owns 32 consecutive frequencies, so its lanes' windows sit about one
// bin apart (consecutive records, conflict-free) and their kappa agree to
// within 32 x |tdot - 1| of a bin: the record changes on the same rows for
// the whole warp.  Going from row d to d + 1 moves khat by dkh = dfdot dtau
// tdot T (0 to 0.6 bins on the workunit); a row whose window base and half
// bin are those of the row before reuses the record held in registers, so
// each 48-byte record is read once for every run of rows that shares it
// instead of once per template.  The twiddle steps between rows by the
// bases' rot = e^{-2 pi i dph}, flipping sign with the parity of k0.
template <int R>
__device__ __forceinline__ void rows_sft(const DirichletParams& p, const SkySftMeta& m, const SkySftBase& bs,
                                         int d0, int j, int lo_rel, const float4* __restrict__ cf, int plane4,
                                         float2 (&fa)[R], float2 (&fb)[R]) {
    long long kh = bs.kh0 + (long long)d0 * bs.dkh + (long long)j * m.dk;
    const unsigned int ph = bs.ph0 + (unsigned int)d0 * bs.dph + (unsigned int)j * m.dphi;
    // key = 2 k0 + half (32 bits hold it: |k0| < 2^30): the record a row reads
    int key = (int)(kh >> 31);
    float sn, cs;
    __sincosf((float)(int)(ph + ((unsigned int)(key >> 1) << 31)) * kPhaseToRad, &sn, &cs);
    float tr = cs, ti = -sn;
    const float2 a2 = make_float2(m.a, m.a), b2 = make_float2(m.b, m.b);
    // stage position of the record of window k0: k0 - k_lo - lo_rel
    const int pos_base = -(int)p.k_lo - lo_rel;
    float4 e0, e1, e2;
    float centre;   // kappa at the centre of the half bin, in units of 2^32 bins (v = kappa - centre)
    auto load = [&](int k) {
        int pos = (k >> 1) + pos_base;
        if (pos < 0 || pos >= p.w_pairs) {   // outside the staged rows (clamped); cannot happen with the planner's bound
            atomicOr(p.err, 1);
            pos = max(0, min(pos, p.w_pairs - 1));
        }
        const float4* r = cf + ((k & 1) ? plane4 : 0) + 3 * pos;
        e0 = r[0];
        e1 = r[1];
        e2 = r[2];
        centre = (k & 1) ? 3221225472.0f : 1073741824.0f;   // 3/4 and 1/4 of 2^32
    };
    load(key);
#pragma unroll
    for (int d = 0; d < R; ++d) {
        if (d > 0) {
            kh += bs.dkh;
            const float t = fmaf(tr, bs.rot_re, -ti * bs.rot_im);
            ti = fmaf(tr, bs.rot_im, ti * bs.rot_re);
            tr = t;
            const int kd = (int)(kh >> 31);
            if (kd != key) {
                if ((kd ^ key) & 2) {   // k0 changed parity: (-1)^k0 flips
                    tr = -tr;
                    ti = -ti;
                }
                key = kd;
                load(key);
            }
        }
        // v: kappa relative to the centre of its half bin
        const float v = ((float)(unsigned int)kh - centre) * 2.3283064365386963e-10f;
        const float2 vv = make_float2(v, v);
        float2 P = __ffma2_rn(make_float2(e2.z, e2.w), vv, make_float2(e2.x, e2.y));
        P = __ffma2_rn(P, vv, make_float2(e1.z, e1.w));
        P = __ffma2_rn(P, vv, make_float2(e1.x, e1.y));
        P = __ffma2_rn(P, vv, make_float2(e0.z, e0.w));
        P = __ffma2_rn(P, vv, make_float2(e0.x, e0.y));
        const float2 z = make_float2(fmaf(tr, P.x, -ti * P.y), fmaf(tr, P.y, ti * P.x));
        fa[d] = __ffma2_rn(a2, z, fa[d]);
        fb[d] = __ffma2_rn(b2, z, fb[d]);
    }
}

// A block: one sky point, NWC warps x 32 consecutive frequencies (F = 32 NWC,
// p.lg_row = F), R spindown rows (p.chunks_per_col row chunks), plus the ring's
// producer warp; the stages hold plain sinc tables (two planes).
template <int R, int NWC>
__device__ __forceinline__ void rows_ring_block(const DirichletParams& p, long long bid, unsigned char* smem) {
    const int S = p.sft_chunk;
    const RingSmem lay = ring_smem(S, p.w_tab, true);
    const int rc = (int)(bid % p.chunks_per_col);
    bid /= p.chunks_per_col;
    const int sky = (int)(bid % p.n_sky);
    const int col = (int)(bid / p.n_sky);
    const int j_col0 = col * 32 * NWC;
    const int d0 = rc * R;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = (warp == NWC);
    const int j = j_col0 + warp * 32 + lane;
    const bool active = !producer && j < p.n_f;
    const bool warp_live = __any_sync(0xffffffffu, active);

    const uint32_t sb = smem_u32(smem);
    volatile int* ctrl = reinterpret_cast<volatile int*>(smem + lay.ctrl);   // [0] issued, [1] abort
    auto full_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s); };
    auto empty_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s + 8); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), (uint32_t)NWC);
        }
        ctrl[0] = 0;
        ctrl[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();

    const size_t meta0 = (size_t)sky * p.n_sft;
    if (producer) {
        const int issued = ring_produce<true, false, 1>(p, lay, S, smem, sb, ctrl, meta0, j_col0, lane);
        if (lane == 0) ctrl[0] = issued;
    } else {
        float2 fa[R], fb[R];
#pragma unroll
        for (int q = 0; q < R; ++q) fa[q] = fb[q] = make_float2(0.f, 0.f);
        const int jj = active ? j : j_col0;   // idle lanes follow a valid frequency
        int slot = 0;
        uint32_t parity = 0;
        for (int a = 0; a < p.n_sft; ++a) {
            const unsigned char* st = smem + (size_t)slot * lay.stage;
            if (!mbar_wait(full_bar(slot), parity)) {
                ctrl[1] = 1;
                atomicOr(p.err, 4);
                break;
            }
            if (warp_live) {
                const int lo_rel = *reinterpret_cast<const int*>(st + lay.lo);
                const SkySftMeta m = *reinterpret_cast<const SkySftMeta*>(st + lay.meta);
                const SkySftBase bs = *reinterpret_cast<const SkySftBase*>(st + lay.base);
                rows_sft<R>(p, m, bs, d0, jj, lo_rel, reinterpret_cast<const float4*>(st + lay.coef),
                            (int)(lay.plane >> 4), fa, fb);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_bar(slot));
            if (ctrl[1]) break;
            if (++slot == S) {
                slot = 0;
                parity ^= 1u;
            }
        }
        if (active) {
            const float4 cm = p.comb[sky];
#pragma unroll
            for (int d = 0; d < R; ++d) {
                if (d0 + d < p.n_fdot) {
                    const float2 A_ = fa[d], B_ = fb[d];
                    const float v = cm.x * fmaf(A_.x, A_.x, A_.y * A_.y) + cm.y * fmaf(B_.x, B_.x, B_.y * B_.y) +
                                    cm.z * fmaf(A_.x, B_.x, A_.y * B_.y);
                    p.twoF[((size_t)sky * p.n_fdot + d0 + d) * p.n_f + j] = fmaxf(v, 0.0f);
                }
            }
        }
    }
    // after a give-up, wait for the copies still in flight (bounded), then
    // invalidate the barriers
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ctrl[1]) {
            const int issued = ctrl[0];
            for (int a = max(0, issued - S); a < issued; ++a) mbar_wait(full_bar(a % S), (uint32_t)((a / S) & 1));
        }
        for (int s = 0; s < S; ++s) {
            mbar_inval(full_bar(s));
            mbar_inval(empty_bar(s));
        }
    }
}

template <int R, int NWC>
__global__ void __launch_bounds__(32 * (NWC + 1)) dirichlet_rows_kernel(const DirichletParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    rows_ring_block<R, NWC>(p, (long long)blockIdx.x, smem);
}

// Two-row tiles of the sinc form (L = 2, uniform spindown grid): a thread
// owns the templates j_t + P q (q < M) of two adjacent spindown rows A and B.
// Per SFT the constants, the twiddle's sine and cosine and the checks are
// paid once for 2 M templates, and when the rows' windows start at the same
// bin and take the same half (the rows differ by dkh = dfdot dtau tdot T in
// khat), each record serves both rows; otherwise each row reads its own.
// Row B's twiddle is row A's times rot = e^{-2 pi i dph}, with the sign of
// (-1)^k0 when the windows' parity differs.  Threads whose windows straddle
// a bin boundary, or whose kappa drifts more than kSincSlack over their
// templates, run the one-row code for each row.
template <int M>
__device__ __forceinline__ void sinc_sft2(const DirichletParams& p, const SkySftMeta& m, const SkySftBase& bs,
                                          long long kh_row, unsigned int ph0, int lo_rel,
                                          const float4* __restrict__ cf, int plane4, int half, int j_t,
                                          float2 (&fa)[2][M], float2 (&fb)[2][M]) {
    constexpr int D = 8, L = 2;
    const long long khA = kh_row + (long long)j_t * m.dk;
    const long long khB = khA + bs.dkh;
    const int k0A = (int)(khA >> 32), k0B = (int)(khB >> 32);
    const bool fast = ((int)((khA + m.span) >> 32) == k0A + (M - 1) * L) &&
                      ((int)((khB + m.span) >> 32) == k0B + (M - 1) * L) &&
                      fabsf(m.eps) * (float)(M - 1) <= kSincSlack;
    if (!fast) {
        sinc_sft<M, L, false>(p, m, kh_row, ph0, lo_rel, cf, plane4, half, j_t, 0, 0x7fffffff, fa[0], fb[0]);
        sinc_sft<M, L, false>(p, m, kh_row + bs.dkh, ph0 + bs.dph, lo_rel, cf, plane4, half, j_t, 0, 0x7fffffff,
                              fa[1], fb[1]);
        return;
    }
    const float2 a2 = make_float2(m.a, m.a), b2 = make_float2(m.b, m.b);
    auto horner = [&](const float4* __restrict__ r, float v) -> float2 {
        const float4 e0 = r[0], e1 = r[1], e2 = r[2];
        const float2 vv = make_float2(v, v);
        float2 P = __ffma2_rn(make_float2(e2.z, e2.w), vv, make_float2(e2.x, e2.y));
        P = __ffma2_rn(P, vv, make_float2(e1.z, e1.w));
        P = __ffma2_rn(P, vv, make_float2(e1.x, e1.y));
        P = __ffma2_rn(P, vv, make_float2(e0.z, e0.w));
        return __ffma2_rn(P, vv, make_float2(e0.x, e0.y));
    };
    auto add = [&](float tr, float ti, float2 P, float2& fa_q, float2& fb_q) {
        const float2 z = make_float2(fmaf(tr, P.x, -ti * P.y), fmaf(tr, P.y, ti * P.x));
        fa_q = __ffma2_rn(a2, z, fa_q);
        fb_q = __ffma2_rn(b2, z, fb_q);
    };
    // window start and half bin of each row (the half chosen at its middle template)
    auto place = [&](long long kh, int k0, const float4*& cq, float& v0) {
        int bb = (k0 - (int)p.k_lo) - (D - 1) - lo_rel;
        if (bb < 0 || bb + (M - 1) * L + 2 * (D - 1) >= p.w_pairs) {
            atomicOr(p.err, 1);
            bb = max(0, min(bb, p.w_pairs - 1 - (M - 1) * L - 2 * (D - 1)));
        }
        const float u0 = frac_to_float((unsigned int)kh) - 0.5f;
        const bool up = fmaf(0.5f * (float)(M - 1), m.eps, u0) >= 0.f;
        cq = cf + (up ? plane4 : 0) + 3 * tab_pos<L>(bb + 7, half);
        v0 = u0 + (up ? -0.25f : 0.25f);
    };
    const float4 *cA, *cB;
    float vA, vB;
    place(khA, k0A, cA, vA);
    place(khB, k0B, cB, vB);
    const unsigned int ph = ph0 + (unsigned int)j_t * m.dphi + ((unsigned int)k0A << 31);
    float sn, cs;
    __sincosf((float)(int)ph * kPhaseToRad, &sn, &cs);
    float ar = cs, ai = -sn;
    float br = fmaf(ar, bs.rot_re, -ai * bs.rot_im), bi = fmaf(ar, bs.rot_im, ai * bs.rot_re);
    if ((k0B - k0A) & 1) {
        br = -br;
        bi = -bi;
    }
    if (cA == cB) {   // both rows read the same records
#pragma unroll
        for (int q = 0; q < M; ++q) {
            const float4* r = cA + 3 * q;
            const float4 e0 = r[0], e1 = r[1], e2 = r[2];
            const float2 va = make_float2(fmaf((float)q, m.eps, vA), fmaf((float)q, m.eps, vA));
            const float2 vb = make_float2(fmaf((float)q, m.eps, vB), fmaf((float)q, m.eps, vB));
            float2 PA = __ffma2_rn(make_float2(e2.z, e2.w), va, make_float2(e2.x, e2.y));
            float2 PB = __ffma2_rn(make_float2(e2.z, e2.w), vb, make_float2(e2.x, e2.y));
            PA = __ffma2_rn(PA, va, make_float2(e1.z, e1.w));
            PB = __ffma2_rn(PB, vb, make_float2(e1.z, e1.w));
            PA = __ffma2_rn(PA, va, make_float2(e1.x, e1.y));
            PB = __ffma2_rn(PB, vb, make_float2(e1.x, e1.y));
            PA = __ffma2_rn(PA, va, make_float2(e0.z, e0.w));
            PB = __ffma2_rn(PB, vb, make_float2(e0.z, e0.w));
            PA = __ffma2_rn(PA, va, make_float2(e0.x, e0.y));
            PB = __ffma2_rn(PB, vb, make_float2(e0.x, e0.y));
            add(ar, ai, PA, fa[0][q], fb[0][q]);
            add(br, bi, PB, fa[1][q], fb[1][q]);
            if (q + 1 < M) {
                const float ta = fmaf(ar, m.rot_re, -ai * m.rot_im);
                ai = fmaf(ar, m.rot_im, ai * m.rot_re);
                ar = ta;
                const float tb = fmaf(br, m.rot_re, -bi * m.rot_im);
                bi = fmaf(br, m.rot_im, bi * m.rot_re);
                br = tb;
            }
        }
    } else {
#pragma unroll
        for (int q = 0; q < M; ++q) {
            add(ar, ai, horner(cA + 3 * q, fmaf((float)q, m.eps, vA)), fa[0][q], fb[0][q]);
            add(br, bi, horner(cB + 3 * q, fmaf((float)q, m.eps, vB)), fa[1][q], fb[1][q]);
            if (q + 1 < M) {
                const float ta = fmaf(ar, m.rot_re, -ai * m.rot_im);
                ai = fmaf(ar, m.rot_im, ai * m.rot_re);
                ar = ta;
                const float tb = fmaf(br, m.rot_re, -bi * m.rot_im);
                bi = fmaf(br, m.rot_im, bi * m.rot_re);
                br = tb;
            }
        }
    }
}

// The ring block with two-row tiles: a lane-group holds rows 2 t and 2 t + 1
// (t = lane-group row pair); the last pair of an odd row count repeats its
// first row and stores one.
template <int M>
__device__ __forceinline__ void ring2_block(const DirichletParams& p, long long bid, unsigned char* smem) {
    const int S = p.sft_chunk;
    const RingSmem lay = ring_smem(S, p.w_tab, true);
    const int NW = (int)(blockDim.x >> 5) - 1;
    const int chunk = (int)(bid % p.chunks_per_col);
    bid /= p.chunks_per_col;
    const int sky = (int)(bid % p.n_sky);
    const int col = (int)(bid / p.n_sky);
    const int PM = p.P * M;
    const int col_w = p.lg_row * PM;
    const int j_col0 = col * col_w;
    const int width = min(col_w, p.n_f - j_col0);
    const int Gc = (width + PM - 1) / PM;
    const int n_pairs = (p.n_fdot + 1) >> 1;
    const int LG = n_pairs * Gc;
    const int u0 = chunk * p.lg_cta;
    if (u0 >= LG) return;   // block-uniform, before any barrier exists
    const int u_end = min(u0 + p.lg_cta, LG);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = (warp == NW);
    const int r = producer ? 0 : warp % p.P;
    const int ul = producer ? p.lg_cta : (warp / p.P) * 32 + lane;
    const int u = u0 + ul;
    const bool active = !producer && (ul < p.lg_cta) && (u < u_end);
    const int uu = active ? u : u0;
    const int pr = uu / Gc;
    const int g = uu - pr * Gc;
    const int dA = 2 * pr;
    const int dB = min(dA + 1, p.n_fdot - 1);
    const int j_t = j_col0 + g * PM + r;
    const bool warp_live = __any_sync(0xffffffffu, active);

    const uint32_t sb = smem_u32(smem);
    volatile int* ctrl = reinterpret_cast<volatile int*>(smem + lay.ctrl);
    auto full_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s); };
    auto empty_bar = [&](int s) { return sb + (uint32_t)(lay.bars + 16 * (size_t)s + 8); };
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), (uint32_t)NW);
        }
        ctrl[0] = 0;
        ctrl[1] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const size_t meta0 = (size_t)sky * p.n_sft;
    if (producer) {
        const int issued = ring_produce<true, false, 2>(p, lay, S, smem, sb, ctrl, meta0, j_col0, lane);
        if (lane == 0) ctrl[0] = issued;
    } else {
        float2 fa[2][M], fb[2][M];
#pragma unroll
        for (int q = 0; q < M; ++q) fa[0][q] = fb[0][q] = fa[1][q] = fb[1][q] = make_float2(0.f, 0.f);
        const int half = p.w_tab >> 1;
        int slot = 0;
        uint32_t parity = 0;
        for (int a = 0; a < p.n_sft; ++a) {
            const unsigned char* st = smem + (size_t)slot * lay.stage;
            if (!mbar_wait(full_bar(slot), parity)) {
                ctrl[1] = 1;
                atomicOr(p.err, 4);
                break;
            }
            if (warp_live) {
                const int lo_rel = *reinterpret_cast<const int*>(st + lay.lo);
                const SkySftMeta m = *reinterpret_cast<const SkySftMeta*>(st + lay.meta);
                SkySftBase bs = *reinterpret_cast<const SkySftBase*>(st + lay.base);
                const long long kh_row = bs.kh0 + (long long)dA * bs.dkh;
                const unsigned int ph_row = bs.ph0 + (unsigned int)dA * bs.dph;
                if (dB == dA) {   // odd row count: the last pair repeats its row (rot = 1, no step)
                    bs.dkh = 0;
                    bs.dph = 0u;
                    bs.rot_re = 1.f;
                    bs.rot_im = 0.f;
                }
                sinc_sft2<M>(p, m, bs, kh_row, ph_row, lo_rel, reinterpret_cast<const float4*>(st + lay.coef),
                             (int)(lay.plane >> 4), half, j_t, fa, fb);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(empty_bar(slot));
            if (ctrl[1]) break;
            if (++slot == S) {
                slot = 0;
                parity ^= 1u;
            }
        }
        if (active) {
            far_store<M>(p, sky, dA, j_t, j_col0 + width, fa[0], fb[0]);
            if (dB != dA) far_store<M>(p, sky, dB, j_t, j_col0 + width, fa[1], fb[1]);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (ctrl[1]) {
            const int issued = ctrl[0];
            for (int a = max(0, issued - S); a < issued; ++a) mbar_wait(full_bar(a % S), (uint32_t)((a / S) & 1));
        }
        for (int s = 0; s < S; ++s) {
            mbar_inval(full_bar(s));
            mbar_inval(empty_bar(s));
        }
    }
}

template <int M, int NWC, int MINB>
__global__ void __launch_bounds__(32 * (NWC + 1), MINB) dirichlet_ring2_kernel(const DirichletParams p) {
    extern __shared__ __align__(16) unsigned char smem[];
    ring2_block<M>(p, (long long)blockIdx.x, smem);
}

// Persistent ring form over many template banks (workunits): every block
// takes the next (bank, block) item from a device counter until all items of
// all banks are done, runs it as far_ring_block (whose barriers it sets up and
// invalidates), and the block that completes a bank's last item stamps its
// completion time.  At most `total` items per block; no block waits on another.
template <int M, int NWC, bool SINC, int SR = 1>
__global__ void __launch_bounds__(32 * (NWC + 1), 2)
    dirichlet_far_ring_batch_kernel(const DirichletParams* __restrict__ banks,
                                    const long long* __restrict__ item_prefix, int n_wu,
                                    unsigned long long* __restrict__ queue, int* __restrict__ remaining,
                                    unsigned long long* __restrict__ done_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_wu;
    const long long total = item_prefix[n_wu];
    for (long long guard = 0; guard <= total; ++guard) {
        __syncthreads();   // previous item fully consumed (shared memory and barriers free)
        if (threadIdx.x == 0) {
            const long long it = (long long)atomicAdd(queue, 1ULL);
            int lo = 0, hi = n_wu;   // last bank with item_prefix <= it
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (item_prefix[mid] <= it) lo = mid; else hi = mid;
            }
            s_item = it;
            s_wu = lo;
        }
        __syncthreads();
        const long long it = s_item;
        if (it >= total) break;
        const int w = s_wu;
        const DirichletParams p = banks[w];
        far_ring_block<M, SINC, false, 2, SR>(p, it - item_prefix[w], smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicSub(&remaining[w], 1) == 1) done_ns[w] = global_ns();
        }
    }
}
}  // namespace

// Compiled variants of the far-field form: (ID, M, L); IDs 7.. are the ring
// form (L = 2).
#define FS_FAR_VARIANTS(X) \
    X(0, 7, 2)             \
    X(1, 5, 2)             \
    X(2, 9, 2)             \
    X(3, 7, 1)             \
    X(4, 9, 1)             \
    X(5, 5, 1)             \
    X(6, 1, 1)
#define FS_RING_VARIANTS(X) \
    X(7, 5, 8, false)       \
    X(8, 7, 8, false)       \
    X(9, 9, 8, false)       \
    X(10, 5, 10, false)     \
    X(11, 7, 10, false)     \
    X(12, 5, 10, true)      \
    X(13, 7, 10, true)      \
    X(14, 5, 8, true)       \
    X(15, 7, 8, true)       \
    X(29, 5, 4, true)       \
    X(30, 5, 2, true)
// the same kernels with per-SFT frequency coverage (single launches only)
#define FS_RING_COV_VARIANTS(X) \
    X(16, 5, 10, true)          \
    X(17, 5, 10, false)
// blocks of 4 sky points: (ID, M, NWC, sinc, L)
#define FS_RING_SKY_VARIANTS(X) \
    X(31, 5, 10, true, 2)       \
    X(32, 5, 10, false, 2)      \
    X(33, 5, 8, true, 1)        \
    X(34, 1, 8, true, 1)
// the L = 2 ones also in the persistent batch kernel: (ID, M, NWC, sinc)
#define FS_RING_SKY2_VARIANTS(X) \
    X(31, 5, 10, true)           \
    X(32, 5, 10, false)
#define FS_BRCASE_SKY(ID, M_, W_, S_) FS_BRCASE(ID, M_, W_, S_, 4)
#define FS_BOCASE_SKY(ID, M_, W_, S_) FS_BOCASE(ID, M_, W_, S_, 4)
// sinc form for L = 1 banks (P = 8 threads per lane-group; single launches only)
#define FS_RING_L1_VARIANTS(X) \
    X(18, 5, 8, true)          \
    X(19, 1, 8, true)
// two-row tiles of the sinc form (L = 2): (ID, M, NWC compute warps, resident blocks per SM)
#define FS_RING2_VARIANTS(X) \
    X(27, 5, 8, 2)           \
    X(28, 3, 10, 2)
// rows form of the sinc polynomial: (ID, R rows per lane, NWC compute warps)
#define FS_ROWS_VARIANTS(X) \
    X(20, 10, 3)            \
    X(21, 10, 4)            \
    X(22, 10, 8)            \
    X(23, 5, 4)             \
    X(24, 5, 8)             \
    X(25, 8, 4)             \
    X(26, 4, 4)

cudaError_t launch_dirichlet_far(int v, const DirichletParams& p, int threads, size_t smem, long long grid,
                                 cudaStream_t s) {
    switch (v) {
#define FS_FCASE(ID, M_, L_)                                                                              \
    case ID: {                                                                                            \
        auto fn = dirichlet_far_kernel<M_, L_>;                                                           \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<(unsigned)grid, threads, smem, s>>>(p);                                                      \
        return cudaGetLastError();                                                                        \
    }
        FS_FAR_VARIANTS(FS_FCASE)
#undef FS_FCASE
#define FS_RCASE(ID, M_, W_, S_, C_, L_, ...)                                                             \
    case ID: {                                                                                            \
        auto fn = dirichlet_far_ring_kernel<M_, W_, S_, C_, L_, ##__VA_ARGS__>;                           \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<(unsigned)grid, threads, smem, s>>>(p);                                                      \
        return cudaGetLastError();                                                                        \
    }
#define FS_RCASE_PLAIN(ID, M_, W_, S_) FS_RCASE(ID, M_, W_, S_, false, 2)
#define FS_RCASE_COV(ID, M_, W_, S_) FS_RCASE(ID, M_, W_, S_, true, 2)
#define FS_RCASE_L1(ID, M_, W_, S_) FS_RCASE(ID, M_, W_, S_, false, 1)
#define FS_RCASE_SKY(ID, M_, W_, S_, L_) FS_RCASE(ID, M_, W_, S_, false, L_, 4)
        FS_RING_VARIANTS(FS_RCASE_PLAIN)
        FS_RING_COV_VARIANTS(FS_RCASE_COV)
        FS_RING_L1_VARIANTS(FS_RCASE_L1)
        FS_RING_SKY_VARIANTS(FS_RCASE_SKY)
#define FS_ROWCASE(ID, R_, W_)                                                                            \
    case ID: {                                                                                            \
        auto fn = dirichlet_rows_kernel<R_, W_>;                                                          \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<(unsigned)grid, threads, smem, s>>>(p);                                                      \
        return cudaGetLastError();                                                                        \
    }
        FS_ROWS_VARIANTS(FS_ROWCASE)
#undef FS_ROWCASE
#define FS_R2CASE(ID, M_, W_, B_)                                                                         \
    case ID: {                                                                                            \
        auto fn = dirichlet_ring2_kernel<M_, W_, B_>;                                                     \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<(unsigned)grid, threads, smem, s>>>(p);                                                      \
        return cudaGetLastError();                                                                        \
    }
        FS_RING2_VARIANTS(FS_R2CASE)
#undef FS_R2CASE
#undef FS_RCASE_SKY
#undef FS_RCASE_L1
#undef FS_RCASE_COV
#undef FS_RCASE_PLAIN
#undef FS_RCASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dirichlet_far_batch(int v, const DirichletBatch& b, int threads, size_t smem, int grid,
                                       cudaStream_t s) {
    switch (v) {
#define FS_BRCASE(ID, M_, W_, S_, ...)                                                                    \
    case ID: {                                                                                            \
        auto fn = dirichlet_far_ring_batch_kernel<M_, W_, S_, ##__VA_ARGS__>;                             \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<grid, threads, smem, s>>>(b.banks, b.item_prefix, b.n_wu, b.queue, b.remaining, b.done_ns);  \
        return cudaGetLastError();                                                                        \
    }
        FS_RING_VARIANTS(FS_BRCASE)
        FS_RING_SKY2_VARIANTS(FS_BRCASE_SKY)
#undef FS_BRCASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t dirichlet_far_batch_occupancy(int v, int threads, size_t smem, int* blocks_per_sm) {
    switch (v) {
#define FS_BOCASE(ID, M_, W_, S_, ...)                                                                    \
    case ID: {                                                                                            \
        auto fn = dirichlet_far_ring_batch_kernel<M_, W_, S_, ##__VA_ARGS__>;                             \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);           \
    }
        FS_RING_VARIANTS(FS_BOCASE)
        FS_RING_SKY2_VARIANTS(FS_BOCASE_SKY)
#undef FS_BOCASE
        default:
            return cudaErrorInvalidValue;
    }
}

cudaError_t launch_sinc_tables(const void* bins, int form, long long row, int n_sft, int n_bins,
                               const SincGamma& gam, float4* pcoef, int n_pos, int xoff, bool split,
                               cudaStream_t s) {
    const long long total = (long long)n_sft * n_pos;
    const int grid = (int)std::min<long long>((total + 255) / 256, (long long)current_sm_count() * 16);
    if (form == FSTAT_BINS_C64)
        sinc_tables_kernel<FSTAT_BINS_C64><<<grid, 256, 0, s>>>(static_cast<const float2*>(bins), row, n_sft, n_bins,
                                                                 gam, pcoef, n_pos, xoff, split);
    else if (form == FSTAT_BINS_F16)
        sinc_tables_kernel<FSTAT_BINS_F16><<<grid, 256, 0, s>>>(static_cast<const __half2*>(bins), row, n_sft,
                                                                 n_bins, gam, pcoef, n_pos, xoff, split);
    else
        sinc_tables_kernel<FSTAT_BINS_BF16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat162*>(bins), row, n_sft,
                                                                  n_bins, gam, pcoef, n_pos, xoff, split);
    return cudaGetLastError();
}

cudaError_t launch_far_tables(const void* bins, int form, long long row, int n_sft, int n_bins, const FarGamma& gam,
                              float4* ptab, float4* pcoef, int n_pos, int xoff, cudaStream_t s) {
    const long long total = (long long)n_sft * n_pos;
    const int grid = (int)std::min<long long>((total + 255) / 256, (long long)current_sm_count() * 16);
    if (form == FSTAT_BINS_C64)
        far_tables_kernel<FSTAT_BINS_C64><<<grid, 256, 0, s>>>(static_cast<const float2*>(bins), row, n_sft, n_bins,
                                                                gam, ptab, pcoef, n_pos, xoff);
    else if (form == FSTAT_BINS_F16)
        far_tables_kernel<FSTAT_BINS_F16><<<grid, 256, 0, s>>>(static_cast<const __half2*>(bins), row, n_sft, n_bins,
                                                                gam, ptab, pcoef, n_pos, xoff);
    else
        far_tables_kernel<FSTAT_BINS_BF16><<<grid, 256, 0, s>>>(static_cast<const __nv_bfloat162*>(bins), row, n_sft,
                                                                 n_bins, gam, ptab, pcoef, n_pos, xoff);
    return cudaGetLastError();
}

}  // namespace fs
