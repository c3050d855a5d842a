// Dirichlet-kernel accumulation of Fa, Fb over SFTs with the 2F combine fused
// into the epilogue: the per-SFT term of the F-statistic loop (the SFT loop of
// Listing 1, "some_calculations") for many templates at once.
//
// Work decomposition (one thread block):
//   one sky point, one "column" of frequencies, a contiguous run of
//   (spindown row, lane-group) slots.  A lane-group is P threads that
//   together own P*M consecutive frequencies; thread r of the group owns
//   frequencies j_t + P*q, q = 0..M-1, whose bin windows sit L bins apart
//   (P * df * T ~= L), so the M windows of a thread overlap and their bins
//   are read once from shared memory into registers.
// Per SFT round the block stages, for every SFT of the round, the bin span
// its templates can touch as a table of adjacent-bin pairs
//   (X_p + X_{p+1}, X_{p+1} - X_p)
// so that a pair of Dirichlet terms costs one reciprocal:
//   X_p/(c+1/2) + X_{p+1}/(c-1/2) = 2 (Y Sigma + Delta) / (Y^2 - 1),  Y = 2c,
// with c = khat - p - 1/2.  The two pairs next to the singular points
// (kappa -> 0 and kappa -> 1) take their denominators in a cancellation-free
// product form.
#pragma once
#include "fstat_internal.cuh"

namespace fs {

constexpr int kPadShift = 4;              // one padding entry per 16 pair entries
constexpr float kKapMin = 5.9604645e-8f;  // 2^-24: below this the kernel is at its limit
constexpr float kKapMax = 0.99999994f;    // 1 - 2^-24
constexpr float kPhaseToRad = 1.4629180792671596e-09f;  // 2 pi / 2^32

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <int FORM>
__device__ __forceinline__ float2 load_bin(const void* __restrict__ bins, long long off) {
    if (FORM == FSTAT_BINS_C64) {
        return __ldg(reinterpret_cast<const float2*>(bins) + off);
    } else if (FORM == FSTAT_BINS_F16) {
        const __half2 h = reinterpret_cast<const __half2*>(bins)[off];
        return __half22float2(h);
    } else {
        const __nv_bfloat162 h = reinterpret_cast<const __nv_bfloat162*>(bins)[off];
        return __bfloat1622float2(h);
    }
}

__device__ __forceinline__ int pad_idx(int i) { return i + (i >> kPadShift); }

// Denominator of pair gi (bins k0-D+1+2gi, k0-D+2+2gi) times 4: Y^2 - 1 with
// Y = 2 kappa + 2D - 3 - 4 gi, in product form where it can vanish.
template <int D>
__device__ __forceinline__ float pair_den(float Y, float kap, int gi) {
    if ((D & 1) == 0 && gi == D / 2 - 1) {        // offsets -1, 0: 4 kappa (kappa + 1)
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, k4);
    } else if ((D & 1) == 0 && gi == D / 2) {     // offsets 1, 2: 4 (kappa-1)(kappa-2)
        const float u = kap - 1.0f;
        const float u4 = 4.0f * u;
        return fmaf(u4, u, -u4);
    } else if ((D & 1) == 1 && gi == (D - 1) / 2) {   // offsets 0, 1: 4 kappa (kappa - 1)
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, -k4);
    }
    return fmaf(Y, Y, -1.0f);
}

__device__ __forceinline__ float pair_den_rt(int D, float Y, float kap, int gi) {
    if ((D & 1) == 0 && gi == D / 2 - 1) {
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, k4);
    } else if ((D & 1) == 0 && gi == D / 2) {
        const float u = kap - 1.0f;
        const float u4 = 4.0f * u;
        return fmaf(u4, u, -u4);
    } else if ((D & 1) == 1 && gi == (D - 1) / 2) {
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, -k4);
    }
    return fmaf(Y, Y, -1.0f);
}

// Sum over the 2D window of one template: Q = sum_pairs (Y Sigma + Delta) / (Y^2 - 1)
// (the factor 2 of the pair form and 1/pi are folded into a, b).
template <int D>
__device__ __forceinline__ void window_sum(const float4* __restrict__ row, int base, float kap,
                                           float& Qre, float& Qim) {
    const float y0 = fmaf(2.0f, kap, (float)(2 * D - 3));
    Qre = 0.f;
    Qim = 0.f;
#pragma unroll
    for (int gi = 0; gi < D; ++gi) {
        const float4 e = row[pad_idx(base + 2 * gi)];
        const float Y = y0 - (float)(4 * gi);
        const float r = rcp_approx(pair_den<D>(Y, kap, gi));
        Qre = fmaf(fmaf(Y, e.x, e.z), r, Qre);
        Qim = fmaf(fmaf(Y, e.y, e.w), r, Qim);
    }
}

__device__ __forceinline__ void window_sum_rt(int D, const float4* __restrict__ row, int base, float kap,
                                              float& Qre, float& Qim) {
    const float y0 = fmaf(2.0f, kap, (float)(2 * D - 3));
    Qre = 0.f;
    Qim = 0.f;
    for (int gi = 0; gi < D; ++gi) {
        const float4 e = row[pad_idx(base + 2 * gi)];
        const float Y = y0 - (float)(4 * gi);
        const float r = rcp_approx(pair_den_rt(D, Y, kap, gi));
        Qre = fmaf(fmaf(Y, e.x, e.z), r, Qre);
        Qim = fmaf(fmaf(Y, e.y, e.w), r, Qim);
    }
}

// Fixed-point fraction (2^-32 units) to float in [0, 1), truncated to 23 bits.
__device__ __forceinline__ float frac_to_float(unsigned int fr) {
    return __int_as_float(0x3f800000u | (fr >> 9)) - 1.0f;
}

__device__ __forceinline__ float clamp_kappa(float k) { return fminf(fmaxf(k, kKapMin), kKapMax); }

// sin(pi x) for x in [0, 1) with small relative error near both ends (the
// kernel multiplies it by ~1/kappa): reflect to t = min(x, 1-x) in [0, 1/2]
// and sum the Taylor series of sin(pi t) through t^11 (truncation < 6e-8
// relative on [0, 1/2]).
__device__ __forceinline__ float sinpi_unit(float x) {
    const float t = fminf(x, 1.0f - x);
    const float t2 = t * t;
    float p = -7.370431e-03f;          // -pi^11 / 11!
    p = fmaf(p, t2, 8.2145885e-02f);   //  pi^9 / 9!
    p = fmaf(p, t2, -0.5992645f);      // -pi^7 / 7!
    p = fmaf(p, t2, 2.550164f);        //  pi^5 / 5!
    p = fmaf(p, t2, -5.1677127f);      // -pi^3 / 3!
    p = fmaf(p, t2, 3.1415927f);       //  pi
    return p * t;
}

struct Accum {
    float re, im;
};

// Kahan step: t += x with running compensation c.
__device__ __forceinline__ void kahan_add(float& t, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float s = __fadd_rn(t, y);
    c = __fsub_rn(__fsub_rn(s, t), y);
    t = s;
}

constexpr int kMaxThreads = 320;

// DV = D (compile time) or 0 (D taken from the runtime argument).
template <int DV, int M, int L, int FORM, bool KAHAN>
__global__ void __launch_bounds__(kMaxThreads, 2)
dirichlet_kernel(const DirichletParams p, const int d_rt) {
    const int THREADS = blockDim.x;
    constexpr bool RT = (DV == 0);
    const int D = RT ? d_rt : DV;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int C = p.sft_chunk;
    float4* s_pairs = reinterpret_cast<float4*>(smem_raw);
    SkySftMeta* s_meta = reinterpret_cast<SkySftMeta*>(s_pairs + (size_t)C * p.w_pad);
    long long* s_kh0 = reinterpret_cast<long long*>(s_meta + C);
    unsigned int* s_ph0 = reinterpret_cast<unsigned int*>(s_kh0 + (size_t)C * p.n_fdot);
    int* s_lo = reinterpret_cast<int*>(s_ph0 + (size_t)C * p.n_fdot);

    long long bid = blockIdx.x;
    const int chunk = (int)(bid % p.chunks_per_col);
    bid /= p.chunks_per_col;
    const int col = (int)(bid % p.n_col);
    const int sky = (int)(bid / p.n_col);
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

    Accum fa[M], fb[M];
    Accum ca[M], cb[M];   // Kahan compensation (KAHAN only)
    Accum ta[M], tb[M];   // Kahan totals (KAHAN only)
#pragma unroll
    for (int q = 0; q < M; ++q) {
        fa[q] = {0.f, 0.f};
        fb[q] = {0.f, 0.f};
        ca[q] = {0.f, 0.f};
        cb[q] = {0.f, 0.f};
        ta[q] = {0.f, 0.f};
        tb[q] = {0.f, 0.f};
    }
    const size_t meta0 = (size_t)sky * p.n_sft;
    const size_t base0 = (size_t)sky * p.n_fdot * p.n_sft;
    int bad = 0;

    for (int a0 = 0; a0 < p.n_sft; a0 += C) {
        const int nc = min(C, p.n_sft - a0);
        __syncthreads();   // the previous round's readers are done
        // ---- stage per-SFT constants and the window base of this block
        for (int i = threadIdx.x; i < nc; i += THREADS) {
            const SkySftMeta m = p.meta[meta0 + a0 + i];
            s_meta[i] = m;
            // lowest window start over the block's spindown rows (any order)
            long long kmin = p.kh0[base0 + (size_t)d_lo * p.n_sft + a0 + i];
            for (int rr = d_lo + 1; rr <= d_hi; ++rr) {
                const long long k = p.kh0[base0 + (size_t)rr * p.n_sft + a0 + i];
                kmin = k < kmin ? k : kmin;
            }
            s_lo[i] = (int)((kmin + (long long)j_col0 * m.dk) >> 32) - (D - 1);
        }
        for (int i = threadIdx.x; i < nc * n_rows; i += THREADS) {
            const int c = i / n_rows, rr = i - c * n_rows;
            const size_t o = base0 + (size_t)(d_lo + rr) * p.n_sft + a0 + c;
            s_kh0[c * p.n_fdot + rr] = p.kh0[o];
            s_ph0[c * p.n_fdot + rr] = p.ph0[o];
        }
        __syncthreads();
        // ---- pair table of the bins this block can touch (zero outside the band)
        for (int e = threadIdx.x; e < nc * p.w_pairs; e += THREADS) {
            const int c = e / p.w_pairs;
            const int i = e - c * p.w_pairs;
            const long long off = (long long)s_lo[c] + i - p.k_lo;
            const long long rowoff = (long long)(a0 + c) * p.row;
            float2 x0 = make_float2(0.f, 0.f), x1 = make_float2(0.f, 0.f);
            if (off >= 0 && off < p.n_bins) x0 = load_bin<FORM>(p.bins, rowoff + off);
            if (off + 1 >= 0 && off + 1 < p.n_bins) x1 = load_bin<FORM>(p.bins, rowoff + off + 1);
            s_pairs[(size_t)c * p.w_pad + pad_idx(i)] = make_float4(x0.x + x1.x, x0.y + x1.y, x1.x - x0.x, x1.y - x0.y);
        }
        __syncthreads();
        // ---- accumulate this round's SFTs (warps without templates only stage)
        for (int c = 0; c < (warp_live ? nc : 0); ++c) {
            const SkySftMeta m = s_meta[c];
            const long long kh = s_kh0[c * p.n_fdot + row_i] + (long long)j_t * m.dk;
            const int k0 = (int)(kh >> 32);
            const unsigned int ph = s_ph0[c * p.n_fdot + row_i] + (unsigned int)j_t * m.dphi + ((unsigned int)k0 << 31);
            const float4* prow = s_pairs + (size_t)c * p.w_pad;
            const int lo = s_lo[c];
            const bool fast = ((int)((kh + m.span) >> 32) == k0 + (M - 1) * L);
            float sn, cs;
            __sincosf((float)(int)ph * kPhaseToRad, &sn, &cs);
            float tw_re = cs, tw_im = -sn;
            if (fast) {
                int base = k0 - (D - 1) - lo;
                const int last = base + (M - 1) * L + 2 * (D - 1);
                if (base < 0 || last >= p.w_pairs) {
                    bad = 1;
                    base = max(0, min(base, p.w_pairs - 1 - (M - 1) * L - 2 * (D - 1)));
                }
                const float kap0 = frac_to_float((unsigned int)kh);
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float kap = clamp_kappa(fmaf((float)q, m.eps, kap0));
                    float Qre, Qim;
                    if (RT)
                        window_sum_rt(D, prow, base + q * L, kap, Qre, Qim);
                    else
                        window_sum<(RT ? 8 : DV)>(prow, base + q * L, kap, Qre, Qim);
                    const float sk = sinpi_unit(kap);
                    const float gre = tw_re * sk, gim = tw_im * sk;
                    const float zre = fmaf(gre, Qre, -gim * Qim);
                    const float zim = fmaf(gre, Qim, gim * Qre);
                    fa[q].re = fmaf(m.a, zre, fa[q].re);
                    fa[q].im = fmaf(m.a, zim, fa[q].im);
                    fb[q].re = fmaf(m.b, zre, fb[q].re);
                    fb[q].im = fmaf(m.b, zim, fb[q].im);
                    if (q + 1 < M) {
                        const float t = fmaf(tw_re, m.rot_re, -tw_im * m.rot_im);
                        tw_im = fmaf(tw_re, m.rot_im, tw_im * m.rot_re);
                        tw_re = t;
                    }
                }
            } else {
                const long long pdk = (long long)p.P * m.dk;
                const unsigned int pdphi = (unsigned int)p.P * m.dphi;
#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const long long khq = kh + (long long)q * pdk;
                    const int k0q = (int)(khq >> 32);
                    const float kap = clamp_kappa(frac_to_float((unsigned int)khq));
                    const unsigned int phq = s_ph0[c * p.n_fdot + row_i] + (unsigned int)(j_t + q * p.P) * m.dphi +
                                             ((unsigned int)k0q << 31);
                    (void)pdphi;
                    float s2, c2;
                    __sincosf((float)(int)phq * kPhaseToRad, &s2, &c2);
                    int base = k0q - (D - 1) - lo;
                    if (base < 0 || base + 2 * (D - 1) >= p.w_pairs) {
                        bad = 1;
                        base = max(0, min(base, p.w_pairs - 1 - 2 * (D - 1)));
                    }
                    float Qre, Qim;
                    if (RT)
                        window_sum_rt(D, prow, base, kap, Qre, Qim);
                    else
                        window_sum<(RT ? 8 : DV)>(prow, base, kap, Qre, Qim);
                    const float sk = sinpi_unit(kap);
                    const float gre = c2 * sk, gim = -s2 * sk;
                    const float zre = fmaf(gre, Qre, -gim * Qim);
                    const float zim = fmaf(gre, Qim, gim * Qre);
                    fa[q].re = fmaf(m.a, zre, fa[q].re);
                    fa[q].im = fmaf(m.a, zim, fa[q].im);
                    fb[q].re = fmaf(m.b, zre, fb[q].re);
                    fb[q].im = fmaf(m.b, zim, fb[q].im);
                }
            }
        }
        if (KAHAN) {
            // compensated addition of this round's partial sums into the totals
#pragma unroll
            for (int q = 0; q < M; ++q) {
                kahan_add(ta[q].re, ca[q].re, fa[q].re);
                kahan_add(ta[q].im, ca[q].im, fa[q].im);
                kahan_add(tb[q].re, cb[q].re, fb[q].re);
                kahan_add(tb[q].im, cb[q].im, fb[q].im);
                fa[q] = {0.f, 0.f};
                fb[q] = {0.f, 0.f};
            }
        }
    }
    if (bad) atomicOr(p.err, 1);
    // ---- 2F combine
    if (!active) return;
    const float4 cm = p.comb[sky];
    float* out = p.twoF + ((size_t)sky * p.n_fdot + drow) * p.n_f;
    const int j_end = j_col0 + width;
#pragma unroll
    for (int q = 0; q < M; ++q) {
        const int j = j_t + q * p.P;
        if (j < j_end) {
            const Accum A_ = KAHAN ? ta[q] : fa[q];
            const Accum B_ = KAHAN ? tb[q] : fb[q];
            float v = cm.x * fmaf(A_.re, A_.re, A_.im * A_.im) + cm.y * fmaf(B_.re, B_.re, B_.im * B_.im) +
                      cm.z * fmaf(A_.re, B_.re, A_.im * B_.im);
            out[j] = fmaxf(v, 0.0f);
        }
    }
}

// Compiled variants: (D, M, L, KAHAN); D = 0 takes D at run time.
#define FS_DIRICHLET_VARIANTS(X) \
    X(0, 8, 9, 2, false)          \
    X(1, 8, 8, 2, false)          \
    X(2, 8, 8, 1, false)          \
    X(3, 8, 1, 1, false)          \
    X(4, 8, 4, 2, true)           \
    X(5, 8, 4, 1, true)           \
    X(6, 8, 1, 1, true)           \
    X(7, 0, 1, 1, false)          \
    X(8, 0, 1, 1, true)

constexpr int kNumDirichletVariants = 9;

template <int FORM>
cudaError_t launch_dirichlet_form(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                                  long long grid, cudaStream_t s) {
    switch (v) {
#define FS_CASE(ID, D_, M_, L_, K_)                                                                  \
    case ID: {                                                                                       \
        auto fn = dirichlet_kernel<D_, M_, L_, FORM, K_>;                                            \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                              \
        fn<<<(unsigned)grid, threads, smem, s>>>(p, d_rt);                                           \
        return cudaGetLastError();                                                                   \
    }
        FS_DIRICHLET_VARIANTS(FS_CASE)
#undef FS_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace fs
