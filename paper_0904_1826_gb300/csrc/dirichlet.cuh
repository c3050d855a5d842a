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
// SFTs are processed in rounds of C.  While a round is being accumulated,
// cp.async copies bring in the next round's raw bins and the constants of the
// round after it; at the start of a round the raw bins become a table of
// adjacent-bin pairs (X_p + X_{p+1}, X_{p+1} - X_p) so that a pair of
// Dirichlet terms costs one reciprocal:
//   X_p/(c+1/2) + X_{p+1}/(c-1/2) = 2 (Y Sigma + Delta) / (Y^2 - 1),  Y = 2c,
// with c = khat - p - 1/2.  The two pairs next to the singular points
// (kappa -> 0 and kappa -> 1) take their denominators in a cancellation-free
// product form.
// Pair-table layout: when windows step by L = 2 bins the table is split by
// the parity of the pair index, so a thread's pairs are consecutive entries
// and neighbouring threads (M odd) sit an odd number of 16-byte slots apart:
// all loads are base + constant and free of bank conflicts.
#pragma once
#include "fstat_internal.cuh"

namespace fs {

constexpr float kKapMin = 5.9604645e-8f;  // 2^-24: below this the kernel is at its limit
constexpr float kKapMax = 0.99999994f;    // 1 - 2^-24
constexpr float kPhaseToRad = 1.4629180792671596e-09f;  // 2 pi / 2^32
constexpr int kMaxThreads = 320;

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ unsigned int smem_u32(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Raw storage element of one complex bin, and bins per 16-byte copy.
template <int FORM>
struct RawT;
template <>
struct RawT<FSTAT_BINS_C64> {
    using T = float2;
    static constexpr int G = 2;
    static __device__ __forceinline__ float2 f2(T x) { return x; }
};
template <>
struct RawT<FSTAT_BINS_F16> {
    using T = __half2;
    static constexpr int G = 4;
    static __device__ __forceinline__ float2 f2(T x) { return __half22float2(x); }
};
template <>
struct RawT<FSTAT_BINS_BF16> {
    using T = __nv_bfloat162;
    static constexpr int G = 4;
    static __device__ __forceinline__ float2 f2(T x) { return __bfloat1622float2(x); }
};

// Position of pair index i in the table row (split by parity for L = 2).
template <int L>
__device__ __forceinline__ int tab_pos(int i, int half) {
    return (L == 2) ? ((i & 1) * half + (i >> 1)) : i;
}

// Denominator of pair gi (bins k0-D+1+2gi, k0-D+2+2gi) times 4: Y^2 - 1 with
// Y = 2 kappa + 2D - 3 - 4 gi, in product form where it can vanish.
__device__ __forceinline__ float pair_den(int D, float Y, float kap, int gi) {
    if ((D & 1) == 0 && gi == D / 2 - 1) {          // offsets -1, 0: 4 kappa (kappa + 1)
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, k4);
    } else if ((D & 1) == 0 && gi == D / 2) {       // offsets 1, 2: 4 (kappa-1)(kappa-2)
        const float u = kap - 1.0f;
        const float u4 = 4.0f * u;
        return fmaf(u4, u, -u4);
    } else if ((D & 1) == 1 && gi == (D - 1) / 2) { // offsets 0, 1: 4 kappa (kappa - 1)
        const float k4 = 4.0f * kap;
        return fmaf(k4, kap, -k4);
    }
    return fmaf(Y, Y, -1.0f);
}

// Window sum of one template, Q = sum_pairs (Y Sigma + Delta) / (Y^2 - 1)
// (the pair form's factor 2 and the 1/pi of the kernel are folded into a, b);
// consecutive pairs of the window are STRIDE table entries apart.  The
// complex numerator and accumulator use packed FP32 (f32x2) operations.
template <int DV, int STRIDE>
__device__ __forceinline__ float2 window_sum(const float4* __restrict__ pp, float kap, int d_rt) {
    const int D = DV ? DV : d_rt;
    const float y0 = fmaf(2.0f, kap, (float)(2 * D - 3));
    const float2 y02 = make_float2(y0, y0);
    float2 Q = make_float2(0.f, 0.f);
#pragma unroll
    for (int gi = 0; gi < (DV ? DV : 64); ++gi) {
        if (!DV && gi >= D) break;
        const float4 e = pp[gi * STRIDE];
        const float Y = y0 - (float)(4 * gi);
        const float r = rcp_approx(pair_den(D, Y, kap, gi));
        const float2 S = __ffma2_rn(make_float2(Y, Y), make_float2(e.x, e.y), make_float2(e.z, e.w));
        Q = __ffma2_rn(S, make_float2(r, r), Q);
    }
    return Q;
}

// Pairs next to the singular points kappa = 0, 1 (exact reciprocal needed).
__host__ __device__ constexpr bool pair_is_singular(int D, int gi) {
    return ((D & 1) == 0) ? (gi == D / 2 - 1 || gi == D / 2) : (gi == (D - 1) / 2);
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

// Kahan step: t += x with running compensation c.
__device__ __forceinline__ void kahan_add(float& t, float& c, float x) {
    const float y = __fsub_rn(x, c);
    const float s = __fadd_rn(t, y);
    c = __fsub_rn(__fsub_rn(s, t), y);
    t = s;
}

// z = tw * sk * Q accumulated into Fa, Fb with weights a, b (packed pairs).
__device__ __forceinline__ void accumulate(float tw_re, float tw_im, float sk, float2 Q, float2 a2, float2 b2,
                                           float2& fa, float2& fb) {
    const float gre = tw_re * sk, gim = tw_im * sk;
    const float2 z = make_float2(fmaf(gre, Q.x, -gim * Q.y), fmaf(gre, Q.y, gim * Q.x));
    fa = __ffma2_rn(a2, z, fa);
    fb = __ffma2_rn(b2, z, fb);
}

// One thread block's work item: block index `bid` of the grid that covers
// (sky, column, chunk) of one template bank.  DV = D (compile time) or 0 (D
// taken from the runtime argument, M = 1).  Every exit is block-uniform
// except the final per-thread epilogue, so callers may loop over items.
template <int DV, int M, int L, int FORM, bool KAHAN>
__device__ __forceinline__ void dirichlet_block(const DirichletParams& p, const int d_rt, long long bid,
                                                unsigned char* smem) {
    using RT = RawT<FORM>;
    using Raw = typename RT::T;
    constexpr int G = RT::G;
    constexpr int STRIDE = (L == 2) ? 1 : 2;
    const int D = DV ? DV : d_rt;
    const int NT = blockDim.x;
    const int C = p.sft_chunk;
    const DirSmem lay = dirichlet_smem(C, p.w_tab, p.w_raw, p.n_fdot, (int)sizeof(Raw));
    float4* s_tab = reinterpret_cast<float4*>(smem + lay.pairs);            // [C][w_tab]
    Raw* s_raw = reinterpret_cast<Raw*>(smem + lay.raw);                    // [2][C][w_raw]
    SkySftMeta* s_meta = reinterpret_cast<SkySftMeta*>(smem + lay.meta);    // [3][C]
    SkySftBase* s_base = reinterpret_cast<SkySftBase*>(smem + lay.base);    // [3][C]
    long long* s_kh0 = reinterpret_cast<long long*>(smem + lay.kh0);        // [3][C][n_fdot]
    unsigned int* s_ph0 = reinterpret_cast<unsigned int*>(smem + lay.ph0);  // [3][C][n_fdot]
    int* s_lo = reinterpret_cast<int*>(smem + lay.lo);                      // [2][C][2]: window base, raw start

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
    const int half = p.w_tab >> 1;

    const size_t meta0 = (size_t)sky * p.n_sft;
    const size_t base0 = (size_t)sky * p.n_fdot * p.n_sft;
    const int n_rounds = (p.n_sft + C - 1) / C;

    // ---- staging helpers -------------------------------------------------
    auto issue_consts = [&](int rd) {
        const int a0 = rd * C, slot = rd % 3;
        const int nc = min(C, p.n_sft - a0);
        const char* msrc = reinterpret_cast<const char*>(p.meta + meta0 + a0);
        char* mdst = reinterpret_cast<char*>(s_meta + slot * C);
        for (int t = threadIdx.x; t < nc * 3; t += NT) cp_async16(mdst + 16 * t, msrc + 16 * t, 16);
        if (p.base) {   // uniform spindown grid: two 16-byte halves per SFT
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
    auto compute_lo = [&](int rd) {
        const int a0 = rd * C, cslot = rd % 3, lslot = rd & 1;
        const int nc = min(C, p.n_sft - a0);
        for (int c = threadIdx.x; c < nc; c += NT) {
            const SkySftMeta& m = s_meta[cslot * C + c];
            const long long kb = m.khmin + (long long)j_col0 * m.dk;
            const int lo_rel = (int)((kb >> 32) - p.k_lo) - (D - 1);
            const int raw_rel = (lo_rel >= 0) ? (lo_rel / G) * G : -((-lo_rel + G - 1) / G) * G;
            s_lo[(lslot * C + c) * 2] = lo_rel;
            s_lo[(lslot * C + c) * 2 + 1] = raw_rel;
        }
    };
    auto issue_raw = [&](int rd) {
        const int a0 = rd * C, slot = rd & 1;
        const int nc = min(C, p.n_sft - a0);
        const int gpr = p.w_raw / G;
        const Raw* bins = reinterpret_cast<const Raw*>(p.bins);
        for (int t = threadIdx.x; t < nc * gpr; t += NT) {
            const int c = t / gpr, gi = t - c * gpr;
            const long long x = (long long)s_lo[(slot * C + c) * 2 + 1] + (long long)gi * G;
            const bool in = (x >= 0) && (x < p.row);
            const Raw* src = bins + (size_t)(a0 + c) * p.row + (in ? x : 0);
            cp_async16(s_raw + ((size_t)slot * C + c) * p.w_raw + gi * G, src, in ? 16 : 0);
        }
    };
    auto build_pairs = [&](int rd) {
        const int a0 = rd * C, slot = rd & 1;
        const int nc = min(C, p.n_sft - a0);
        for (int e = threadIdx.x; e < nc * p.w_pairs; e += NT) {
            const int c = e / p.w_pairs, i = e - c * p.w_pairs;
            const int ri = s_lo[(slot * C + c) * 2] - s_lo[(slot * C + c) * 2 + 1] + i;
            const Raw* rw = s_raw + ((size_t)slot * C + c) * p.w_raw;
            const float2 x0 = RT::f2(rw[ri]), x1 = RT::f2(rw[ri + 1]);
            s_tab[(size_t)c * p.w_tab + tab_pos<L>(i, half)] =
                make_float4(x0.x + x1.x, x0.y + x1.y, x1.x - x0.x, x1.y - x0.y);
        }
    };

    float2 fa[M], fb[M];
    float2 ca[M], cb[M];   // Kahan compensation (KAHAN only)
    float2 ta[M], tb[M];   // Kahan totals (KAHAN only)
#pragma unroll
    for (int q = 0; q < M; ++q) {
        fa[q] = fb[q] = ca[q] = cb[q] = ta[q] = tb[q] = make_float2(0.f, 0.f);
    }
    int bad = 0;

    // ---- prologue: constants of rounds 0 and 1, raw bins of round 0
    issue_consts(0);
    if (n_rounds > 1) issue_consts(1);
    cp_async_commit();
    cp_async_wait_all();
    __syncthreads();
    compute_lo(0);
    __syncthreads();
    issue_raw(0);
    cp_async_commit();

    for (int rd = 0; rd < n_rounds; ++rd) {
        const int a0 = rd * C;
        const int nc = min(C, p.n_sft - a0);
        const int cslot = rd % 3, lslot = rd & 1;
        cp_async_wait_all();
        __syncthreads();   // raw(rd), consts(rd+1) visible; everyone done with round rd-1
        build_pairs(rd);
        if (rd + 1 < n_rounds) compute_lo(rd + 1);
        __syncthreads();   // pair table and next window bases ready
        if (rd + 1 < n_rounds) issue_raw(rd + 1);
        if (rd + 2 < n_rounds) issue_consts(rd + 2);
        cp_async_commit();

        // warps walk the round's SFTs from different starting points so that
        // their reciprocal-heavy and multiply-add-heavy phases interleave
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
            // frequency coverage: skip the SFT if it covers none of the
            // thread's templates, mask per template if it covers some
            int clo = 0, chi = 0x7fffffff;
            if (p.cov) {
                const int2 cv = __ldg(p.cov + a0 + c);
                clo = cv.x;
                chi = cv.y;
            }
            const int j_last = j_t + (M - 1) * p.P;
            if (j_last < clo || j_t >= chi) continue;
            const bool part = j_t < clo || j_last >= chi;
            const long long kh = kh_row + (long long)j_t * m.dk;
            const int k0 = (int)(kh >> 32);
            const int lo_rel = s_lo[(lslot * C + c) * 2];
            const int b = (k0 - (int)p.k_lo) - (D - 1) - lo_rel;   // first pair of template 0
            const float4* tab = s_tab + (size_t)c * p.w_tab;
            const float2 a2 = make_float2(m.a, m.a), b2 = make_float2(m.b, m.b);
            const bool fast = !part && ((int)((kh + m.span) >> 32) == k0 + (M - 1) * L);
            if (fast) {
                int bb = b;
                if (bb < 0 || bb + (M - 1) * L + 2 * (D - 1) >= p.w_pairs) {
                    bad = 1;
                    bb = max(0, min(bb, p.w_pairs - 1 - (M - 1) * L - 2 * (D - 1)));
                }
                const float4* pp = tab + tab_pos<L>(bb, half);
                const unsigned int ph = ph0 + (unsigned int)j_t * m.dphi + ((unsigned int)k0 << 31);
                float sn, cs;
                __sincosf((float)(int)ph * kPhaseToRad, &sn, &cs);
                float tw_re = cs, tw_im = -sn;
                const float kap0 = clamp_kappa(frac_to_float((unsigned int)kh));

#pragma unroll
                for (int q = 0; q < M; ++q) {
                    const float kap = clamp_kappa(fmaf((float)q, m.eps, kap0));
                    const float2 Q = window_sum<DV, STRIDE>(pp + q, kap, d_rt);
                    const float sk = sinpi_unit(kap);
                    accumulate(tw_re, tw_im, sk, Q, a2, b2, fa[q], fb[q]);
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
                    if (part && (j_t + q * p.P < clo || j_t + q * p.P >= chi)) continue;
                    const long long khq = kh + (long long)q * pdk;
                    const int k0q = (int)(khq >> 32);
                    const float kap = clamp_kappa(frac_to_float((unsigned int)khq));
                    const unsigned int phq = ph0 + (unsigned int)(j_t + q * p.P) * m.dphi + ((unsigned int)k0q << 31);
                    float s2, c2;
                    __sincosf((float)(int)phq * kPhaseToRad, &s2, &c2);
                    int bq = (k0q - (int)p.k_lo) - (D - 1) - lo_rel;
                    if (bq < 0 || bq + 2 * (D - 1) >= p.w_pairs) {
                        bad = 1;
                        bq = max(0, min(bq, p.w_pairs - 1 - 2 * (D - 1)));
                    }
                    const float2 Q = window_sum<DV, STRIDE>(tab + tab_pos<L>(bq, half), kap, d_rt);
                    accumulate(c2, -s2, sinpi_unit(kap), Q, a2, b2, fa[q], fb[q]);
                }
            }
        }
        if (KAHAN) {
            // compensated addition of this round's partial sums into the totals
#pragma unroll
            for (int q = 0; q < M; ++q) {
                kahan_add(ta[q].x, ca[q].x, fa[q].x);
                kahan_add(ta[q].y, ca[q].y, fa[q].y);
                kahan_add(tb[q].x, cb[q].x, fb[q].x);
                kahan_add(tb[q].y, cb[q].y, fb[q].y);
                fa[q] = fb[q] = make_float2(0.f, 0.f);
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
            const float4 cw = p.comb_j ? p.comb_j[(size_t)sky * p.n_f + j] : cm;
            const float2 A_ = KAHAN ? ta[q] : fa[q];
            const float2 B_ = KAHAN ? tb[q] : fb[q];
            const float v = cw.x * fmaf(A_.x, A_.x, A_.y * A_.y) + cw.y * fmaf(B_.x, B_.x, B_.y * B_.y) +
                            cw.z * fmaf(A_.x, B_.x, A_.y * B_.y);
            out[j] = fmaxf(v, 0.0f);
        }
    }
}

template <int DV, int M, int L, int FORM, bool KAHAN>
__global__ void __launch_bounds__(kMaxThreads, 2) dirichlet_kernel(const DirichletParams p, const int d_rt) {
    extern __shared__ __align__(16) unsigned char smem[];
    dirichlet_block<DV, M, L, FORM, KAHAN>(p, d_rt, (long long)blockIdx.x, smem);
}

// Persistent form over many template banks (workunits): every block takes
// the next item from a device queue until all items of all banks are done.
// item_prefix[w] is the first item of bank w (item_prefix[n_wu] = total);
// the block that completes a bank's last item stamps its completion time.
// The loop ends after at most `total` items per block; nothing waits on
// another block.
template <int DV, int M, int L, int FORM, bool KAHAN>
__global__ void __launch_bounds__(kMaxThreads, 2)
    dirichlet_batch_kernel(const DirichletParams* __restrict__ banks, const long long* __restrict__ item_prefix,
                           int n_wu, unsigned long long* __restrict__ queue, int* __restrict__ remaining,
                           unsigned long long* __restrict__ done_ns, const int d_rt) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_item;
    __shared__ int s_wu;
    const long long total = item_prefix[n_wu];
    for (long long guard = 0; guard <= total; ++guard) {
        __syncthreads();   // previous item fully consumed (shared memory free)
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
        dirichlet_block<DV, M, L, FORM, KAHAN>(p, d_rt, it - item_prefix[w], smem);
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicSub(&remaining[w], 1) == 1) {
                unsigned long long t;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
                done_ns[w] = t;
            }
        }
    }
}

// Compiled variants: (ID, D, M, L, KAHAN); D = 0 takes D at run time.
#define FS_DIRICHLET_VARIANTS(X) \
    X(0, 8, 9, 2, false)          \
    X(1, 8, 7, 2, false)          \
    X(2, 8, 5, 2, false)          \
    X(3, 8, 9, 1, false)          \
    X(4, 8, 7, 1, false)          \
    X(5, 8, 1, 1, false)          \
    X(6, 8, 5, 2, true)           \
    X(7, 8, 5, 1, true)           \
    X(8, 8, 1, 1, true)           \
    X(9, 0, 1, 1, false)          \
    X(10, 0, 1, 1, true)

template <int FORM>
cudaError_t launch_dirichlet_batch_form(int v, const DirichletBatch& b, int d_rt, int threads, size_t smem,
                                        int grid, cudaStream_t s) {
    switch (v) {
#define FS_BCASE(ID, D_, M_, L_, K_)                                                                      \
    case ID: {                                                                                            \
        auto fn = dirichlet_batch_kernel<D_, M_, L_, FORM, K_>;                                           \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<grid, threads, smem, s>>>(b.banks, b.item_prefix, b.n_wu, b.queue, b.remaining, b.done_ns,   \
                                       d_rt);                                                             \
        return cudaGetLastError();                                                                        \
    }
        FS_DIRICHLET_VARIANTS(FS_BCASE)
#undef FS_BCASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <int FORM>
cudaError_t dirichlet_occupancy_form(int v, int threads, size_t smem, int* blocks_per_sm) {
    switch (v) {
#define FS_OCASE(ID, D_, M_, L_, K_)                                                                          \
    case ID: {                                                                                                \
        auto fn = dirichlet_batch_kernel<D_, M_, L_, FORM, K_>;                                               \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);     \
        if (e != cudaSuccess) return e;                                                                       \
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, threads, smem);               \
    }
        FS_DIRICHLET_VARIANTS(FS_OCASE)
#undef FS_OCASE
        default:
            return cudaErrorInvalidValue;
    }
}

template <int FORM>
cudaError_t launch_dirichlet_form(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                                  long long grid, cudaStream_t s) {
    switch (v) {
#define FS_CASE(ID, D_, M_, L_, K_)                                                                       \
    case ID: {                                                                                            \
        auto fn = dirichlet_kernel<D_, M_, L_, FORM, K_>;                                                 \
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
        if (e != cudaSuccess) return e;                                                                   \
        fn<<<(unsigned)grid, threads, smem, s>>>(p, d_rt);                                                \
        return cudaGetLastError();                                                                        \
    }
        FS_DIRICHLET_VARIANTS(FS_CASE)
#undef FS_CASE
        default:
            return cudaErrorInvalidValue;
    }
}

}  // namespace fs
