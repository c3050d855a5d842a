// Semicoherent stack-slide over segments: the stage after the coherent
// F-statistic (the paper's client runs a semicoherent Hough stage there,
// Section "Einstein@Home"; this is the generic stack-slide form).
//
//   out[sky][m][j] = sum_s twoF_s[sky][m][i_s(m, j)]   (FP32, segment order)
//   i_s(m, j) = (A_fx[s][m] + j B_fx[s] + 2^31) >> 32
//
// A_fx, B_fx are the 32.32 fixed-point forms of
//   A = ((f0 - f0_s) + fdot_m (t_s - t_ref)) / df_s,  B = df / df_s,
// evaluated in FP64 with round-to-nearest operations in that order (no
// fused multiply-add), then scaled by 2^32 and rounded half to even.
//
// The sum is a gather of contiguous runs (consecutive j read consecutive i
// when df = df_s): HBM-bound, one read of each segment's 2F and one write.
#include "fstat_internal.cuh"

namespace fs {
namespace {

constexpr int kSlideBlock = 256;

__global__ void slide_prep_kernel(const SlideSeg* __restrict__ seg, int n_seg, const double* __restrict__ fdot,
                                  int n_fdot, double f0, double df, double t_ref, long long* __restrict__ A_fx,
                                  long long* __restrict__ B_fx) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_seg * n_fdot) return;
    const int s = t / n_fdot, m = t - s * n_fdot;
    const SlideSeg g = seg[s];
    const double d1 = __dsub_rn(f0, g.f0);
    const double d2 = __dsub_rn(g.t, t_ref);
    const double A = __ddiv_rn(__dadd_rn(d1, __dmul_rn(fdot[m], d2)), g.df);
    A_fx[t] = __double2ll_rn(__dmul_rn(A, 4294967296.0));
    if (m == 0) B_fx[s] = __double2ll_rn(__dmul_rn(__ddiv_rn(df, g.df), 4294967296.0));
}

// A block is one sky point (blockIdx.x) and one chunk of kJ * kSlideBlock
// frequencies (blockIdx.y) over all spindowns; each thread sums kJ
// frequencies j0 + q * kSlideBlock of each (sky, fdot) row in turn.  The
// segment table and every segment's slide constants sit in shared memory.
// All kJ x 4 loads of four segments are issued before their additions, which
// stay in segment order.  n_outside may be null (no counting).
constexpr int kJ = 4;

// UNIT: every segment has df_s = df (B = 1 exactly), so the index is j plus a
// per-(segment, fdot) integer offset floor(A + 1/2), clamped to +-2^30 (past
// that every lookup is outside the band anyway; n_f < 2^30).
template <bool UNIT>
__global__ void __launch_bounds__(kSlideBlock, 6) stackslide_kernel(const SlideSeg* __restrict__ seg, int n_seg,
                                                                    const long long* __restrict__ A_fx,
                                                                    const long long* __restrict__ B_fx, int n_fdot,
                                                                    int n_f, float* __restrict__ out,
                                                                    unsigned long long* __restrict__ n_outside) {
    // [n_seg] SlideSeg, [n_seg] B, [n_seg][n_fdot] A (+ 2^31; for UNIT its integer part)
    extern __shared__ __align__(16) unsigned char slide_smem[];
    SlideSeg* sg = reinterpret_cast<SlideSeg*>(slide_smem);
    long long* sB = reinterpret_cast<long long*>(sg + n_seg);
    long long* sA = sB + n_seg;
    for (int s = threadIdx.x; s < n_seg; s += blockDim.x) {
        sg[s] = seg[s];
        sB[s] = B_fx[s];
    }
    for (int t = threadIdx.x; t < n_seg * n_fdot; t += blockDim.x) {
        const long long a = A_fx[t] + (1LL << 31);
        sA[t] = UNIT ? max(-(1LL << 30), min(1LL << 30, a >> 32)) : a;
    }
    __syncthreads();
    const int j0 = (int)blockIdx.y * (kJ * kSlideBlock) + threadIdx.x;
    unsigned int outside = 0;
    for (int m = 0; m < n_fdot; ++m) {
        const long long row = (long long)blockIdx.x * n_fdot + m;
        float acc[kJ];
#pragma unroll
        for (int q = 0; q < kJ; ++q) acc[q] = 0.f;
        for (int s = 0; s < n_seg; s += 4) {
            float v[4][kJ];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const bool seg_ok = s + u < n_seg;
                const int su = seg_ok ? s + u : s;
                const long long nf = sg[su].n_f;
                const float* base = sg[su].twoF + row * nf;
                const long long a = sA[su * n_fdot + m], b = sB[su];
#pragma unroll
                for (int q = 0; q < kJ; ++q) {
                    const int j = j0 + q * kSlideBlock;
                    bool ok;
                    long long i;
                    const bool live = seg_ok && j < n_f;
                    if (UNIT) {
                        const int i32 = j + (int)a;
                        ok = live && (unsigned int)i32 < (unsigned int)nf;
                        i = i32;
                    } else {
                        i = (a + (long long)j * b) >> 32;
                        ok = live && i >= 0 && i < nf;
                    }
                    outside += live && !ok;
                    v[u][q] = ok ? __ldg(base + i) : 0.f;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int q = 0; q < kJ; ++q) acc[q] = __fadd_rn(acc[q], v[u][q]);
        }
#pragma unroll
        for (int q = 0; q < kJ; ++q) {
            const int j = j0 + q * kSlideBlock;
            if (j < n_f) out[row * n_f + j] = acc[q];
        }
    }
    if (n_outside) {
        for (int o = 16; o > 0; o >>= 1) outside += __shfl_xor_sync(0xffffffffu, outside, o);
        if ((threadIdx.x & 31) == 0 && outside) atomicAdd(n_outside, (unsigned long long)outside);
    }
}

}  // namespace

cudaError_t launch_stackslide(const SlideSeg* seg, int n_seg, const double* fdot, int n_fdot, double f0, double df,
                              double t_ref, long long* A_fx, long long* B_fx, bool prep, bool unit, long long n_rows,
                              int n_f, float* out, unsigned long long* n_outside, cudaStream_t s) {
    if (prep) {
        const int n_prep = n_seg * n_fdot;
        slide_prep_kernel<<<(n_prep + 127) / 128, 128, 0, s>>>(seg, n_seg, fdot, n_fdot, f0, df, t_ref, A_fx, B_fx);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    const long long n_sky = n_rows / n_fdot;
    if (n_sky > 0x7fffffffLL || (n_f + kJ * kSlideBlock - 1) / (kJ * kSlideBlock) > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)n_sky, (unsigned)((n_f + kJ * kSlideBlock - 1) / (kJ * kSlideBlock)));
    const size_t smem = (size_t)n_seg * (sizeof(SlideSeg) + sizeof(long long) * (1 + n_fdot));
    auto fn = unit && n_f < (1 << 30) ? stackslide_kernel<true> : stackslide_kernel<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    fn<<<grid, kSlideBlock, smem, s>>>(seg, n_seg, A_fx, B_fx, n_fdot, n_f, out, n_outside);
    return cudaGetLastError();
}

}  // namespace fs
