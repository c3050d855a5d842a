// Patch-scoring network of the learned-proposal search: BF16 matrix products
// on the tcgen05 tensor cores (FP32 accumulation in tensor memory) for the two
// hidden layers forward and backward, FP32 output layer, loss and Adam.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/fstat_mlp.h"
#include "fstat_internal.cuh"

using bf16 = __nv_bfloat16;

namespace fs {
namespace {

enum { EPI_F32 = 0, EPI_RELU = 1, EPI_MASK = 2 };

// ---- matrix products on the tcgen05 tensor cores ----------------------------
// C(m, n) = sum_k A(m, k) B(k, n) (+ bias(n)), A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n]; K, lda, ldb multiples of 8.
// EPI_F32: Cf = C.  EPI_RELU: Cf = C (pre-activation), Cb = bf16(max(C, 0)).
// EPI_MASK: C *= (zref > 0); Cf = C, Cb = bf16(C).
// One CTA (4 warps) computes a TC_M x TC_N tile of C over the K range of its
// chunk (blockIdx.z).  Per TC_K-wide slice of K the threads stage A (TC_M x TC_K)
// and B (TC_N x TC_K, i.e. B^T) into shared memory in the K-major core-matrix
// layout without swizzle: a core matrix is 8 rows x 8 elements (8 x 16 bytes,
// rows 16 bytes apart), and the core matrix of rows 8i.. and columns 8j.. of
// an R-row tile sits at byte (j * R / 8 + i) * 128.  One thread then issues
// TC_K / 16 MMAs of kind::f16 (BF16 A and B, FP32 D, M = 128, N = 64, K = 16)
// on shared-memory descriptors (leading-dimension step: the next 8 columns,
// R * 16 bytes; stride step: the next 8 rows, 128 bytes) into a TMEM
// accumulator of 64 columns and commits them to the stage's mbarrier.  Two
// stages: the threads stage slice k + 1 while the tensor core runs slice k,
// and wait (bounded) for slice k - 1's MMAs before reusing its stage.  The
// epilogue reads the tile back with tcgen05.ld (warp w owns TMEM lanes, i.e.
// rows, 32w .. 32w + 31); with several K chunks it writes the raw FP32 tile of
// its chunk to part[z][M][N] and splitk_epi_kernel finishes the sum.
constexpr int TC_M = 128, TC_N = 64, TC_K = 64;
constexpr int TC_A_BYTES = TC_M * TC_K * 2, TC_B_BYTES = TC_N * TC_K * 2;
constexpr int TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr int TC_SMEM = 2 * TC_STAGE_BYTES + 32;   // two stages, two mbarriers, the TMEM address
// instruction descriptor: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
// both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t TC_IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

// Shared-memory matrix descriptor: start address >> 4 (bits 0-13), leading-
// dimension byte offset >> 4 (16-29), stride-dimension byte offset >> 4
// (32-45), the fixed value 1 at bits 46-48, no swizzle (bits 61-63 = 0).
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Byte offset of element (r, k) of an R-row tile in the core-matrix layout.
__device__ __forceinline__ uint32_t tc_off(int R, int r, int k) {
    return (uint32_t)((((k >> 3) * (R >> 3) + (r >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

// Bounded wait (about two seconds) for the phase of parity `parity`; every
// thread of the block takes the same decision.
__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t parity) {
    uint32_t done = 0;
    unsigned long long t0 = 0;
    for (unsigned int it = 0;; ++it) {
        asm volatile(
            "{\n"
            " .reg .pred p;\n"
            " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
            " selp.u32 %0, 1, 0, p;\n"
            "}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) break;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (it == 0) t0 = t;
        else if (t - t0 > 2000000000ull) break;
    }
    return __syncthreads_and(done != 0) != 0;
}

template <bool TA, bool TB>
__device__ __forceinline__ void tc_stage(unsigned char* As, unsigned char* Bs, int M, int N, int K, const bf16* A,
                                         int lda, const bf16* B, int ldb, int m0, int n0, int k0, int kend) {
    const int tid = threadIdx.x;
    const bf16 zero = __float2bfloat16(0.f);
    // A slice: TC_M rows x TC_K columns (K-major in shared memory)
    for (int v = tid; v < TC_M * TC_K / 8; v += 128) {
        if (!TA) {   // 8 consecutive k of one row
            const int r = v / (TC_K / 8), kk = (v % (TC_K / 8)) * 8;
            const int gm = m0 + r, gk = k0 + kk;
            uint4 q = make_uint4(0, 0, 0, 0);
            if (gm < M && gk < kend) q = *reinterpret_cast<const uint4*>(A + (size_t)gm * lda + gk);
            *reinterpret_cast<uint4*>(As + tc_off(TC_M, r, kk)) = q;
        } else {     // 8 consecutive rows of one k
            const int kk = v / (TC_M / 8), r = (v % (TC_M / 8)) * 8;
            const int gm = m0 + r, gk = k0 + kk;
            bf16 e[8];
            if (gk < kend && gm + 7 < M) {
                *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(A + (size_t)gk * lda + gm);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) e[i] = (gk < kend && gm + i < M) ? A[(size_t)gk * lda + gm + i] : zero;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) *reinterpret_cast<bf16*>(As + tc_off(TC_M, r + i, kk)) = e[i];
        }
    }
    // B slice as B^T: TC_N rows (n) x TC_K columns (k)
    for (int v = tid; v < TC_N * TC_K / 8; v += 128) {
        if (TB) {    // 8 consecutive k of one n
            const int r = v / (TC_K / 8), kk = (v % (TC_K / 8)) * 8;
            const int gn = n0 + r, gk = k0 + kk;
            uint4 q = make_uint4(0, 0, 0, 0);
            if (gn < N && gk < kend) q = *reinterpret_cast<const uint4*>(B + (size_t)gn * ldb + gk);
            *reinterpret_cast<uint4*>(Bs + tc_off(TC_N, r, kk)) = q;
        } else {     // 8 consecutive n of one k
            const int kk = v / (TC_N / 8), r = (v % (TC_N / 8)) * 8;
            const int gn = n0 + r, gk = k0 + kk;
            bf16 e[8];
            if (gk < kend && gn + 7 < N) {
                *reinterpret_cast<uint4*>(e) = *reinterpret_cast<const uint4*>(B + (size_t)gk * ldb + gn);
            } else {
#pragma unroll
                for (int i = 0; i < 8; ++i) e[i] = (gk < kend && gn + i < N) ? B[(size_t)gk * ldb + gn + i] : zero;
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) *reinterpret_cast<bf16*>(Bs + tc_off(TC_N, r + i, kk)) = e[i];
        }
    }
}

template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(128) gemm_tc_kernel(int M, int N, int K, const bf16* __restrict__ A, int lda,
                                                      const bf16* __restrict__ B, int ldb,
                                                      const float* __restrict__ bias, float* __restrict__ Cf,
                                                      bf16* __restrict__ Cb, const float* __restrict__ zref, int ldc,
                                                      float* __restrict__ part, int kchunk, int* __restrict__ flag) {
    extern __shared__ __align__(128) unsigned char tsm[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(tsm + 2 * TC_STAGE_BYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(tsm + 2 * TC_STAGE_BYTES + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_M, n0 = blockIdx.x * TC_N;
    const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
    const int n_sl = (ke - kb + TC_K - 1) / TC_K;   // >= 1 (the host makes every chunk non-empty)
    const uint32_t bar0 = tc_smem_u32(bars);
    if (warp == 0) {   // the whole warp allocates the 64 accumulator columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 64;" ::"r"(tc_smem_u32(tslot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    uint32_t ph0 = 0, ph1 = 0;   // parity of the next wait on each stage's barrier
    bool ok = true;
    int it = 0;
    for (; it < n_sl; ++it) {
        const int st = it & 1;
        if (it >= 2) {   // the MMAs of slice it - 2 read this stage
            ok = tc_wait(bar0 + 8 * st, st ? ph1 : ph0);
            if (st) ph1 ^= 1u; else ph0 ^= 1u;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        }
        unsigned char* As = tsm + st * TC_STAGE_BYTES;
        unsigned char* Bs = As + TC_A_BYTES;
        tc_stage<TA, TB>(As, Bs, M, N, K, A, lda, B, ldb, m0, n0, kb + it * TC_K, ke);
        // the tensor core reads shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a_base = tc_smem_u32(As), b_base = tc_smem_u32(Bs);
#pragma unroll
            for (int s = 0; s < TC_K / 16; ++s) {
                const uint64_t ad = tc_desc(a_base + (uint32_t)(2 * s * (TC_M / 8) * 128), (TC_M / 8) * 128, 128);
                const uint64_t bd = tc_desc(b_base + (uint32_t)(2 * s * (TC_N / 8) * 128), (TC_N / 8) * 128, 128);
                const uint32_t acc = (it > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n"
                    " .reg .pred p;\n"
                    " setp.ne.u32 p, %4, 0;\n"
                    " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
                    "}\n" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             bar0 + 8 * st)
                         : "memory");
        }
    }
    // drain: the commits of the last two slices
    if (ok) {
        for (int j = max(0, n_sl - 2); j < n_sl && ok; ++j) {
            const int st = j & 1;
            ok = tc_wait(bar0 + 8 * st, st ? ph1 : ph0);
            if (st) ph1 ^= 1u; else ph0 ^= 1u;
        }
    }
    if (!ok && tid == 0) atomicOr(flag, 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        const int row = m0 + warp * 32 + lane;
        float* pz = part ? part + (size_t)blockIdx.z * M * N : nullptr;
#pragma unroll 1
        for (int c0 = 0; c0 < TC_N; c0 += 16) {
            uint32_t v[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col >= N) continue;
                    float x = __uint_as_float(v[j]);
                    if (pz) {   // one K chunk of several: raw partial sum
                        pz[(size_t)row * N + col] = x;
                        continue;
                    }
                    if (bias) x += bias[col];
                    const size_t o = (size_t)row * ldc + col;
                    if (EPI == EPI_F32) {
                        Cf[o] = x;
                    } else if (EPI == EPI_RELU) {
                        Cf[o] = x;
                        Cb[o] = __float2bfloat16_rn(fmaxf(x, 0.f));
                    } else {
                        x = zref[o] > 0.f ? x : 0.f;
                        Cf[o] = x;
                        Cb[o] = __float2bfloat16_rn(x);
                    }
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 64;" ::"r"(tmem) : "memory");
    }
    if (ok && tid == 0) {
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(bar0 + 8) : "memory");
    }
}

// Sum of the K chunks' partial tiles in chunk order, then the epilogue.
template <int EPI>
__global__ void splitk_epi_kernel(int M, int N, int splits, const float* __restrict__ part,
                                  const float* __restrict__ bias, float* __restrict__ Cf, bf16* __restrict__ Cb,
                                  const float* __restrict__ zref, int ldc) {
    const long long MN = (long long)M * N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < MN; i += (long long)gridDim.x * blockDim.x) {
        float x = part[i];
        for (int z = 1; z < splits; ++z) x += part[z * MN + i];
        const int row = (int)(i / N), col = (int)(i - (long long)row * N);
        if (bias) x += bias[col];
        const size_t o = (size_t)row * ldc + col;
        if (EPI == EPI_F32) {
            Cf[o] = x;
        } else if (EPI == EPI_RELU) {
            Cf[o] = x;
            Cb[o] = __float2bfloat16_rn(fmaxf(x, 0.f));
        } else {
            x = zref[o] > 0.f ? x : 0.f;
            Cf[o] = x;
            Cb[o] = __float2bfloat16_rn(x);
        }
    }
}

// Output layer and loss, one warp per row: s = relu(z2) . w3 + b3;
// l = w (softplus(s) - y s), ds = w (sigmoid(s) - y) / B.
__global__ void head_kernel(const float* __restrict__ z2, const float* __restrict__ w3, const float* __restrict__ b3,
                            int B, int H, const float* __restrict__ y, float pos_weight, float* __restrict__ s,
                            float* __restrict__ ds, float* __restrict__ lrow) {
    const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (row >= B) return;
    float acc = 0.f;
    for (int n = lane; n < H; n += 32) acc = fmaf(fmaxf(z2[(size_t)row * H + n], 0.f), w3[n], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
        const float v = acc + b3[0];
        s[row] = v;
        if (y) {
            const float yy = y[row];
            const float w = yy > 0.5f ? pos_weight : 1.0f;
            const float sp = fmaxf(v, 0.f) + log1pf(expf(-fabsf(v)));
            lrow[row] = w * (sp - yy * v);
            ds[row] = w * (1.f / (1.f + expf(-v)) - yy) / (float)B;
        }
    }
}

// Deterministic sum of n values by one block.
__global__ void sum_kernel(const float* __restrict__ v, int n, float* __restrict__ out, float scale) {
    __shared__ float red[256];
    float a = 0.f;
    for (int i = threadIdx.x; i < n; i += 256) a += v[i];
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0] * scale;
}

// Layer-3 backward: dw3[n] = sum_b relu(z2) ds, dz2 = ds w3 (z2 > 0) (FP32 and BF16).
__global__ void head_back_kernel(const float* __restrict__ z2, const float* __restrict__ w3,
                                 const float* __restrict__ ds, int B, int H, float* __restrict__ dw3,
                                 float* __restrict__ dz2, bf16* __restrict__ dz2b) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= H) return;
    float a = 0.f;
    for (int b = 0; b < B; ++b) {
        const float z = z2[(size_t)b * H + n];
        a = fmaf(fmaxf(z, 0.f), ds[b], a);
        const float d = z > 0.f ? ds[b] * w3[n] : 0.f;
        dz2[(size_t)b * H + n] = d;
        dz2b[(size_t)b * H + n] = __float2bfloat16_rn(d);
    }
    dw3[n] = a;
}

// Column sums (bias gradients) of a [B][H] FP32 array.
__global__ void colsum_kernel(const float* __restrict__ v, int B, int H, float* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= H) return;
    float a = 0.f;
    for (int b = 0; b < B; ++b) a += v[(size_t)b * H + n];
    out[n] = a;
}

__global__ void adam_kernel(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ gr, long long n, float lr, float c1, float c2,
                            bf16* __restrict__ pb) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float gi = gr[i];
        const float mi = 0.9f * m[i] + 0.1f * gi;
        const float vi = 0.999f * v[i] + 0.001f * gi * gi;
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi * c1) / (sqrtf(vi * c2) + 1e-8f);
        p[i] = pi;
        if (pb) pb[i] = __float2bfloat16_rn(pi);
    }
}

__global__ void to_bf16_kernel(const float* __restrict__ x, long long n, bf16* __restrict__ y) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        y[i] = __float2bfloat16_rn(x[i]);
}

__global__ void patch_kernel(const float* __restrict__ twoF, int n_f, int n_d, int s_a, int s_d, int n_fp,
                             const int* __restrict__ f_start, int n_q, int n_pd, float shift, float scale,
                             bf16* __restrict__ out) {
    const int p = blockIdx.x;
    const int pa = p / (n_pd * n_q);
    const int r = p - pa * n_pd * n_q;
    const int pd = r / n_q, q = r - pd * n_q;
    const int row = s_a * s_d * n_fp;
    const int f0 = f_start[q];
    for (int e = threadIdx.x; e < row; e += blockDim.x) {
        const int fl = e % n_fp;
        const int sl = e / n_fp;
        const int ia = pa * s_a + sl / s_d, id = pd * s_d + sl % s_d;
        const float v = twoF[(size_t)(ia * n_d + id) * n_f + f0 + fl];
        out[(size_t)p * row + e] = __float2bfloat16_rn(fmaxf(v - shift, 0.f) * scale);
    }
}

// Windows at arbitrary origins (a0, d0, f0): alpha wraps around the grid, the
// other two stay inside it (checked by the caller).
__global__ void window_kernel(const float* __restrict__ twoF, int n_f, int n_a, int n_d, int s_a, int s_d, int n_fp,
                              const int* __restrict__ origin, float shift, float scale, bf16* __restrict__ out) {
    const int w = blockIdx.x;
    const int a0 = origin[3 * w], d0 = origin[3 * w + 1], f0 = origin[3 * w + 2];
    const int row = s_a * s_d * n_fp;
    for (int e = threadIdx.x; e < row; e += blockDim.x) {
        const int fl = e % n_fp;
        const int sl = e / n_fp;
        int ia = a0 + sl / s_d;
        if (ia >= n_a) ia -= n_a;
        const int id = d0 + sl % s_d;
        const float v = twoF[(size_t)(ia * n_d + id) * n_f + f0 + fl];
        out[(size_t)w * row + e] = __float2bfloat16_rn(fmaxf(v - shift, 0.f) * scale);
    }
}

// Device scratch of the products: the give-up flag and the K-chunk partial
// tiles (capacity `cap` floats).
struct TcWork {
    int* flag = nullptr;
    float* part = nullptr;
    size_t cap = 0;
};

// Tiles of the tcgen05 form; a product with few tiles splits K into chunks
// (at least 4 slices each) so that about two CTAs per SM run, and sums them
// in chunk order.
template <bool TA, bool TB, int EPI>
cudaError_t gemm(int M, int N, int K, const bf16* A, int lda, const bf16* B, int ldb, const float* bias, float* Cf,
                 bf16* Cb, const float* zref, int ldc, cudaStream_t s, const TcWork& w) {
    float* part = w.part;
    int* flag = w.flag;
    const size_t cap = w.cap;
    auto fn = gemm_tc_kernel<TA, TB, EPI>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    if (e != cudaSuccess) return e;
    const int tiles = ((N + TC_N - 1) / TC_N) * ((M + TC_M - 1) / TC_M);
    const int n_sl = (K + TC_K - 1) / TC_K;
    int splits = std::min((2 * current_sm_count() + tiles - 1) / tiles, std::max(1, n_sl / 4));
    while (splits > 1 && (size_t)splits * M * N > cap) --splits;
    const int kchunk = ((n_sl + splits - 1) / splits) * TC_K;
    splits = (K + kchunk - 1) / kchunk;   // every chunk non-empty
    dim3 grid((N + TC_N - 1) / TC_N, (M + TC_M - 1) / TC_M, splits);
    fn<<<grid, 128, TC_SMEM, s>>>(M, N, K, A, lda, B, ldb, bias, Cf, Cb, zref, ldc, splits > 1 ? part : nullptr,
                                  kchunk, flag);
    if (splits > 1) {
        const long long MN = (long long)M * N;
        const int g = (int)std::min<long long>((MN + 255) / 256, 4LL * current_sm_count());
        splitk_epi_kernel<EPI><<<g, 256, 0, s>>>(M, N, splits, part, bias, Cf, Cb, zref, ldc);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_patches(const float* twoF, int n_f, int n_d, int s_a, int s_d, int n_fp, const int* f_start_dev,
                           int n_q, int n_patches, int n_pd, float shift, float scale, void* out, cudaStream_t s) {
    patch_kernel<<<n_patches, 256, 0, s>>>(twoF, n_f, n_d, s_a, s_d, n_fp, f_start_dev, n_q, n_pd, shift, scale,
                                           reinterpret_cast<bf16*>(out));
    return cudaGetLastError();
}

cudaError_t launch_windows(const float* twoF, int n_f, int n_a, int n_d, int s_a, int s_d, int n_fp,
                           const int* origin_dev, int n_w, float shift, float scale, void* out, cudaStream_t s) {
    window_kernel<<<n_w, 256, 0, s>>>(twoF, n_f, n_a, n_d, s_a, s_d, n_fp, origin_dev, shift, scale,
                                      reinterpret_cast<bf16*>(out));
    return cudaGetLastError();
}

}  // namespace fs

using namespace fs;

struct fstat_mlp {
    int device = 0;
    int n_in = 0, H = 0, maxB = 0;
    std::string err;
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
    bf16 *W1b = nullptr, *W2b = nullptr;
    float* mom[12] = {};    // m, v per parameter
    float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr, *gw3 = nullptr, *gb3 = nullptr;
    bf16* Xb = nullptr;
    float *y = nullptr, *z1 = nullptr, *z2 = nullptr, *s = nullptr, *ds = nullptr, *lrow = nullptr, *loss = nullptr;
    bf16 *h1 = nullptr, *h2 = nullptr;
    float *dz2 = nullptr, *dz1 = nullptr;
    bf16 *dz2b = nullptr, *dz1b = nullptr;
    int t = 0;
    TcWork tcw;                 // flag (bit 0: a tensor-core wait gave up) and K-chunk partial products
    cudaStream_t stream = nullptr;
    std::vector<void*> allocs;
};

namespace {

int mfail(fstat_mlp* m, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (m) m->err = buf;
    return code;
}

#define MLP_TRY(m, call)                                                                              \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) return mfail(m, FSTAT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <class T>
int alloc(fstat_mlp* m, T** p, size_t n) {
    if (cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess)
        return mfail(m, FSTAT_ENOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
    m->allocs.push_back((void*)*p);
    return cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T)) == cudaSuccess ? FSTAT_OK : FSTAT_ECUDA;
}

// After a synchronisation: a tensor-core completion wait that gave up makes
// the call fail (its products were not written).
int check_flag(fstat_mlp* m) {
    int f = 0;
    MLP_TRY(m, cudaMemcpy(&f, m->tcw.flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (f) return mfail(m, FSTAT_ECUDA, "a tensor-core completion wait gave up (flag %d)", f);
    return FSTAT_OK;
}

// Stage X (host or device) into the network's BF16 input buffer.
int stage_input(fstat_mlp* m, const uint16_t* X, int B, int mem, cudaStream_t s, const bf16** Xd) {
    if (mem == FSTAT_MEM_DEVICE) {
        *Xd = reinterpret_cast<const bf16*>(X);
        return FSTAT_OK;
    }
    MLP_TRY(m, cudaMemcpyAsync(m->Xb, X, (size_t)B * m->n_in * sizeof(uint16_t), cudaMemcpyHostToDevice, s));
    *Xd = m->Xb;
    return FSTAT_OK;
}

int run_forward(fstat_mlp* m, const bf16* X, int B, cudaStream_t s) {
    const int n_in = m->n_in, H = m->H;
    MLP_TRY(m, (gemm<false, false, EPI_RELU>(B, H, n_in, X, n_in, m->W1b, H, m->b1, m->z1, m->h1,
                                             nullptr, H, s, m->tcw)));
    MLP_TRY(m, (gemm<false, false, EPI_RELU>(B, H, H, m->h1, H, m->W2b, H, m->b2, m->z2, m->h2,
                                             nullptr, H, s, m->tcw)));
    return FSTAT_OK;
}

}  // namespace

extern "C" {

int fstat_mlp_create(fstat_mlp** out, int device, int32_t n_in, int32_t n_hidden, int32_t max_batch) {
    if (!out) return FSTAT_EINVAL;
    *out = nullptr;
    if (n_in < 8 || n_in % 8 || n_hidden < 8 || n_hidden % 8 || max_batch < 1 || max_batch > 65536) return FSTAT_EINVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return FSTAT_ECUDA;
    if (cudaSetDevice(device) != cudaSuccess) return FSTAT_ECUDA;
    fstat_mlp* m = new fstat_mlp();
    m->device = device;
    m->n_in = n_in;
    m->H = n_hidden;
    m->maxB = (max_batch + 7) & ~7;
    const size_t H = n_hidden, I = n_in, Bm = m->maxB;
    int rc = FSTAT_OK;
    const size_t sizes[6] = {I * H, H, H * H, H, H, 1};
    float** params[6] = {&m->W1, &m->b1, &m->W2, &m->b2, &m->w3, &m->b3};
    float** grads[6] = {&m->gW1, &m->gb1, &m->gW2, &m->gb2, &m->gw3, &m->gb3};
    for (int i = 0; i < 6 && rc == FSTAT_OK; ++i) {
        rc = alloc(m, params[i], sizes[i]);
        if (rc == FSTAT_OK) rc = alloc(m, grads[i], sizes[i]);
        if (rc == FSTAT_OK) rc = alloc(m, &m->mom[2 * i], sizes[i]);
        if (rc == FSTAT_OK) rc = alloc(m, &m->mom[2 * i + 1], sizes[i]);
    }
    if (rc == FSTAT_OK) rc = alloc(m, &m->W1b, I * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->W2b, H * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->Xb, Bm * I);
    if (rc == FSTAT_OK) rc = alloc(m, &m->y, Bm);
    if (rc == FSTAT_OK) rc = alloc(m, &m->z1, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->z2, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->h1, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->h2, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->s, Bm);
    if (rc == FSTAT_OK) rc = alloc(m, &m->ds, Bm);
    if (rc == FSTAT_OK) rc = alloc(m, &m->lrow, Bm);
    if (rc == FSTAT_OK) rc = alloc(m, &m->loss, 1);
    if (rc == FSTAT_OK) rc = alloc(m, &m->dz2, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->dz1, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->dz2b, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->dz1b, Bm * H);
    if (rc == FSTAT_OK) rc = alloc(m, &m->tcw.flag, 1);
    m->tcw.cap = 16 * std::max(Bm, H) * H;
    if (rc == FSTAT_OK) rc = alloc(m, &m->tcw.part, m->tcw.cap);
    if (rc != FSTAT_OK) {
        fstat_mlp_destroy(m);
        return rc;
    }
    *out = m;
    return FSTAT_OK;
}

void fstat_mlp_destroy(fstat_mlp* m) {
    if (!m) return;
    cudaSetDevice(m->device);
    cudaDeviceSynchronize();
    for (void* p : m->allocs) cudaFree(p);
    delete m;
}

const char* fstat_mlp_last_error(const fstat_mlp* m) { return m ? m->err.c_str() : ""; }

int fstat_mlp_set_params(fstat_mlp* m, const float* W1, const float* b1, const float* W2, const float* b2,
                         const float* w3, const float* b3) {
    if (!m || !W1 || !b1 || !W2 || !b2 || !w3 || !b3) return FSTAT_EINVAL;
    m->err.clear();
    MLP_TRY(m, cudaSetDevice(m->device));
    const size_t H = m->H, I = m->n_in;
    const float* src[6] = {W1, b1, W2, b2, w3, b3};
    float* dst[6] = {m->W1, m->b1, m->W2, m->b2, m->w3, m->b3};
    const size_t n[6] = {I * H, H, H * H, H, H, 1};
    for (int i = 0; i < 6; ++i) {
        for (size_t k = 0; k < n[i]; ++k)
            if (!std::isfinite(src[i][k])) return mfail(m, FSTAT_EINVAL, "non-finite parameter");
        MLP_TRY(m, cudaMemcpy(dst[i], src[i], n[i] * sizeof(float), cudaMemcpyHostToDevice));
        MLP_TRY(m, cudaMemset(m->mom[2 * i], 0, n[i] * sizeof(float)));
        MLP_TRY(m, cudaMemset(m->mom[2 * i + 1], 0, n[i] * sizeof(float)));
    }
    to_bf16_kernel<<<256, 256>>>(m->W1, (long long)(I * H), m->W1b);
    to_bf16_kernel<<<64, 256>>>(m->W2, (long long)(H * H), m->W2b);
    MLP_TRY(m, cudaGetLastError());
    MLP_TRY(m, cudaDeviceSynchronize());
    m->t = 0;
    return FSTAT_OK;
}

int fstat_mlp_get_params(fstat_mlp* m, float* W1, float* b1, float* W2, float* b2, float* w3, float* b3) {
    if (!m || !W1 || !b1 || !W2 || !b2 || !w3 || !b3) return FSTAT_EINVAL;
    MLP_TRY(m, cudaSetDevice(m->device));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    const size_t H = m->H, I = m->n_in;
    float* dst[6] = {W1, b1, W2, b2, w3, b3};
    const float* src[6] = {m->W1, m->b1, m->W2, m->b2, m->w3, m->b3};
    const size_t n[6] = {I * H, H, H * H, H, H, 1};
    for (int i = 0; i < 6; ++i) MLP_TRY(m, cudaMemcpy(dst[i], src[i], n[i] * sizeof(float), cudaMemcpyDeviceToHost));
    return FSTAT_OK;
}

int fstat_mlp_forward(fstat_mlp* m, const uint16_t* X, int32_t B, float* logits, int32_t mem, void* cuda_stream) {
    if (!m || !X || !logits) return FSTAT_EINVAL;
    m->err.clear();
    if (B < 1 || B > m->maxB) return mfail(m, FSTAT_EINVAL, "batch %d outside 1..%d", B, m->maxB);
    MLP_TRY(m, cudaSetDevice(m->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    m->stream = s;
    const bf16* Xd = nullptr;
    int rc = stage_input(m, X, B, mem, s, &Xd);
    if (rc != FSTAT_OK) return rc;
    if ((rc = run_forward(m, Xd, B, s)) != FSTAT_OK) return rc;
    head_kernel<<<(B + 7) / 8, 256, 0, s>>>(m->z2, m->w3, m->b3, B, m->H, nullptr, 1.f, m->s, nullptr, nullptr);
    MLP_TRY(m, cudaGetLastError());
    if (mem == FSTAT_MEM_DEVICE) {
        MLP_TRY(m, cudaMemcpyAsync(logits, m->s, B * sizeof(float), cudaMemcpyDeviceToDevice, s));
    } else {
        MLP_TRY(m, cudaMemcpyAsync(logits, m->s, B * sizeof(float), cudaMemcpyDeviceToHost, s));
        MLP_TRY(m, cudaStreamSynchronize(s));
        return check_flag(m);
    }
    return FSTAT_OK;
}

int fstat_mlp_train_step(fstat_mlp* m, const uint16_t* X, const float* y, int32_t B, float pos_weight, float lr,
                         float* loss, int32_t mem, void* cuda_stream) {
    if (!m || !X || !y) return FSTAT_EINVAL;
    m->err.clear();
    if (B < 8 || B > m->maxB || B % 8) return mfail(m, FSTAT_EINVAL, "training batch must be a multiple of 8 in 8..%d", m->maxB);
    if (!(lr > 0.f) || !(pos_weight > 0.f)) return mfail(m, FSTAT_EINVAL, "lr and pos_weight must be > 0");
    MLP_TRY(m, cudaSetDevice(m->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    m->stream = s;
    const int H = m->H, I = m->n_in;
    const bf16* Xd = nullptr;
    int rc = stage_input(m, X, B, mem, s, &Xd);
    if (rc != FSTAT_OK) return rc;
    MLP_TRY(m, cudaMemcpyAsync(m->y, y, B * sizeof(float),
                               mem == FSTAT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if ((rc = run_forward(m, Xd, B, s)) != FSTAT_OK) return rc;
    head_kernel<<<(B + 7) / 8, 256, 0, s>>>(m->z2, m->w3, m->b3, B, H, m->y, pos_weight, m->s, m->ds, m->lrow);
    sum_kernel<<<1, 256, 0, s>>>(m->lrow, B, m->loss, 1.f / (float)B);
    sum_kernel<<<1, 256, 0, s>>>(m->ds, B, m->gb3, 1.f);
    head_back_kernel<<<(H + 127) / 128, 128, 0, s>>>(m->z2, m->w3, m->ds, B, H, m->gw3, m->dz2, m->dz2b);
    colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(m->dz2, B, H, m->gb2);
    MLP_TRY(m, cudaGetLastError());
    // dW2 = h1^T dz2;  dz1 = (dz2 W2^T) * (z1 > 0);  dW1 = X^T dz1
    MLP_TRY(m, (gemm<true, false, EPI_F32>(H, H, B, m->h1, H, m->dz2b, H, nullptr, m->gW2, nullptr,
                                           nullptr, H, s, m->tcw)));
    MLP_TRY(m, (gemm<false, true, EPI_MASK>(B, H, H, m->dz2b, H, m->W2b, H, nullptr, m->dz1, m->dz1b,
                                            m->z1, H, s, m->tcw)));
    colsum_kernel<<<(H + 127) / 128, 128, 0, s>>>(m->dz1, B, H, m->gb1);
    MLP_TRY(m, (gemm<true, false, EPI_F32>(I, H, B, Xd, I, m->dz1b, H, nullptr, m->gW1, nullptr,
                                           nullptr, H, s, m->tcw)));
    // Adam
    m->t += 1;
    const float c1 = 1.f / (1.f - powf(0.9f, (float)m->t)), c2 = 1.f / (1.f - powf(0.999f, (float)m->t));
    float* P[6] = {m->W1, m->b1, m->W2, m->b2, m->w3, m->b3};
    float* Gr[6] = {m->gW1, m->gb1, m->gW2, m->gb2, m->gw3, m->gb3};
    bf16* Pb[6] = {m->W1b, nullptr, m->W2b, nullptr, nullptr, nullptr};
    const long long n[6] = {(long long)I * H, H, (long long)H * H, H, H, 1};
    for (int i = 0; i < 6; ++i)
        adam_kernel<<<(int)std::min<long long>(1024, (n[i] + 255) / 256), 256, 0, s>>>(P[i], m->mom[2 * i], m->mom[2 * i + 1],
                                                                                       Gr[i], n[i], lr, c1, c2, Pb[i]);
    MLP_TRY(m, cudaGetLastError());
    if (loss) {
        MLP_TRY(m, cudaMemcpyAsync(loss, m->loss, sizeof(float), cudaMemcpyDeviceToHost, s));
        MLP_TRY(m, cudaStreamSynchronize(s));
        return check_flag(m);
    }
    return FSTAT_OK;
}

int fstat_mlp_get_grads(fstat_mlp* m, float* dW1, float* db1, float* dW2, float* db2, float* dw3, float* db3) {
    if (!m || !dW1 || !db1 || !dW2 || !db2 || !dw3 || !db3) return FSTAT_EINVAL;
    MLP_TRY(m, cudaSetDevice(m->device));
    MLP_TRY(m, cudaStreamSynchronize(m->stream));
    const size_t H = m->H, I = m->n_in;
    float* dst[6] = {dW1, db1, dW2, db2, dw3, db3};
    const float* src[6] = {m->gW1, m->gb1, m->gW2, m->gb2, m->gw3, m->gb3};
    const size_t n[6] = {I * H, H, H * H, H, H, 1};
    for (int i = 0; i < 6; ++i) MLP_TRY(m, cudaMemcpy(dst[i], src[i], n[i] * sizeof(float), cudaMemcpyDeviceToHost));
    return check_flag(m);
}

}  // extern "C"
