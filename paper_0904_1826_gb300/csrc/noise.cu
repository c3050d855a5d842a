// Noise-floor normalisation and per-SFT noise weights: the step before the
// F-statistic path for coloured, non-stationary noise (the paper's client
// assumes white SFTs; the weighted multi-detector sum is the reading of
// Listing 1's per-detector sum and normalized(result) used here).
//
//   P_k   = Re^2 + Im^2 in FP32 (squares rounded, then the sum rounded)
//   S(k)  = median{P_j : |j - k| <= W, j stored} / ln 2, FP32, computed as
//           (m1 + m2) * 0.5 / ln 2 with m1, m2 the two middle values (equal
//           for an odd count; the window is clipped at the band edges)
//   X'_k  = X_k / sqrt(S(k))   (0 where S(k) = 0)
//   w     = (1 / Sbar) / mean over SFTs of (1 / Sbar), Sbar = mean_k S(k)
//           (0 where Sbar = 0, left out of the mean), FP64
//
// The median is selected by stable rank counting over the window, which
// picks exactly the elements a sort would, so S matches an FP32 reference
// bit for bit.
#include "fstat_internal.cuh"

namespace fs {
namespace {

constexpr float kLn2f = 0.69314718055994530942f;
constexpr int kNoiseBlock = 256;

// One block per SFT: powers into shared memory, then per bin the running
// median, the whitened bin, and the SFT's mean floor.
__global__ void __launch_bounds__(kNoiseBlock) noise_floor_kernel(const float2* __restrict__ bins, long long row,
                                                                 int n_bins, int half, float* __restrict__ floor,
                                                                 float2* __restrict__ white,
                                                                 double* __restrict__ sbar) {
    extern __shared__ float pw[];   // [n_bins]
    __shared__ double red[kNoiseBlock / 32];
    const int s = blockIdx.x;
    const float2* x = bins + (size_t)s * row;
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
        const float2 v = x[k];
        pw[k] = __fadd_rn(__fmul_rn(v.x, v.x), __fmul_rn(v.y, v.y));
    }
    __syncthreads();
    double acc = 0.0;
    for (int k = threadIdx.x; k < n_bins; k += blockDim.x) {
        const int lo = max(0, k - half), hi = min(n_bins - 1, k + half);
        const int n = hi - lo + 1;
        const int r1 = (n - 1) >> 1, r2 = n >> 1;   // equal for an odd count
        const int need = (r1 == r2) ? 1 : 2;
        float m1 = 0.f, m2 = 0.f;
        int found = 0;
        for (int i = lo; i <= hi && found < need; ++i) {
            const float vi = pw[i];
            int rank = 0;   // stable rank: smaller values, then equal values further left
            for (int j = lo; j <= hi; ++j) {
                const float vj = pw[j];
                rank += (vj < vi) || (vj == vi && j < i);
            }
            if (rank == r1) {
                m1 = vi;
                ++found;
            } else if (rank == r2) {
                m2 = vi;
                ++found;
            }
        }
        if (need == 1) m2 = m1;
        const float S = __fdiv_rn(__fmul_rn(__fadd_rn(m1, m2), 0.5f), kLn2f);
        floor[(size_t)s * n_bins + k] = S;
        acc += (double)S;
        const float2 v = x[k];
        float2 o = make_float2(0.f, 0.f);
        if (S > 0.f) {
            const float inv = __fdiv_rn(1.0f, __fsqrt_rn(S));
            o = make_float2(v.x * inv, v.y * inv);
        }
        white[(size_t)s * row + k] = o;
    }
    for (long long k = n_bins + threadIdx.x; k < row; k += blockDim.x) white[(size_t)s * row + k] = make_float2(0.f, 0.f);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kNoiseBlock / 32; ++w) t += red[w];
        sbar[s] = t / (double)n_bins;
    }
}

// Weights from the mean floors of all SFTs (one block).
__global__ void __launch_bounds__(kNoiseBlock) noise_weight_kernel(const double* __restrict__ sbar, int n_sft,
                                                                  double* __restrict__ weight) {
    __shared__ double rs[kNoiseBlock / 32];
    __shared__ int rc[kNoiseBlock / 32];
    double sum = 0.0;
    int cnt = 0;
    for (int i = threadIdx.x; i < n_sft; i += blockDim.x)
        if (sbar[i] > 0.0) {
            sum += 1.0 / sbar[i];
            ++cnt;
        }
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xffffffffu, sum, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        rs[threadIdx.x >> 5] = sum;
        rc[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    __shared__ double mean;
    if (threadIdx.x == 0) {
        double t = 0.0;
        int c = 0;
        for (int w = 0; w < kNoiseBlock / 32; ++w) {
            t += rs[w];
            c += rc[w];
        }
        mean = c > 0 ? t / (double)c : 1.0;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n_sft; i += blockDim.x) weight[i] = sbar[i] > 0.0 ? (1.0 / sbar[i]) / mean : 0.0;
}

}  // namespace

cudaError_t launch_noise_floor(const float2* bins, long long row, int n_sft, int n_bins, int half, float* floor,
                               float2* white, double* sbar, double* weight, cudaStream_t s) {
    const size_t smem = (size_t)n_bins * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(noise_floor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    noise_floor_kernel<<<n_sft, kNoiseBlock, smem, s>>>(bins, row, n_bins, half, floor, white, sbar);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    noise_weight_kernel<<<1, kNoiseBlock, 0, s>>>(sbar, n_sft, weight);
    return cudaGetLastError();
}

}  // namespace fs
