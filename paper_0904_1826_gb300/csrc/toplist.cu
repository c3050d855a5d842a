// Toplist: the K largest 2F of a bank, ordered by (2F descending, template
// index ascending).  2F >= 0, so the FP32 bit patterns order like the values
// and a three-level radix select (11 + 11 + 10 bits) finds the exact K-th
// value tau with warp-aggregated shared-memory histograms.  Values above tau
// are gathered with an atomic slot counter (at most K - 1 of them); values
// equal to tau are taken in index order through per-block counts, so the
// result is deterministic.  A single block then sorts the K candidates.
#include "fstat_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <mutex>

#include "../../include/fstat_noalloc.h"

namespace fs {
namespace {

constexpr int kBins = 2048;
constexpr int kBlk = 256;

__device__ __forceinline__ void warp_hist_add(unsigned int* h, unsigned int bin, bool valid) {
    const unsigned int act = __ballot_sync(0xffffffffu, valid);
    if (!valid) return;
    const unsigned int peers = __match_any_sync(act, bin);
    const int leader = __ffs(peers) - 1;
    if ((int)(threadIdx.x & 31) == leader) atomicAdd(&h[bin], (unsigned int)__popc(peers));
}

// Ranking key of a value: its FP32 bit pattern, with -0.0 taken as +0.0 (for
// the non-negative values ranked here the patterns order like the values).
__device__ __forceinline__ unsigned int key_bits(float x) {
    const unsigned int b = __float_as_uint(x);
    return b == 0x80000000u ? 0u : b;
}

template <int LEVEL>
__device__ __forceinline__ void classify(unsigned int b, unsigned int prefix, unsigned int& bin, bool& ok) {
    if (LEVEL == 0) {
        bin = b >> 21;
        ok = true;
    } else if (LEVEL == 1) {
        bin = (b >> 10) & 2047u;
        ok = (b >> 21) == prefix;
    } else {
        bin = b & 1023u;
        ok = (b >> 10) == prefix;
    }
}

// v + head is 16-byte aligned (head < 4): the head, the float4 body and the
// tail of fewer than four values are histogrammed separately.
template <int LEVEL>
__global__ void __launch_bounds__(kBlk) hist_kernel(const float* __restrict__ v, long long n, int head,
                                                    const unsigned int* __restrict__ state,
                                                    unsigned int* __restrict__ hist) {
    __shared__ unsigned int h[kBins];
    for (int i = threadIdx.x; i < kBins; i += kBlk) h[i] = 0;
    __syncthreads();
    const unsigned int prefix = LEVEL == 0 ? 0u : state[0];
    const long long n4 = (n - head) >> 2;
    const float4* v4 = reinterpret_cast<const float4*>(v + head);
    const long long stride = (long long)gridDim.x * kBlk;
    // every thread of a warp runs the same number of iterations (ballot below)
    for (long long base = (long long)blockIdx.x * kBlk; base < n4; base += stride) {
        const long long i = base + threadIdx.x;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        const bool in = i < n4;
        if (in) x = __ldg(v4 + i);
        const float xs[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            unsigned int bin;
            bool ok;
            classify<LEVEL>(key_bits(xs[c]), prefix, bin, ok);
            warp_hist_add(h, bin, ok && in);
        }
    }
    // head (before the 16-byte boundary) and tail (after the last float4)
    if (blockIdx.x == 0 && threadIdx.x < 32) {
        const long long t = threadIdx.x;
        const long long n_tail = n - head - 4 * n4;
        long long i = -1;
        if (t < head) i = t;
        else if (t - head < n_tail) i = head + 4 * n4 + (t - head);
        const bool in = i >= 0;
        unsigned int bin = 0;
        bool ok = false;
        if (in) classify<LEVEL>(key_bits(v[i]), prefix, bin, ok);
        warp_hist_add(h, bin, ok && in);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kBins; i += kBlk)
        if (h[i]) atomicAdd(&hist[LEVEL * kBins + i], h[i]);
}

// state: [0] prefix of the bucket holding the K-th value, [1] rank still
// needed inside it, [2] threshold bits, [3] count above the threshold,
// [4] ties needed.
template <int LEVEL>
__global__ void select_kernel(const unsigned int* __restrict__ hist, unsigned int* __restrict__ state, unsigned int k) {
    if (threadIdx.x != 0) return;
    const unsigned int* h = hist + LEVEL * kBins;
    unsigned int need = LEVEL == 0 ? k : state[1];
    const int top = LEVEL == 2 ? 1023 : 2047;
    unsigned int above = 0;
    int b = top;
    for (; b > 0; --b) {
        if (above + h[b] >= need) break;
        above += h[b];
    }
    need -= above;
    if (LEVEL == 0) {
        state[0] = (unsigned int)b;
    } else if (LEVEL == 1) {
        state[0] = (state[0] << 11) | (unsigned int)b;
    } else {
        state[2] = (state[0] << 10) | (unsigned int)b;
        state[3] = k - need;
        state[4] = need;
    }
    state[1] = need;
}

__global__ void __launch_bounds__(kBlk) collect_kernel(const float* __restrict__ v, long long n, long long per_block,
                                                       const unsigned int* __restrict__ state,
                                                       long long* __restrict__ cand_idx, float* __restrict__ cand_val,
                                                       unsigned int* __restrict__ n_cand,
                                                       unsigned int* __restrict__ tie_count) {
    __shared__ unsigned int ties;
    if (threadIdx.x == 0) ties = 0;
    __syncthreads();
    const unsigned int tau = state[2];
    const long long lo = (long long)blockIdx.x * per_block;
    const long long hi = min(n, lo + per_block);
    unsigned int my_ties = 0;
    for (long long i = lo + threadIdx.x; i < hi; i += kBlk) {
        const float x = v[i];
        const unsigned int b = key_bits(x);
        if (b > tau) {
            const unsigned int s = atomicAdd(n_cand, 1u);
            cand_idx[s] = i;
            cand_val[s] = x;
        } else if (b == tau) {
            ++my_ties;
        }
    }
    for (int o = 16; o > 0; o >>= 1) my_ties += __shfl_xor_sync(0xffffffffu, my_ties, o);
    if ((threadIdx.x & 31) == 0 && my_ties) atomicAdd(&ties, my_ties);
    __syncthreads();
    if (threadIdx.x == 0) tie_count[blockIdx.x] = ties;
}

__global__ void __launch_bounds__(kBlk) tie_kernel(const float* __restrict__ v, long long n, long long per_block,
                                                   const unsigned int* __restrict__ state,
                                                   const unsigned int* __restrict__ tie_count,
                                                   long long* __restrict__ cand_idx, float* __restrict__ cand_val) {
    __shared__ unsigned int wsum[kBlk / 32];
    __shared__ unsigned int s_prefix;
    const unsigned int tau = state[2];
    const unsigned int n_gt = state[3];
    const unsigned int need = state[4];
    if (threadIdx.x == 0) {
        unsigned int pre = 0;
        for (unsigned int b = 0; b < blockIdx.x; ++b) pre += tie_count[b];
        s_prefix = pre;
    }
    __syncthreads();
    unsigned int prefix = s_prefix;
    if (prefix >= need || tie_count[blockIdx.x] == 0) return;
    const long long lo = (long long)blockIdx.x * per_block;
    const long long hi = min(n, lo + per_block);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    for (long long base = lo; base < hi && prefix < need; base += kBlk) {
        const long long i = base + threadIdx.x;
        const bool t = (i < hi) && (key_bits(v[i]) == tau);
        const unsigned int bal = __ballot_sync(0xffffffffu, t);
        if (l == 0) wsum[w] = __popc(bal);
        __syncthreads();
        unsigned int before = 0, total = 0;
        for (int k = 0; k < kBlk / 32; ++k) {
            if (k < w) before += wsum[k];
            total += wsum[k];
        }
        const unsigned int rank = prefix + before + __popc(bal & ((1u << l) - 1u));
        if (t && rank < need) {
            cand_idx[n_gt + rank] = i;
            cand_val[n_gt + rank] = tau == 0 ? 0.f : __uint_as_float(tau);
        }
        prefix += total;
        __syncthreads();
    }
}

// Bitonic sort of k candidates by (value desc, index asc); k <= 16384.
__global__ void __launch_bounds__(1024) sort_kernel(const long long* __restrict__ cand_idx,
                                                    const float* __restrict__ cand_val, int k, int kp2,
                                                    long long* __restrict__ out_idx, float* __restrict__ out_val) {
    extern __shared__ __align__(16) unsigned char sm[];
    long long* si = reinterpret_cast<long long*>(sm);
    unsigned int* sv = reinterpret_cast<unsigned int*>(si + kp2);
    for (int i = threadIdx.x; i < kp2; i += blockDim.x) {
        if (i < k) {
            si[i] = cand_idx[i];
            sv[i] = __float_as_uint(cand_val[i]);
        } else {
            si[i] = 0x7fffffffffffffffLL;
            sv[i] = 0u;
        }
    }
    __syncthreads();
    // "a before b" iff a.v > b.v or (a.v == b.v and a.i < b.i)
    for (int size = 2; size <= kp2; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int t = threadIdx.x; t < kp2 / 2; t += blockDim.x) {
                const int i = 2 * t - (t & (stride - 1));
                const int j = i + stride;
                const bool up = (i & size) == 0;
                const unsigned int vi = sv[i], vj = sv[j];
                const long long ii = si[i], ij = si[j];
                const bool i_first = (vi > vj) || (vi == vj && ii < ij);
                if (i_first != up) {
                    sv[i] = vj;
                    sv[j] = vi;
                    si[i] = ij;
                    si[j] = ii;
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < k; i += blockDim.x) {
        out_idx[i] = si[i];
        out_val[i] = __uint_as_float(sv[i]);
    }
}

}  // namespace

cudaError_t launch_topk(const float* v, long long n, int k, TopkWork& w, cudaStream_t s) {
    if (k <= 0 || n <= 0) return cudaSuccess;
    cudaError_t e;
    e = cudaMemsetAsync(w.hist, 0, sizeof(unsigned int) * 3 * kBins, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.state, 0, sizeof(unsigned int) * 16, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(w.n_cand, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    const int hgrid = current_sm_count() * 8;
    // values before the first 16-byte boundary (v itself is 4-byte aligned)
    const int head = (int)std::min<long long>(n, (long long)(((16u - ((uintptr_t)v & 15u)) & 15u) / 4u));
    hist_kernel<0><<<hgrid, kBlk, 0, s>>>(v, n, head, w.state, w.hist);
    select_kernel<0><<<1, 32, 0, s>>>(w.hist, w.state, (unsigned int)k);
    hist_kernel<1><<<hgrid, kBlk, 0, s>>>(v, n, head, w.state, w.hist);
    select_kernel<1><<<1, 32, 0, s>>>(w.hist, w.state, (unsigned int)k);
    hist_kernel<2><<<hgrid, kBlk, 0, s>>>(v, n, head, w.state, w.hist);
    select_kernel<2><<<1, 32, 0, s>>>(w.hist, w.state, (unsigned int)k);
    const long long per_block = (n + w.n_blocks - 1) / w.n_blocks;
    collect_kernel<<<w.n_blocks, kBlk, 0, s>>>(v, n, per_block, w.state, w.cand_idx, w.cand_val, w.n_cand,
                                               w.tie_count);
    tie_kernel<<<w.n_blocks, kBlk, 0, s>>>(v, n, per_block, w.state, w.tie_count, w.cand_idx, w.cand_val);
    int kp2 = 1;
    while (kp2 < k) kp2 <<= 1;
    if (kp2 < 2) kp2 = 2;
    const size_t sm = (size_t)kp2 * 12;
    e = cudaFuncSetAttribute(sort_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sort_kernel<<<1, 1024, sm, s>>>(w.cand_idx, w.cand_val, k, kp2, w.out_idx, w.out_val);
    return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// Toplist without device allocation: the same launch sequence as above, with
// its scratch in one static device array instead of context buffers.
// Sections (byte offsets, each start 4-byte aligned, the candidates 256-byte
// aligned): histograms 3 x 2048 words, state 16 words, tie counts for the
// 1024 collect blocks, the candidate slot counter, then the candidates.
namespace {
constexpr int kNaBlocks = 1024;
constexpr size_t kNaHist = 0;
constexpr size_t kNaState = kNaHist + sizeof(unsigned int) * 3 * kBins;
constexpr size_t kNaTies = kNaState + sizeof(unsigned int) * 16;
constexpr size_t kNaCount = kNaTies + sizeof(unsigned int) * kNaBlocks;
constexpr size_t kNaIdx = (kNaCount + sizeof(unsigned int) + 255) / 256 * 256;
constexpr size_t kNaVal = kNaIdx + sizeof(long long) * FSTAT_NOALLOC_MAX_K;
constexpr size_t kNaBytes = kNaVal + sizeof(float) * FSTAT_NOALLOC_MAX_K;
static_assert(kNaBytes == 225536, "scratch size stated in fstat_noalloc.h");
constexpr int kNaMaxDevices = 64;

std::mutex g_na_mutex;
void* g_na_addr[kNaMaxDevices] = {};
}  // namespace
}  // namespace fs

static __device__ __align__(256) unsigned char g_noalloc_scratch[fs::kNaBytes];

namespace {
int na_fail(char* msg, int32_t msg_len, int code, const char* text, long long a = 0, long long b = 0) {
    if (msg && msg_len > 0) snprintf(msg, (size_t)msg_len, text, a, b);
    return code;
}
}  // namespace

extern "C" int fstat_toplist_noalloc(int device, const float* v, int64_t n, int32_t k, int64_t* idx_out,
                                     float* val_out, void* cuda_stream, char* msg, int32_t msg_len) {
    using namespace fs;
    if (msg && msg_len > 0) msg[0] = 0;
    if (!v || !idx_out || !val_out) return na_fail(msg, msg_len, FSTAT_EINVAL, "null array pointer");
    if (((uintptr_t)v & 3u) || ((uintptr_t)val_out & 3u) || ((uintptr_t)idx_out & 7u))
        return na_fail(msg, msg_len, FSTAT_EINVAL,
                       "misaligned array: v and val_out need 4-byte, idx_out 8-byte alignment");
    if (k > FSTAT_NOALLOC_MAX_K)
        return na_fail(msg, msg_len, FSTAT_ERANGE, "k = %lld is above the static scratch limit of %lld", k,
                       FSTAT_NOALLOC_MAX_K);
    if (n < 1 || k < 1 || (int64_t)k > n)
        return na_fail(msg, msg_len, FSTAT_EINVAL, "need 1 <= k <= n (k = %lld, n = %lld)", k, (long long)n);
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return na_fail(msg, msg_len, FSTAT_ECUDA, "cudaGetDeviceCount failed (error %lld)", (long long)e);
    if (device < 0 || device >= count || device >= kNaMaxDevices)
        return na_fail(msg, msg_len, FSTAT_EINVAL, "device %lld not available (%lld devices)", device, count);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return na_fail(msg, msg_len, FSTAT_ECUDA, "cudaSetDevice(%lld) failed (error %lld)", device, (long long)e);
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[device]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p)
                return na_fail(msg, msg_len, FSTAT_ECUDA, "cudaGetSymbolAddress of the scratch failed on device %lld (error %lld)",
                               device, (long long)e);
            g_na_addr[device] = p;
        }
        base = static_cast<unsigned char*>(g_na_addr[device]);
    }
    TopkWork w{};
    w.hist = reinterpret_cast<unsigned int*>(base + kNaHist);
    w.state = reinterpret_cast<unsigned int*>(base + kNaState);
    w.tie_count = reinterpret_cast<unsigned int*>(base + kNaTies);
    w.n_cand = reinterpret_cast<unsigned int*>(base + kNaCount);
    w.cand_idx = reinterpret_cast<long long*>(base + kNaIdx);
    w.cand_val = reinterpret_cast<float*>(base + kNaVal);
    w.out_idx = reinterpret_cast<long long*>(idx_out);
    w.out_val = val_out;
    w.n_blocks = kNaBlocks;
    e = launch_topk(v, (long long)n, (int)k, w, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) return na_fail(msg, msg_len, FSTAT_ECUDA, "toplist launch failed (error %lld)", (long long)e);
    return FSTAT_OK;
}

