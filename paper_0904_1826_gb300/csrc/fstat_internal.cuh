// Internal definitions shared by the CUDA translation units of libfstat.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/fstat.h"
#include "../../include/fstat_semi.h"

namespace fs {

// Synthetic Sun-centred ephemeris: circular orbit in the ecliptic plane and a
// spherical Earth rotating at the sidereal rate; equatorial coordinates.
constexpr double kC = 299792458.0;                  // speed of light, m/s
constexpr double kAU = 1.495978707e11;              // orbital radius, m
constexpr double kObliquity = 23.4393 * 3.1415926535897932384626433832795 / 180.0;  // rad
constexpr double kYear = 3.15581498e7;              // orbital period, s
constexpr double kEarthR = 6.371e6;                 // Earth radius, m
constexpr double kSidereal = 86164.0905;            // sidereal day, s
constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.1415926535897932384626433832795;

constexpr int kMaxDet = 8;

// Per-SFT detector state at the SFT midpoint (FP64), written once per SFT load.
struct SftState {
    double t_mid;        // t_start + T/2
    double r[3];         // position, m
    double v[3];         // velocity, m/s
    double dt[6];        // response tensor D (xx, xy, xz, yy, yz, zz)
};

// Per-(sky, SFT) constants of the Dirichlet kernel (48 bytes, 16-aligned).
//   khat(j) = khat0(fdot) + j * dk  (fixed point, 2^-32 bins)
//   Phi(j)  = Phi0(fdot) + j * dphi (fixed point, 2^-32 cycles, wraps mod 1)
// span = (M-1) * P * dk checks that a thread's M templates (stride P) keep
// their bin windows L bins apart; eps = P*dk - L in bins (float drift);
// rot = e^{-2 pi i (P*dphi + L/2)} steps the twiddle between them; a, b are the
// antenna weights times the storage scale times the kernel constant 2/pi;
// khmin = min over the spindowns of khat0 (lower bound of every window base).
struct __align__(16) SkySftMeta {
    long long dk;
    long long span;
    unsigned int dphi;
    float eps;
    float rot_re, rot_im;
    float a, b;
    long long khmin;
};
static_assert(sizeof(SkySftMeta) == 48, "SkySftMeta layout");

// Bases of a uniform spindown grid fdot_d = fdot_0 + d * dfdot, per (sky, SFT):
//   khat0(d) = kh0 + d * dkh   (32.32 fixed-point bins)
//   Phi0(d)  = ph0 + d * dph   (0.32 fixed-point cycles, wraps mod 1)
//   rot = e^{-2 pi i dph}      (FP32, the twiddle step from row d to d + 1)
struct __align__(16) SkySftBase {
    long long kh0, dkh;
    unsigned int ph0, dph;
    float rot_re, rot_im;
};
static_assert(sizeof(SkySftBase) == 32, "SkySftBase layout");

struct DirichletParams {
    const void* bins;          // [n_sft][row] complex64 (float2) or 16-bit (half2 / bf162)
    long long row;             // elements per stored SFT row (>= n_bins, padded)
    long long k_lo;            // absolute bin of element 0
    int n_bins;                // valid bins per row
    int n_sft;
    const SkySftMeta* meta;    // [n_sky][n_sft]
    const long long* kh0;      // [n_sky][n_fdot][n_sft] (any spindown list) or null
    const unsigned int* ph0;   // [n_sky][n_fdot][n_sft] or null
    const SkySftBase* base;    // [n_sky][n_sft] (uniform spindown grid) or null
    const float4* comb;        // [n_sky] (2B/D, 2A/D, -4C/D, valid)
    float* twoF;               // [n_sky][n_fdot][n_f]
    int n_sky, n_fdot, n_f;
    int P;                     // template stride inside a thread
    int lg_row;                // lane-groups per row of a full column
    int lg_cta;                // lane-groups per block
    int chunks_per_col;        // blocks per column
    int n_col;                 // columns per sky
    int w_pairs;               // staged pair entries per SFT
    int w_tab;                 // pair-table row length (entries, >= w_pairs)
    int w_raw;                 // raw staging row length (bins, multiple of 4)
    int sft_chunk;             // SFTs per staging round
    int* err;                  // device error flags
    // far-field polynomial form only (null otherwise): per SFT, per window
    // position x (bin k_lo - xoff + x), the adjacent-bin pair table and the
    // far-bin polynomial coefficients, one 48-byte record per position
    const float4* ptab;        // [n_sft][n_pos]
    const float4* pcoef;       // [n_sft][n_pos][3]
    int n_pos;                 // positions per SFT row
    int xoff;                  // position of bin k_lo
    int ring_stop;             // testing aid: the ring's copy warp stops after this many SFTs (< 0: never)
    const int2* cov;           // [n_sft] frequency-index range [x, y) each SFT contributes to, or null (all)
    const float4* comb_j;      // [n_sky][n_f] per-frequency combine weights with coverage, or null
    const int* sky_perm;       // blocks of several sky points: the sky point at each place of the
                               // grouping order (meta and bases SFT-major in that order), or null
};

// Far-field polynomial form (D = 8): the window's 12 bins at offsets -7..-2
// and 3..8 from k0 = floor(khat) contribute (1/2) sum X_k / (kappa - k), a
// smooth function of kappa in [0, 1) (nearest pole 2 away), replaced by its
// degree-5 interpolant sum_n c_n kappa^n; c_n = sum_k X_{k0+k} gamma[k][n].
// The four bins -1..2 next to the poles keep the exact pair form.
constexpr int kFarDeg = 5;
constexpr int kFarTerms = 12;
constexpr int kFarXoff = 10;          // positions below k_lo kept in the tables
struct FarGamma {
    float g[kFarTerms][kFarDeg + 1];  // [far offset index][power]
};
__host__ __device__ constexpr int far_offset(int i) { return i < 6 ? i - 7 : i - 3; }

// Sinc-polynomial form (D = 8): the whole window term
//   P(kappa) = (sin(pi kappa) / 2) sum_{k=-7..8} X_{k0+k} / (kappa - k)
// is entire in kappa (sin vanishes at every integer), so on each half of the
// bin, kappa in [0, 1/2) (h = 0) and [1/2, 1) (h = 1), it is replaced by its
// degree-5 interpolant in v = kappa - 1/4 - h/2 (|v| <= 1/4),
// sum_n c_{h,n} v^n with c_{h,n} = sum_k X_{k0+k} gamma[h][k][n]; no
// reciprocal, sine or clamp remains.  One 48-byte record per (SFT, position,
// half) holds c_{h,0..5} in FP32.
constexpr int kSincDeg = 5;
constexpr int kSincTerms = 16;
// Largest kappa drift over one thread's templates for which one half bin
// serves them all (the interpolant's error grows by < 30 % at 1e-3 outside).
constexpr float kSincSlack = 2e-3f;
struct SincGamma {
    float g[2][kSincTerms][kSincDeg + 1];   // [half][offset k + 7][power]
};

// Shared-memory layout of the far-field kernel (offsets in bytes).
struct PolySmem {
    size_t pairs, coef, meta, base, kh0, ph0, total;
};

// Shared-memory layout of the Dirichlet kernel (offsets in bytes).
struct DirSmem {
    size_t pairs, raw, meta, base, kh0, ph0, lo, total;
};
__host__ __device__ inline size_t smem_align16(size_t x) { return (x + 15) & ~(size_t)15; }
__host__ __device__ inline DirSmem dirichlet_smem(int sft_chunk, int w_tab, int w_raw, int n_fdot,
                                                  int raw_elem_bytes) {
    DirSmem m;
    const size_t C = (size_t)sft_chunk;
    m.pairs = 0;                                                           // float4 pair table [C][w_tab]
    m.raw = smem_align16(m.pairs + C * w_tab * 16);                        // [2][C][w_raw] raw bins
    m.meta = smem_align16(m.raw + 2 * C * w_raw * raw_elem_bytes);         // [3][C] constants
    m.base = smem_align16(m.meta + 3 * C * sizeof(SkySftMeta));            // [3][C] uniform-grid bases
    m.kh0 = smem_align16(m.base + 3 * C * sizeof(SkySftBase));             // [3][C][n_fdot]
    m.ph0 = smem_align16(m.kh0 + 3 * C * n_fdot * 8);                      // [3][C][n_fdot]
    m.lo = smem_align16(m.ph0 + 3 * C * n_fdot * 4);                       // [2][C][2]
    m.total = smem_align16(m.lo + 2 * C * 8);
    return m;
}

__host__ __device__ inline PolySmem farpoly_smem(int sft_chunk, int w_tab, int n_fdot) {
    PolySmem m;
    const size_t C = (size_t)sft_chunk;
    m.pairs = 0;                                                     // float4 [2][C][w_tab]
    m.coef = smem_align16(m.pairs + 2 * C * w_tab * 16);              // float4 [2][C][w_tab][3]
    m.meta = smem_align16(m.coef + 6 * C * w_tab * 16);               // [3][C]
    m.base = smem_align16(m.meta + 3 * C * sizeof(SkySftMeta));       // [3][C]
    m.kh0 = smem_align16(m.base + 3 * C * sizeof(SkySftBase));        // [3][C][n_fdot]
    m.ph0 = smem_align16(m.kh0 + 3 * C * n_fdot * 8);                 // [3][C][n_fdot]
    m.total = smem_align16(m.ph0 + 3 * C * n_fdot * 4);
    return m;
}

// Shared-memory layout of the ring kernel: S stages of
// [pairs w_tab x 16 B][coefficient records w_tab x 48 B] (far field) or
// [half-bin plane 0][half-bin plane 1] (sinc), then [meta 48 B][base 32 B]
// (one of each per sky point of the block) [window base 16 B] (128-byte
// aligned), then a full and an empty mbarrier
// per stage, then two control words (stages issued, abort).
struct RingSmem {
    size_t stage, pairs, coef, plane, meta, base, lo, bars, ctrl, total;
};
// The far-field form stages a 16-byte pair and a 48-byte coefficient record
// per position; the sinc form two 48-byte records (one per half bin) in two
// planes whose distance is a multiple of 128 bytes, so that the half a
// template picks does not change its shared-memory bank.
__host__ __device__ inline RingSmem ring_smem(int stages, int w_tab, bool sinc = false, int sky_rows = 1) {
    RingSmem r;
    r.pairs = 0;
    r.plane = ((size_t)w_tab * 48 + 127) & ~(size_t)127;
    r.coef = sinc ? 0 : (size_t)w_tab * 16;
    r.meta = sinc ? 2 * r.plane : r.coef + (size_t)w_tab * 48;
    r.base = r.meta + 48 * (size_t)sky_rows;   // one meta and one base per sky point of the block
    r.lo = r.base + 32 * (size_t)sky_rows;
    r.stage = (r.lo + 16 + 127) & ~(size_t)127;
    r.bars = (size_t)stages * r.stage;
    r.ctrl = r.bars + 16 * (size_t)stages;
    r.total = r.ctrl + 16;
    return r;
}

// Device-side description of a batch of template banks for the persistent kernel.
struct DirichletBatch {
    const DirichletParams* banks;     // [n_wu]
    const long long* item_prefix;     // [n_wu + 1]
    int n_wu;
    unsigned long long* queue;        // work counter (zeroed per launch)
    int* remaining;                   // [n_wu] items left per bank
    unsigned long long* done_ns;      // [n_wu] completion time (globaltimer)
};

struct TimingParams {
    const SftState* st;        // [n_sft]
    const double* sky;         // [n_sky][2]
    const double* fdot;        // [n_fdot]
    const float* scale;        // [n_sft] storage scale (1 for complex64)
    const double* weight;      // [n_sft] noise weights (null: all 1)
    int n_sky, n_sft, n_fdot;
    double f0, df, T, t_ref;
    int P, L, M;
    int uniform;               // spindowns fdot_0 + d * dfdot: write `base`, else kh0 / ph0
    double dfdot;
    SkySftMeta* meta;          // out [n_sky][n_sft], or [n_sft][n_sky] when sft_major
    SkySftBase* base;          // out [n_sky][n_sft] (uniform), or [n_sft][n_sky] when sft_major
    int sft_major;             // SFT-major meta and bases (blocks of several sky points)
    const int* sky_rank;       // with sft_major: each sky point's place in the grouping order, or null
    int row_rot;               // write the bases' row twiddle step (row-tiled forms)
    long long* kh0;            // out [n_sky][n_fdot][n_sft] (not uniform)
    unsigned int* ph0;         // out [n_sky][n_fdot][n_sft] (not uniform)
    double* abcd;              // out [n_sky][4]
    float4* comb;              // out [n_sky]
    int* err;
};

// Streaming multiprocessors of the calling thread's current device, queried
// once per device (grid sizes are multiples of it).
inline int current_sm_count() {
    static int cache[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
    if (dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    if (dev < 64) cache[dev] = n;
    return n;
}

// ---- launchers (defined in the .cu files) --------------------------------
cudaError_t launch_sft_state(const double* t_start, const int* det_of_sft, const fstat_detector* dets,
                             int n_sft, double T, SftState* out, cudaStream_t s);
cudaError_t launch_timing(const TimingParams& p, cudaStream_t s);
cudaError_t launch_sft_timing_one(const SftState* st, int n_sft, double alpha, double delta,
                                  double t_ref, double* out4, cudaStream_t s);
cudaError_t launch_inject(const SftState* st, int n_sft, const fstat_signal* sig_dev, int n_sig,
                          double T, double t_ref, long long k_lo, int n_bins, long long row,
                          float2* bins, double* work, cudaStream_t s);
cudaError_t launch_noise_floor(const float2* bins, long long row, int n_sft, int n_bins, int half, float* floor,
                               float2* white, double* sbar, double* weight, cudaStream_t s);
cudaError_t launch_quantize(const float2* src, long long row, int n_sft, int n_bins, int form,
                            void* dst, float* scale, cudaStream_t s);


cudaError_t launch_patches(const float* twoF, int n_f, int n_d, int s_a, int s_d, int n_fp, const int* f_start_dev,
                           int n_q, int n_patches, int n_pd, float shift, float scale, void* out, cudaStream_t s);
cudaError_t launch_windows(const float* twoF, int n_f, int n_a, int n_d, int s_a, int s_d, int n_fp,
                           const int* origin_dev, int n_w, float shift, float scale, void* out, cudaStream_t s);

// Toplist (radix select over the FP32 bit patterns of 2F >= 0).
struct TopkWork {
    unsigned int* hist;        // [3][2048]
    unsigned int* state;       // [16] prefix, threshold, counts
    unsigned int* tie_count;   // [n_blocks]
    long long* cand_idx;       // [topk]
    float* cand_val;           // [topk]
    unsigned int* n_cand;      // [1]
    long long* out_idx;        // [topk]
    float* out_val;            // [topk]
    int n_blocks;
};
cudaError_t launch_far_tables(const void* bins, int form, long long row, int n_sft, int n_bins, const FarGamma& gam,
                              float4* ptab, float4* pcoef, int n_pos, int xoff, cudaStream_t s);
// split: positions split by parity (the L = 2 layout) or plain (L = 1).
cudaError_t launch_sinc_tables(const void* bins, int form, long long row, int n_sft, int n_bins,
                               const SincGamma& gam, float4* pcoef, int n_pos, int xoff, bool split,
                               cudaStream_t s);
cudaError_t launch_dirichlet_far(int v, const DirichletParams& p, int threads, size_t smem, long long grid,
                                 cudaStream_t s);
cudaError_t launch_dirichlet_far_batch(int v, const DirichletBatch& b, int threads, size_t smem, int grid,
                                       cudaStream_t s);
cudaError_t dirichlet_far_batch_occupancy(int v, int threads, size_t smem, int* blocks_per_sm);
cudaError_t launch_topk(const float* v, long long n, int k, TopkWork& w, cudaStream_t s);

// One segment of a stack-slide: its device 2F [n_sky][n_fdot][n_f] and grid.
struct SlideSeg {
    const float* twoF;
    long long n_f;
    double f0, df, t;
};
// prep = false reuses A_fx, B_fx of an earlier call with the same segments and
// grid; unit = every segment's df_s equals df exactly (B = 1).
cudaError_t launch_stackslide(const SlideSeg* seg, int n_seg, const double* fdot, int n_fdot, double f0, double df,
                              double t_ref, long long* A_fx, long long* B_fx, bool prep, bool unit, long long n_rows,
                              int n_f, float* out, unsigned long long* n_outside, cudaStream_t s);

// Per-(sky, frequency) combine weights over the SFTs covering each frequency
// index (one block per sky point; n_f <= kCovMaxF).
constexpr int kCovMaxF = 8192;
cudaError_t launch_coverage_comb(const TimingParams& tp, const int2* cov, int n_f, float4* comb_j, cudaStream_t s);

}  // namespace fs
