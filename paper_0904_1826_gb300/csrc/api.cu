// C ABI of libfstat: context, input validation, tile planning and launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "fstat_internal.cuh"
#include "../../include/fstat_mlp.h"

namespace fs {
cudaError_t launch_dirichlet_c64(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                                 long long grid, cudaStream_t s);
cudaError_t launch_dirichlet_f16(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                                 long long grid, cudaStream_t s);
cudaError_t launch_dirichlet_bf16(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                                  long long grid, cudaStream_t s);
cudaError_t launch_dirichlet_batch_c64(int v, const DirichletBatch& b, int d_rt, int threads, size_t smem,
                                     int grid, cudaStream_t s);
cudaError_t launch_dirichlet_batch_f16(int v, const DirichletBatch& b, int d_rt, int threads, size_t smem,
                                     int grid, cudaStream_t s);
cudaError_t launch_dirichlet_batch_bf16(int v, const DirichletBatch& b, int d_rt, int threads, size_t smem,
                                      int grid, cudaStream_t s);
cudaError_t dirichlet_occupancy_c64(int v, int threads, size_t smem, int* blocks_per_sm);
cudaError_t dirichlet_occupancy_f16(int v, int threads, size_t smem, int* blocks_per_sm);
cudaError_t dirichlet_occupancy_bf16(int v, int threads, size_t smem, int* blocks_per_sm);
size_t inject_work_doubles(int n_sig, int n_sft);
}  // namespace fs

using namespace fs;

namespace {

// Variant table, in the order of FS_DIRICHLET_VARIANTS: (D, M, L, kahan).
struct VariantRow {
    int D, M, L, kahan;
};
const VariantRow kVariants[] = {{8, 9, 2, 0}, {8, 7, 2, 0}, {8, 5, 2, 0}, {8, 9, 1, 0}, {8, 7, 1, 0}, {8, 1, 1, 0},
                                {8, 5, 2, 1}, {8, 5, 1, 1}, {8, 1, 1, 1}, {0, 1, 1, 0}, {0, 1, 1, 1}};
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);

// Far-field polynomial variants, in the order of FS_FAR_VARIANTS: (M, L); D = 8.
struct FarRow {
    int M, L;
    int ring;   // compute warps of the TMA-ring staging (L = 2, uniform spindown grid), 0 = cp.async rounds
    bool sinc;  // sinc-polynomial form (whole window as one polynomial), else near pairs + far polynomial
    bool cov;   // per-SFT frequency coverage compiled in (ring only; single launches)
    int rows;   // rows form: spindown rows per lane (one frequency per lane), 0 = templates along frequency
    int minb;   // two-row tiles (sinc, L = 2): resident blocks per SM the kernel is built for, 0 = one row
    int sr;     // one-row ring with blocks of `sr` consecutive sky points (0: one)
};
const FarRow kFarVariants[] = {{7, 2, 0, false, false, 0},  {5, 2, 0, false, false, 0},  {9, 2, 0, false, false, 0},
                               {7, 1, 0, false, false, 0},  {9, 1, 0, false, false, 0},  {5, 1, 0, false, false, 0},
                               {1, 1, 0, false, false, 0},  {5, 2, 8, false, false, 0},  {7, 2, 8, false, false, 0},
                               {9, 2, 8, false, false, 0},  {5, 2, 10, false, false, 0}, {7, 2, 10, false, false, 0},
                               {5, 2, 10, true, false, 0},  {7, 2, 10, true, false, 0},  {5, 2, 8, true, false, 0},
                               {7, 2, 8, true, false, 0},   {5, 2, 10, true, true, 0},   {5, 2, 10, false, true, 0},
                               {5, 1, 8, true, false, 0},   {1, 1, 8, true, false, 0},
                               // rows form, in the order of FS_ROWS_VARIANTS: (R, NWC)
                               {1, 1, 3, true, false, 10},  {1, 1, 4, true, false, 10},  {1, 1, 8, true, false, 10},
                               {1, 1, 4, true, false, 5},   {1, 1, 8, true, false, 5},   {1, 1, 4, true, false, 8},
                               {1, 1, 4, true, false, 4},
                               // two-row tiles, in the order of FS_RING2_VARIANTS: (M, NWC, blocks per SM)
                               {5, 2, 8, true, false, 0, 2},  {3, 2, 10, true, false, 0, 2},
                               // one-row sinc ring with 4 and 2 compute warps (few spindowns: full blocks
                               // with narrow columns), in FS_RING_VARIANTS
                               {5, 2, 4, true, false, 0, 0},  {5, 2, 2, true, false, 0, 0},
                               // blocks of 4 sky points, in the order of FS_RING_SKY_VARIANTS
                               {5, 2, 10, true, false, 0, 0, 4}, {5, 2, 10, false, false, 0, 0, 4},
                               {5, 1, 8, true, false, 0, 0, 4},  {1, 1, 8, true, false, 0, 0, 4}};
constexpr int kNumFar = sizeof(kFarVariants) / sizeof(kFarVariants[0]);
constexpr int kFarIdBase = 100;   // variant ids reported for the far-field form

constexpr int kTimedRing = 256;

struct Plan {
    int P = 1, L = 1, M = 1, W = 8, C = 8, lg_row = 1, lg_cta = 32, n_col = 1, chunks_per_col = 1;
    int w_pairs = 0, w_tab = 0, w_raw = 0, variant = 5;
    bool far = false;   // far-field polynomial form (variant indexes kFarVariants)
    bool ring = false;  // far-field form with TMA-ring staging; C = stages, W includes the producer warp
    bool sinc = false;  // sinc-polynomial form (TMA ring only)
    bool rows = false;  // rows form of the sinc polynomial: M = 1 frequency per lane, R rows (kFarVariants)
    bool two = false;   // two-row tiles of the sinc ring form (L = 2)
    int sky_rows = 1;   // sky points per block of the one-row ring (meta and bases SFT-major when > 1)
    bool sky_perm = false;   // blocks group the sky points in the context's neighbour order
    size_t smem = 0;
    long long grid = 0;
};

struct Det {
    bool set = false;
    fstat_detector g{};
    std::vector<double> t_start;
};

}  // namespace

struct fstat_ctx {
    int device = 0;
    fstat_opts opts{};
    std::string err;
    // SFT store
    bool have_sfts = false;
    double T = 0.0;
    long long k_lo = 0;
    int n_bins = 0;
    long long row = 0;   // padded row length (multiple of 8 elements)
    Det det[kMaxDet];
    int n_sft = 0;
    int sft_capacity = 0;
    float2* d_bins = nullptr;       // complex64 master copy
    int nf_half = 0;                // noise floor: running-median half window (0 = off)
    float2* d_bins_w = nullptr;     // whitened copy (noise floor on)
    float* d_floor = nullptr;       // noise floor S [n_sft][n_bins]
    double* d_sbar = nullptr;       // mean floor per SFT
    double* d_weight = nullptr;     // noise weight per SFT
    // per-SFT frequency coverage (fstat_set_coverage)
    bool have_cov = false;
    int2* d_cov = nullptr;          // [n_sft] frequency-index range [x, y)
    float4* d_comb_j = nullptr;     // [n_sky][n_f] combine weights per frequency
    size_t cap_comb_j = 0;
    // stack-slide scratch (held by the first segment of a call)
    SlideSeg* d_slide_seg = nullptr;
    long long* d_slide_A = nullptr;
    long long* d_slide_B = nullptr;
    unsigned long long* d_slide_out = nullptr;
    size_t cap_slide_seg = 0, cap_slide_A = 0, cap_slide_B = 0, cap_slide_out = 0;
    std::vector<SlideSeg> slide_last;   // segment table, grid and spindowns of the last call (reused when equal)
    std::vector<double> slide_fdot;
    double slide_grid[3] = {0, 0, 0};
    const long long* slide_A_at = nullptr;
    size_t cap_bins_w = 0, cap_floor = 0, cap_sbar = 0, cap_weight = 0;
    void* d_bins16 = nullptr;       // 16-bit copy (precision forms)
    float* d_scale = nullptr;       // per-SFT storage scale
    SftState* d_state = nullptr;
    double* d_tstart = nullptr;
    int* d_det_of = nullptr;
    bool sft_dirty = true;          // state / quantisation need refresh
    bool tab_dirty = true;          // far-field tables need a rebuild
    FarGamma gam{};                 // far-field interpolation weights
    SincGamma sgam{};               // sinc-polynomial interpolation weights
    bool tab_sinc = false;          // kind of the built tables
    bool tab_split = true;          // sinc tables split by position parity (L = 2) or plain (L = 1)
    float4* d_ptab = nullptr;       // far-field pair table [n_sft][n_pos]
    float4* d_pcoef = nullptr;      // far-field coefficients [n_sft][4][n_pos]
    size_t cap_ptab = 0, cap_pcoef = 0;
    int ring_stall = -1;             // testing aid (fstat_test_ring_stall)
    int n_pos = 0, far_xoff = 0;     // table extent of the current plan
    int tab_npos = -1, tab_xoff = -1; // extent the built tables have
    // template bank
    bool have_templates = false;
    int n_sky = 0, n_f = 0, n_fdot = 0;
    double f0 = 0, df = 0, t_ref = 0;
    double* d_sky = nullptr;
    double* d_fdot = nullptr;
    std::vector<double> h_sky, h_fdot;
    bool fdot_uniform = true;         // spindowns fdot_0 + d * dfdot (compact bases)
    bool batch_member = false;        // a workunit of a batch (kernels with a persistent form only)
    std::vector<int> h_order;         // sky points in neighbour order (empty: not computed yet)
    double order_spread4 = -1.0;      // window spread bound of 4 consecutive points of h_order (bins)
    int* d_perm = nullptr;            // [n_sky] h_order on the device
    int* d_rank = nullptr;            // [n_sky] each sky point's place in h_order
    bool perm_on_device = false;
    double dfdot = 0.0;
    // derived per-bank buffers
    size_t cap_meta = 0, cap_kh0 = 0, cap_ph0 = 0, cap_abcd = 0, cap_comb = 0, cap_twoF = 0;
    SkySftMeta* d_meta = nullptr;
    SkySftBase* d_base = nullptr;
    size_t cap_base = 0;
    long long* d_kh0 = nullptr;
    unsigned int* d_ph0 = nullptr;
    double* d_abcd = nullptr;
    float4* d_comb = nullptr;
    float* d_twoF = nullptr;
    int* d_err = nullptr;
    // toplist
    TopkWork tw{};
    int tw_k = 0;
    // plan and bookkeeping
    Plan plan;
    bool plan_valid = false;
    bool computed = false;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_a[kTimedRing]{}, ev_b[kTimedRing]{}, ev_c[kTimedRing]{}, ev_d[kTimedRing]{};
    int n_timed = 0;
    long long launches = 0;   // kernels launched by this context
    double* d_inj_work = nullptr;
    size_t cap_inj = 0;
    fstat_signal* d_sig = nullptr;
    size_t cap_sig = 0;
    // batched form: child contexts, one per workunit
    std::vector<fstat_ctx*> wus;
    bool batch_ran = false;           // first batch compute done (buffers and attributes set)
    bool graph_valid = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    // groups after the first run on side streams forked from and joined to the
    // batch stream, so that one group's blocks fill the SMs another leaves
    std::vector<cudaStream_t> side_streams;
    std::vector<cudaEvent_t> side_events;   // [0] fork, [1 + g] join of side stream g
    DirichletParams* d_banks = nullptr;
    long long* d_prefix = nullptr;
    int* d_rem_init = nullptr;
    int* d_rem = nullptr;
    unsigned long long* d_queue = nullptr;
    unsigned long long* d_done = nullptr;   // [n_wu + 1], last = batch start
    int n_groups = 0;
    cudaEvent_t bev0 = nullptr, bev1 = nullptr;
    long long launches_per_graph = 0;
    std::vector<int> batch_order;     // grouped position -> workunit index
    int* d_fstart = nullptr;          // patch frequency starts
    size_t cap_fstart = 0;
};

namespace {

int fail(fstat_ctx* c, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return code;
}

#define CUDA_TRY(ctx, call)                                                                      \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? FSTAT_ENOMEM : FSTAT_ECUDA,      \
                        "%s: %s", #call, cudaGetErrorString(e_));                                \
    } while (0)

template <class T>
int grow(fstat_ctx* c, T** p, size_t& cap, size_t n) {
    if (n <= cap && *p) return FSTAT_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
    if (e != cudaSuccess) return fail(c, FSTAT_ENOMEM, "cudaMalloc(%zu bytes): %s", n * sizeof(T), cudaGetErrorString(e));
    cap = n;
    return FSTAT_OK;
}

int set_device(fstat_ctx* c) {
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "cudaSetDevice(%d): %s", c->device, cudaGetErrorString(e));
    return FSTAT_OK;
}

int variant_id(int D, int M, int L, int kahan) {
    for (int i = 0; i < kNumVariants; ++i) {
        const VariantRow& v = kVariants[i];
        if (v.D == D && v.M == M && v.L == L && v.kahan == kahan) return i;
    }
    return -1;
}

// Templates in a column the staging range has to cover, and its width in pairs.
int pairs_needed(const fstat_ctx* c, int span_templates, int D) {
    // largest tdot: orbital + rotational speed over c, with margin
    const double tdot_max = 1.0 + 1.1e-4;
    const double dk_max = c->df * c->T * tdot_max;
    double fd_min = c->h_fdot[0], fd_max = c->h_fdot[0];
    for (double v : c->h_fdot) {
        fd_min = std::min(fd_min, v);
        fd_max = std::max(fd_max, v);
    }
    double tau_max = 0.0;
    for (int d = 0; d < kMaxDet; ++d)
        for (double t : c->det[d].t_start) tau_max = std::max(tau_max, std::fabs(t + 0.5 * c->T - c->t_ref));
    tau_max += 500.0;   // Roemer delay bound (AU + R_E)/c < 500 s
    const double spread = (fd_max - fd_min) * tau_max * c->T * tdot_max;
    return (int)std::ceil((span_templates - 1) * dk_max + spread) + 2 * D + 4;
}

// Bound, in bins, on how far apart the windows of `g` consecutive sky points
// of the bank can start: khat = f T tdot with tdot - 1 = v.n / c, |v| / c <=
// 1.1e-4 (orbit and rotation), so two sky points' khat differ by at most
// f_max T 1.1e-4 |n_1 - n_2| (the Roemer delay's share, fdot T dtau, is below
// 1e-3 bins); the maximum over all groups of g, plus one bin.
double sky_spread_bins(const fstat_ctx* c, int g, const std::vector<int>* order = nullptr) {
    const double k_max = (c->f0 + (c->n_f - 1) * c->df) * c->T;
    double chord = 0.0;
    for (int s0 = 0; s0 < c->n_sky; s0 += g) {
        const int s1 = std::min(c->n_sky, s0 + g);
        for (int ia = s0; ia < s1; ++ia)
            for (int ib = ia + 1; ib < s1; ++ib) {
                const int a = order ? (*order)[ia] : ia, b = order ? (*order)[ib] : ib;
                const double aa = c->h_sky[2 * a], da = c->h_sky[2 * a + 1];
                const double ab = c->h_sky[2 * b], db = c->h_sky[2 * b + 1];
                const double dx = std::cos(da) * std::cos(aa) - std::cos(db) * std::cos(ab);
                const double dy = std::cos(da) * std::sin(aa) - std::cos(db) * std::sin(ab);
                const double dz = std::sin(da) - std::sin(db);
                chord = std::max(chord, std::sqrt(dx * dx + dy * dy + dz * dz));
            }
    }
    return k_max * 1.1e-4 * chord + 1.0;
}

// An order of the sky points in which consecutive ones are neighbours: bands
// of equal width in delta (0.6 sqrt(n) of them: on a near-uniform sky this
// gave the smallest largest chord within groups of 4, e.g. 0.21 for 3000
// points and 0.09 for 16 435), alpha ascending in even bands and descending
// in odd ones.
std::vector<int> sky_neighbour_order(const fstat_ctx* c) {
    const int n = c->n_sky;
    const int nb = std::max(1, (int)std::lround(0.6 * std::sqrt((double)n)));
    std::vector<std::pair<double, int>> key(n);
    for (int i = 0; i < n; ++i) {
        double a = std::fmod(c->h_sky[2 * i], 2.0 * kPi);
        if (a < 0) a += 2.0 * kPi;
        const int band = std::min(nb - 1, std::max(0, (int)std::floor((c->h_sky[2 * i + 1] + 0.5 * kPi) / kPi * nb)));
        key[i] = {band * 10.0 + ((band & 1) ? 2.0 * kPi - a : a), i};
    }
    std::sort(key.begin(), key.end());
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = key[i].second;
    return order;
}

// Weights of the far-field form: for each far offset k, the monomial
// coefficients of the degree-kFarDeg polynomial interpolating 0.5 / (kappa - k)
// at the Chebyshev points of [0, 1] (FP64 Gaussian elimination, stored FP32).
FarGamma far_gamma() {
    FarGamma G{};
    constexpr int N = kFarDeg + 1;
    for (int i = 0; i < kFarTerms; ++i) {
        const double k = far_offset(i);
        double A[N][N + 1];
        for (int j = 0; j < N; ++j) {
            const double x = 0.5 + 0.5 * std::cos((2.0 * j + 1.0) * kPi / (2.0 * N));
            double pw = 1.0;
            for (int n = 0; n < N; ++n) {
                A[j][n] = pw;
                pw *= x;
            }
            A[j][N] = 0.5 / (x - k);
        }
        for (int col = 0; col < N; ++col) {
            int piv = col;
            for (int r = col + 1; r < N; ++r)
                if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
            for (int t = 0; t <= N; ++t) std::swap(A[col][t], A[piv][t]);
            for (int r = 0; r < N; ++r) {
                if (r == col) continue;
                const double f = A[r][col] / A[col][col];
                for (int t = col; t <= N; ++t) A[r][t] -= f * A[col][t];
            }
        }
        for (int n = 0; n < N; ++n) G.g[i][n] = (float)(A[n][N] / A[n][n]);
    }
    return G;
}

// Weights of the sinc-polynomial form: for each window offset k = -7..8, the
// monomial coefficients in u = kappa - 1/2 of the degree-kSincDeg polynomial
// interpolating sin(pi kappa) / (2 (kappa - k)) at the Chebyshev points of
// u in [-1/2, 1/2] (FP64 Gaussian elimination, stored FP32).
SincGamma sinc_gamma() {
    SincGamma G{};
    constexpr int N = kSincDeg + 1;
    for (int h = 0; h < 2; ++h) {
        const double centre = 0.25 + 0.5 * h;
        for (int i = 0; i < kSincTerms; ++i) {
            const double k = i - 7;
            double A[N][N + 1];
            for (int j = 0; j < N; ++j) {
                const double v = 0.25 * std::cos((2.0 * j + 1.0) * kPi / (2.0 * N));
                const double kap = centre + v;
                double pw = 1.0;
                for (int n = 0; n < N; ++n) {
                    A[j][n] = pw;
                    pw *= v;
                }
                A[j][N] = std::sin(kPi * kap) / (2.0 * (kap - k));
            }
            for (int col = 0; col < N; ++col) {
                int piv = col;
                for (int r = col + 1; r < N; ++r)
                    if (std::fabs(A[r][col]) > std::fabs(A[piv][col])) piv = r;
                for (int t = 0; t <= N; ++t) std::swap(A[col][t], A[piv][t]);
                for (int r = 0; r < N; ++r) {
                    if (r == col) continue;
                    const double f = A[r][col] / A[col][col];
                    for (int t = col; t <= N; ++t) A[r][t] -= f * A[col][t];
                }
            }
            for (int n = 0; n < N; ++n) G.g[h][i][n] = (float)(A[n][N] / A[n][n]);
        }
    }
    return G;
}

bool far_eligible(const fstat_ctx* c) {
    return c->opts.dterms == 8 && !c->opts.kahan && c->opts.algo != FSTAT_ALGO_DIRECT;
}

// Extent of the far-field tables such that every block's rows [x0, x0 + w_pairs)
// lie inside them: khat is bounded over the bank by the frequency and spindown
// ranges, |tdot - 1| <= 1.1e-4 (orbital + rotational speed over c) and dtau
// within the SFT span of t_ref widened by 500 s of Roemer delay.
void far_extent(const fstat_ctx* c, int w_pairs, int* xoff, int* n_pos) {
    double tmin = 1e300, tmax = -1e300;
    for (int d = 0; d < kMaxDet; ++d)
        for (double t : c->det[d].t_start) {
            tmin = std::min(tmin, t);
            tmax = std::max(tmax, t + c->T);
        }
    double fdmin = c->h_fdot[0], fdmax = c->h_fdot[0];
    for (double v : c->h_fdot) {
        fdmin = std::min(fdmin, v);
        fdmax = std::max(fdmax, v);
    }
    const double fs[2] = {c->f0, c->f0 + (c->n_f - 1) * c->df};
    const double fds[2] = {fdmin, fdmax};
    const double dts[2] = {tmin - c->t_ref - 500.0, tmax - c->t_ref + 500.0};
    const double tds[2] = {1.0 - 1.1e-4, 1.0 + 1.1e-4};
    double kmin = 1e300, kmax = -1e300;
    for (double f : fs)
        for (double fd : fds)
            for (double dt : dts)
                for (double td : tds) {
                    const double k = (f + fd * dt) * td * c->T;
                    kmin = std::min(kmin, k);
                    kmax = std::max(kmax, k);
                }
    const long long lo_min = (long long)std::floor(kmin) - c->k_lo - 7 - 2;
    const long long lo_max = (long long)std::floor(kmax) - c->k_lo - 7 + 2;
    const long long xo = std::max<long long>(kFarXoff, -lo_min);
    long long np = std::max<long long>(c->n_bins + xo + kFarXoff, xo + lo_max + w_pairs + 2);
    *xoff = (int)xo;
    *n_pos = (int)((np + 1) & ~1LL);   // even: two equal parity halves
}

// Plan of the far-field form (D = 8); false when no variant fits.  Cost model
// per block and SFT: ~40 instructions of set-up per thread plus ~58 per
// template (polynomial, two near pairs, twiddle, accumulation, 6 table
// loads), ~8 per staged table entry and plane, ~2000 per round (barrier).
// Plan of the rows form (SINCROWS, uniform spindown grid, no coverage, at
// least 4 spindowns): the (R, NWC) variant with the least modelled work.
// Per lane and SFT ~45 instructions of set-up and ~26 per row, idle lanes of
// the last column and idle rows of the last row chunk included; ~0.05 per
// staged position and byte.
bool make_rows_plan(fstat_ctx* c, Plan& best) {
    if (!c->fdot_uniform || c->have_cov || c->n_fdot < 4) return false;
    if (c->opts.algo != FSTAT_ALGO_SINCROWS) return false;
    if (c->opts.tile_m > 1) return false;   // templates along frequency requested
    double best_cost = 1e300;
    bool have = false;
    for (int i = 0; i < kNumFar; ++i) {
        const FarRow& v = kFarVariants[i];
        if (!v.rows) continue;
        if (c->opts.tile_warps > 0 && c->opts.tile_warps != v.ring + 1) continue;
        const int F = 32 * v.ring;
        const int n_col = (c->n_f + F - 1) / F;
        const int n_rc = (c->n_fdot + v.rows - 1) / v.rows;
        const int w_pairs = pairs_needed(c, F, 8);
        int S = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 8;
        while (S > 3 && ring_smem(S, w_pairs, true).total > 110 * 1024) --S;
        const size_t smem = ring_smem(S, w_pairs, true).total;
        if (smem > 220 * 1024) continue;
        const double lanes = (double)n_col * F * n_rc;
        const double per_lane = (45.0 + 26.0 * v.rows) * (1.0 + 0.2 / S);
        const double cost = (double)c->n_sky * (lanes * per_lane + (double)n_col * n_rc * w_pairs * 96.0 * 0.05);
        if (cost < best_cost * 0.999) {
            best_cost = cost;
            best = Plan{};
            best.P = 1;
            best.L = 1;
            best.M = 1;
            best.W = v.ring + 1;
            best.C = S;
            best.lg_row = F;
            best.lg_cta = F;
            best.n_col = n_col;
            best.chunks_per_col = n_rc;
            best.w_pairs = w_pairs;
            best.w_tab = w_pairs;
            best.variant = i;
            best.far = true;
            best.ring = true;
            best.sinc = true;
            best.rows = true;
            best.smem = smem;
            best.grid = (long long)c->n_sky * n_col * n_rc;
            have = true;
        }
    }
    return have;
}

// Plan of the two-row tiles (SINCPAIRS; sinc form, L = 2, uniform
// spindown grid, no coverage, at least 2 spindowns).  Per thread and SFT
// ~70 instructions of set-up and ~30 per template pair of rows; stages sized
// for the variant's resident blocks per SM.
bool make_ring2_plan(fstat_ctx* c, int P, int L, bool found, Plan& best) {
    if (!found || L != 2 || !c->fdot_uniform || c->have_cov || c->n_fdot < 2) return false;
    if (c->opts.algo != FSTAT_ALGO_SINCPAIRS) return false;
    double best_cost = 1e300;
    bool have = false;
    for (int i = 0; i < kNumFar; ++i) {
        const FarRow& v = kFarVariants[i];
        if (!v.minb) continue;
        if (c->opts.tile_m > 0 && c->opts.tile_m != v.M) continue;
        if (c->opts.tile_warps > 0 && c->opts.tile_warps != v.ring + 1) continue;
        if (v.ring % P != 0) continue;
        const int PM = P * v.M;
        const int lg_cta = 32 * v.ring / P;
        const int n_pairs = (c->n_fdot + 1) / 2;
        const int lg_max = std::min((c->n_f + PM - 1) / PM, lg_cta);
        const size_t cap = (227 * 1024) / v.minb - 2048;
        for (int lg_row = 1; lg_row <= lg_max; ++lg_row) {
            const int col_w = lg_row * PM;
            const int n_col = (c->n_f + col_w - 1) / col_w;
            const int w_pairs = std::max(pairs_needed(c, col_w, 8), (v.M - 1) * L + 2 * 8 + 2);
            int hf = (w_pairs + 1) / 2;
            hf += ((4 - hf % 8) + 8) % 8;
            const int w_tab = 2 * hf;
            int S = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 8;
            while (S > 2 && ring_smem(S, w_tab, true).total > cap) --S;
            const size_t smem = ring_smem(S, w_tab, true).total;
            if (smem > cap) continue;
            double cost = 0.0;
            int chunks_max = 0;
            for (int col = 0; col < n_col; ++col) {
                const int width = std::min(col_w, c->n_f - col * col_w);
                const int Gc = (width + PM - 1) / PM;
                const long long LG = (long long)n_pairs * Gc;
                const int chunks = (int)((LG + lg_cta - 1) / lg_cta);
                chunks_max = std::max(chunks_max, chunks);
                for (int k = 0; k < chunks; ++k) {
                    const long long lgs = std::min<long long>(lg_cta, LG - (long long)k * lg_cta);
                    const long long warps = (lgs + 31) / 32 * P;
                    cost += (double)warps * 32.0 * (70.0 + 30.0 * 2 * v.M) * (1.0 + 0.2 / S) + 0.05 * w_pairs * 96.0;
                }
            }
            if (cost < best_cost * 0.999) {
                best_cost = cost;
                best = Plan{};
                best.P = P;
                best.L = L;
                best.M = v.M;
                best.W = v.ring + 1;
                best.C = S;
                best.lg_row = lg_row;
                best.lg_cta = lg_cta;
                best.n_col = n_col;
                best.chunks_per_col = chunks_max;
                best.w_pairs = w_pairs;
                best.w_tab = w_tab;
                best.variant = i;
                best.far = true;
                best.ring = true;
                best.sinc = true;
                best.two = true;
                best.smem = smem;
                best.grid = (long long)c->n_sky * n_col * chunks_max;
                have = true;
            }
        }
    }
    return have;
}

bool make_far_plan(fstat_ctx* c, int P, int L, bool found, Plan& best) {
    if (c->opts.algo == FSTAT_ALGO_SINCROWS && make_rows_plan(c, best)) return true;
    if (make_ring2_plan(c, P, L, found, best)) return true;
    bool have_ring = false;
    // TMA-ring form first: L = 2, compact spindown bases
    // default: 10 compute warps + 1 copy warp (measured fastest on GB300); tile_warps 9 / 11 choose 8 / 10
    // AUTO takes the sinc-polynomial form where the ring applies (731 ms per
    // workunit launch on GB300 against 1106 ms for near pairs + far polynomial)
    const int tw = c->opts.tile_warps;
    const bool sinc_ok = c->opts.algo == FSTAT_ALGO_SINCPOLY || c->opts.algo == FSTAT_ALGO_AUTO ||
                         c->opts.algo == FSTAT_ALGO_SINCROWS || c->opts.algo == FSTAT_ALGO_SINCPAIRS;
    // With few spindown rows a block's table row serves few templates, and the
    // ring can be bound by its copies: AUTO then also weighs the far-field form
    // (64-byte positions against the sinc form's 96) and blocks of 4 close sky
    // points (one window for all four).  Measured on GB300, 2048 sky x 900 f x
    // 1600 SFTs, one spindown, one sky point a block: sinc 18.6 ms, far field
    // 14.4 ms; with two spindowns they tie.
    const bool few_rows = c->n_fdot <= 2;
    std::vector<bool> forms;
    if (sinc_ok) forms.push_back(true);
    if (!sinc_ok || (c->opts.algo == FSTAT_ALGO_AUTO && L == 2 && few_rows && tw != 3 && tw != 5))
        forms.push_back(false);
    // L = 1 (P = 8) runs the ring in the sinc form only, with plain tables
    const bool ring_l = L == 2 || (L == 1 && sinc_ok && !c->have_cov);
    if (found && ring_l && c->fdot_uniform && (tw == 0 || tw >= 9 || (sinc_ok && L == 2 && (tw == 3 || tw == 5)))) {
        // M = 5 with 8 stages measured fastest on GB300 (1105 ms on the workunit; M = 7: 1139 ms).
        // For L = 1, M = 1 competes: narrow banks leave an M = 5 lane-group's lanes idle.
        std::vector<int> Mr = {5};
        if (L == 1) Mr = {5, 1};
        if (c->opts.tile_m > 0) Mr = {c->opts.tile_m};
        int nwc0 = c->opts.tile_warps ? c->opts.tile_warps - 1 : 10;   // the last warp produces
        // every lane-group needs all P of its threads: P must divide the compute
        // warps (P = 4 takes 8 compute warps unless the caller fixed them)
        if (nwc0 % P != 0 && !c->opts.tile_warps && 8 % P == 0) nwc0 = 8;
        double best_r = 1e300;
        if (nwc0 % P != 0) Mr.clear();
        // blocks of 4 and 2 compute warps (tile_warps 5 and 3) only on request:
        // on GB300 the 10-warp block was faster on every bank measured, by 20-60 %
        // on banks of 1-16 spindowns where the cost model favoured the small ones
        const std::vector<int> nwcs = {nwc0};
        // blocks of 4 sky points whose windows lie within 24 bins (the window widens
        // by that much; the cost model weighs it): 4 consecutive ones of the bank,
        // else 4 consecutive ones of a neighbour order (meta and bases are then
        // written in that order); batched workunits only where a persistent form
        // exists (L = 2)
        std::vector<int> SRs = {1};
        double spread4 = 0.0;
        bool use_perm = false;
        if (few_rows && !c->have_cov && (!c->batch_member || L == 2) && c->n_sky >= 8) {
            spread4 = sky_spread_bins(c, 4);
            if (spread4 > 24.0) {
                if (c->h_order.empty()) {
                    c->h_order = sky_neighbour_order(c);
                    c->order_spread4 = sky_spread_bins(c, 4, &c->h_order);
                }
                if (c->order_spread4 <= 24.0) {
                    spread4 = c->order_spread4;
                    use_perm = true;
                }
            }
            if (spread4 <= 24.0) SRs.push_back(4);
        }
        // one spindown and one sky point a block: the far-field form (measured; the
        // compute model overrates the idle warps of its wide blocks)
        const bool one_row_far = forms.size() > 1 && c->n_fdot == 1;
        for (const bool sinc : forms)
        for (const int SR : SRs)
        for (int M_ : Mr)
        for (int nwc : nwcs) {
            if (nwc % P != 0) continue;
            if (sinc && SR == 1 && one_row_far) continue;
            int fid = -1;
            for (int i = 0; i < kNumFar; ++i)
                if (kFarVariants[i].ring == nwc && kFarVariants[i].M == M_ && kFarVariants[i].L == L &&
                    kFarVariants[i].sinc == sinc && kFarVariants[i].cov == c->have_cov && !kFarVariants[i].rows &&
                    !kFarVariants[i].minb && std::max(1, kFarVariants[i].sr) == SR)
                    fid = i;
            if (fid < 0) continue;
            const int PM = P * M_;
            const int lg_cta = 32 * nwc / P;
            const int lg_max = std::min((c->n_f + PM - 1) / PM, lg_cta);
            const int rows = SR * c->n_fdot;   // rows of a block: (sky point, spindown)
            for (int lg_row = 1; lg_row <= lg_max; ++lg_row) {
                // a quarter-warp (8 lane-groups) must not straddle two rows:
                // its lanes' records then sit 5 positions apart and read conflict-free
                // (a straddling layout measured 23 % slower on the workunit)
                if (rows > 1 && lg_row % 8 != 0 && lg_row < lg_max) continue;
                const int col_w = lg_row * PM;
                const int n_col = (c->n_f + col_w - 1) / col_w;
                const int w_pairs = std::max(pairs_needed(c, col_w, 8) + (SR > 1 ? (int)std::ceil(spread4) : 0),
                                             (M_ - 1) * L + 2 * 8 + 2);
                int hf = (w_pairs + 1) / 2;
                hf += ((4 - hf % 8) + 8) % 8;
                const int w_tab = L == 2 ? 2 * hf : w_pairs;
                // live warps of every block (a block's idle warps still hold its place on
                // the SM), for one block row of SR sky points
                double live = 0.0, blocks = 0.0;
                int chunks_max = 0;
                for (int col = 0; col < n_col; ++col) {
                    const int width = std::min(col_w, c->n_f - col * col_w);
                    const int Gc = (width + PM - 1) / PM;
                    const long long LG = (long long)rows * Gc;
                    const int chunks = (int)((LG + lg_cta - 1) / lg_cta);
                    chunks_max = std::max(chunks_max, chunks);
                    for (int k = 0; k < chunks; ++k) {
                        const long long lgs = std::min<long long>(lg_cta, LG - (long long)k * lg_cta);
                        live += (double)((lgs + 31) / 32 * P);
                        blocks += 1.0;
                    }
                }
                const int S_hi = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 8;
                const int S_lo = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 3;
                for (int S = S_hi; S >= S_lo; --S) {
                    const size_t smem = ring_smem(S, w_tab, sinc, SR).total;
                    if (smem > 220 * 1024) continue;
                    // Compute ~ work / concurrency: the kernel saturates its SM at
                    // about 20 live compute warps; fewer resident live warps (blocks
                    // per SM limited by shared memory, threads or ~80 registers a
                    // thread) leave it latency-bound.  Per live warp and SFT ~40
                    // instructions of set-up and ~50 per template; fewer stages
                    // leave less slack between warps; the far-field form takes 1.5x
                    // the sinc form's time per template (1106 against 731 ms on the
                    // workunit).  Staging: the table rows copied per SFT at ~17.7 TB/s
                    // (L2 to shared memory, measured with one spindown).  The time
                    // is the larger of the two, in ms per sky point and SFT (compute
                    // calibrated on the workunit: 731 ms for 10 000 x 2400).
                    const int threads = 32 * (nwc + 1);
                    int resident = (int)((227 * 1024) / (smem + 1024));
                    resident = std::min(resident, 2048 / threads);
                    resident = std::min(resident, 65536 / (80 * threads));
                    if (resident < 1) continue;
                    const double conc = std::min(20.0, resident * live / blocks);
                    const double work = live * 32.0 * (40.0 + 50.0 * M_) * (1.0 + 0.2 / S);
                    const double t_comp = work / conc * 5.26e-10 * (sinc ? 1.0 : 1.5) / SR;
                    const double t_copy = blocks * w_pairs * (sinc ? 96.0 : 64.0) / 17.7e9 / SR;
                    const double cost = std::max(t_comp, t_copy);
                    if (cost < best_r * 0.999) {
                        best_r = cost;
                        best = Plan{};
                        best.P = P;
                        best.L = L;
                        best.M = M_;
                        best.W = nwc + 1;
                        best.C = S;
                        best.lg_row = lg_row;
                        best.lg_cta = lg_cta;
                        best.n_col = n_col;
                        best.chunks_per_col = chunks_max;
                        best.w_pairs = w_pairs;
                        best.w_tab = w_tab;
                        best.variant = fid;
                        best.far = true;
                        best.ring = true;
                        best.sinc = sinc;
                        best.sky_rows = SR;
                        best.sky_perm = SR > 1 && use_perm;
                        best.smem = smem;
                        best.grid = (long long)((c->n_sky + SR - 1) / SR) * n_col * chunks_max;
                        have_ring = true;
                    }
                }
            }
        }
        if (have_ring) return true;
    }
    if (c->have_cov) return false;   // the rounds staging has no coverage path
    std::vector<int> Ms;
    // M = 5 measured fastest on GB300 (the wider tiles give up round size to
    // shared memory); the autotuner also tries 7 and 9.  M = 1 competes in the
    // cost model: on narrow bands with P = 8 (L = 1) an M = 5 lane-group spans
    // 40 frequencies and most of a block's lanes would idle.
    if (found) Ms = {5, 1};
    else Ms = {1};
    if (c->opts.tile_m > 0) Ms = {c->opts.tile_m};
    double best_cost = 1e300;
    bool have = false;
    for (int M_ : Ms) {
        const int Lq = (M_ == 1) ? 1 : L;
        if (M_ > 1 && !found) continue;
        int fid = -1;
        for (int i = 0; i < kNumFar; ++i)
            if (kFarVariants[i].ring == 0 && !kFarVariants[i].sinc && !kFarVariants[i].rows && kFarVariants[i].M == M_ &&
                kFarVariants[i].L == Lq)
                fid = i;
        if (fid < 0) continue;
        const int Pv = found ? P : 1;
        const int PM = Pv * M_;
        const int lg_full = (c->n_f + PM - 1) / PM;
        const size_t smem_cap = 110 * 1024;
        for (int W = Pv; W <= 10; W += Pv) {
            if (c->opts.tile_warps > 0 && W != c->opts.tile_warps) continue;
            const int lg_cta = 32 * W / Pv;
            const int lg_max = std::min(lg_full, lg_cta);
            for (int lg_row = 1; lg_row <= lg_max; ++lg_row) {
                const int col_w = lg_row * PM;
                const int n_col = (c->n_f + col_w - 1) / col_w;
                const int w_pairs = std::max(pairs_needed(c, col_w, 8), (M_ - 1) * Lq + 2 * 8 + 2);
                int w_tab = w_pairs;
                if (Lq == 2) {
                    int hf = (w_pairs + 1) / 2;
                    hf += ((4 - hf % 8) + 8) % 8;
                    w_tab = 2 * hf;
                }
                int C = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 4;
                size_t smem = farpoly_smem(C, w_tab, c->n_fdot).total;
                while (C > 1 && smem > smem_cap) {
                    --C;
                    smem = farpoly_smem(C, w_tab, c->n_fdot).total;
                }
                if (smem > 220 * 1024) continue;
                double cost = 0.0;
                int chunks_max = 0;
                for (int col = 0; col < n_col; ++col) {
                    const int width = std::min(col_w, c->n_f - col * col_w);
                    const int Gc = (width + PM - 1) / PM;
                    const long long LG = (long long)c->n_fdot * Gc;
                    const int chunks = (int)((LG + lg_cta - 1) / lg_cta);
                    chunks_max = std::max(chunks_max, chunks);
                    for (int k = 0; k < chunks; ++k) {
                        const long long lgs = std::min<long long>(lg_cta, LG - (long long)k * lg_cta);
                        const long long warps = (lgs + 31) / 32 * Pv;
                        // the barrier of each round idles the block's warps: ~30 % of a round's work / C
                        cost += ((double)warps * 32.0 * (40.0 + 50.0 * M_) + (double)w_pairs * 4.0 * 8.0) *
                                (1.0 + 0.3 / C);
                    }
                }
                if (cost < best_cost * 0.999 && !have_ring) {
                    best_cost = cost;
                    best = Plan{};
                    best.P = Pv;
                    best.L = Lq;
                    best.M = M_;
                    best.W = W;
                    best.C = C;
                    best.lg_row = lg_row;
                    best.lg_cta = lg_cta;
                    best.n_col = n_col;
                    best.chunks_per_col = chunks_max;
                    best.w_pairs = w_pairs;
                    best.w_tab = w_tab;
                    best.w_raw = 0;
                    best.variant = fid;
                    best.far = true;
                    best.smem = smem;
                    best.grid = (long long)c->n_sky * n_col * chunks_max;
                    have = true;
                }
            }
        }
    }
    return have;
}

int make_plan(fstat_ctx* c, Plan& out) {
    const int D = c->opts.dterms;
    const int kahan = c->opts.kahan ? 1 : 0;
    const double dk_nom = c->df * c->T;
    int P = 1, L = 1;
    bool found = false;
    if (D == 8) {
        const int Ls[2] = {2, 1};
        const int Ps[4] = {1, 2, 4, 8};
        for (int li = 0; li < 2 && !found; ++li)
            for (int pi = 0; pi < 4 && !found; ++pi)
                if (std::fabs(Ps[pi] * dk_nom - Ls[li]) <= 1e-6 * Ls[li]) {
                    P = Ps[pi];
                    L = Ls[li];
                    found = true;
                }
    }
    if (far_eligible(c)) {
        if (make_far_plan(c, P, L, found, out)) return FSTAT_OK;
        if (c->opts.algo == FSTAT_ALGO_FARPOLY)
            return fail(c, FSTAT_EINVAL, "no far-field tile plan fits this template bank");
    }
    std::vector<int> Ms;
    if (found) {
        // odd M keeps neighbouring threads' pair-table rows on distinct banks
        // M = 7 measured fastest on GB300 for L = 2 (M = 9 spills at 96 registers)
        if (kahan) Ms = {5};
        else if (L == 2) Ms = {7, 5};
        else Ms = {7, 9};
    } else {
        P = 1;
        L = 1;
        Ms = {1};
    }
    if (c->opts.tile_m > 0) Ms = {c->opts.tile_m};
    const int Dv = (D == 8) ? 8 : 0;
    double best_cost = 1e300;
    Plan best;
    bool have = false;
    for (int M_ : Ms) {
        const int Lq = (Dv == 0 || M_ == 1) ? 1 : L;
        const int vid = variant_id(Dv, (Dv == 0 ? 1 : M_), Lq, kahan);
        if (vid < 0) continue;
        const int Mv = kVariants[vid].M, Lv = kVariants[vid].L;
        const int Pv = (Dv == 0 || Mv == 1) && !found ? 1 : P;
        const int PM = Pv * Mv;
        const int lg_full = (c->n_f + PM - 1) / PM;
        for (int W = Pv; W <= 10; W += Pv) {
            if (c->opts.tile_warps > 0 && W != c->opts.tile_warps) continue;
            const int lg_cta = 32 * W / Pv;
            const int lg_max = std::min(lg_full, lg_cta);
            for (int lg_row = 1; lg_row <= lg_max; ++lg_row) {
                const int col_w = lg_row * PM;
                const int n_col = (c->n_f + col_w - 1) / col_w;
                // the table must hold at least one thread's full window set
                const int w_pairs = std::max(pairs_needed(c, col_w, D), (Mv - 1) * Lv + 2 * D + 2);
                int w_tab = w_pairs;
                if (Lv == 2) {   // two parity halves, each offset 4 mod 8 slots from the other
                    int hf = (w_pairs + 1) / 2;
                    hf += ((4 - hf % 8) + 8) % 8;
                    w_tab = 2 * hf;
                }
                const int G = (c->opts.bins_form == FSTAT_BINS_C64) ? 2 : 4;
                const int raw_b = (c->opts.bins_form == FSTAT_BINS_C64) ? 8 : 4;
                const int w_raw = ((w_pairs + G + G - 1) / G) * G;
                int C = c->opts.sft_chunk > 0 ? c->opts.sft_chunk : 8;
                size_t smem = dirichlet_smem(C, w_tab, w_raw, c->n_fdot, raw_b).total;
                while (C > 1 && smem > 110 * 1024) {
                    --C;
                    smem = dirichlet_smem(C, w_tab, w_raw, c->n_fdot, raw_b).total;
                }
                if (smem > 220 * 1024) continue;
                double cost = 0.0;
                int chunks_max = 0;
                for (int col = 0; col < n_col; ++col) {
                    const int width = std::min(col_w, c->n_f - col * col_w);
                    const int Gc = (width + PM - 1) / PM;
                    const long long LG = (long long)c->n_fdot * Gc;
                    const int chunks = (int)((LG + lg_cta - 1) / lg_cta);
                    chunks_max = std::max(chunks_max, chunks);
                    for (int k = 0; k < chunks; ++k) {
                        const long long lgs = std::min<long long>(lg_cta, LG - (long long)k * lg_cta);
                        const long long warps = (lgs + 31) / 32 * Pv;
                        // per thread and SFT: ~40 instructions of set-up and M + 7 table loads,
                        // then ~75 per template; staging ~14 per staged pair; round overhead
                        const double per_thread = 40.0 + (Mv + 7) + 75.0 * Mv;
                        cost += (double)warps * 32.0 * per_thread + (double)w_pairs * 14.0 + 400.0;
                    }
                }
                if (cost < best_cost * 0.999) {
                    best_cost = cost;
                    best.P = Pv;
                    best.L = Lv;
                    best.M = Mv;
                    best.W = W;
                    best.C = C;
                    best.lg_row = lg_row;
                    best.lg_cta = lg_cta;
                    best.n_col = n_col;
                    best.chunks_per_col = chunks_max;
                    best.w_pairs = w_pairs;
                    best.w_tab = w_tab;
                    best.w_raw = w_raw;
                    best.variant = vid;
                    best.smem = smem;
                    best.grid = (long long)c->n_sky * n_col * chunks_max;
                    have = true;
                }
            }
        }
    }
    if (!have) return fail(c, FSTAT_EINVAL, "no Dirichlet tile plan fits this template bank");
    out = best;
    return FSTAT_OK;
}

bool all_finite(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

__global__ void finite_check_kernel(const float* v, long long n, int* bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        if (!isfinite(v[i])) atomicOr(bad, 1);
}

__global__ void fill_kernel(float* v, long long n, float x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = x;
}

int ensure_topk(fstat_ctx* c) {
    const int k = c->opts.topk;
    if (k <= 0) return FSTAT_OK;
    if (c->tw_k >= k) return FSTAT_OK;
    TopkWork& w = c->tw;
    cudaFree(w.hist);
    cudaFree(w.state);
    cudaFree(w.tie_count);
    cudaFree(w.cand_idx);
    cudaFree(w.cand_val);
    cudaFree(w.n_cand);
    cudaFree(w.out_idx);
    cudaFree(w.out_val);
    w = TopkWork{};
    w.n_blocks = 1024;
    CUDA_TRY(c, cudaMalloc(&w.hist, sizeof(unsigned int) * 3 * 2048));
    CUDA_TRY(c, cudaMalloc(&w.state, sizeof(unsigned int) * 16));
    CUDA_TRY(c, cudaMalloc(&w.tie_count, sizeof(unsigned int) * w.n_blocks));
    CUDA_TRY(c, cudaMalloc(&w.cand_idx, sizeof(long long) * k));
    CUDA_TRY(c, cudaMalloc(&w.cand_val, sizeof(float) * k));
    CUDA_TRY(c, cudaMalloc(&w.n_cand, sizeof(unsigned int)));
    CUDA_TRY(c, cudaMalloc(&w.out_idx, sizeof(long long) * k));
    CUDA_TRY(c, cudaMalloc(&w.out_val, sizeof(float) * k));
    c->tw_k = k;
    return FSTAT_OK;
}

int sync_ctx(fstat_ctx* c) {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "stream synchronize: %s", cudaGetErrorString(e));
    return FSTAT_OK;
}

// After a synchronised read-back: the error code for the device flags of the
// last compute (bit 2: a bounded wait gave up; bit 0: a window left the
// staged range).  The outputs were written either way.
int flag_status(fstat_ctx* c) {
    int h = 0;
    CUDA_TRY(c, cudaMemcpy(&h, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h & 4) return fail(c, FSTAT_ETIMEOUT, "a bounded device wait gave up: 2F of some blocks is invalid");
    if (h & 1) return fail(c, FSTAT_ERANGE, "a template window left the staged SFT range (clamped)");
    return FSTAT_OK;
}

// The bins the path reads: the whitened copy when the noise floor is on.
const float2* work_bins(const fstat_ctx* c) { return c->nf_half > 0 ? c->d_bins_w : c->d_bins; }

int refresh_sft_state(fstat_ctx* c, cudaStream_t s) {
    if (!c->sft_dirty) return FSTAT_OK;
    std::vector<double> ts;
    std::vector<int> det_of;
    fstat_detector g[kMaxDet];
    std::memset(g, 0, sizeof(g));
    for (int d = 0; d < kMaxDet; ++d) {
        if (!c->det[d].set) continue;
        g[d] = c->det[d].g;
        for (double t : c->det[d].t_start) {
            ts.push_back(t);
            det_of.push_back(d);
        }
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_tstart, ts.data(), ts.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(c->d_det_of, det_of.data(), det_of.size() * sizeof(int), cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, launch_sft_state(c->d_tstart, c->d_det_of, g, c->n_sft, c->T, c->d_state, s));
    c->launches += 2;   // detector state + scale fill / quantisation
    if (c->nf_half > 0) {
        int rc;
        if ((rc = grow(c, &c->d_bins_w, c->cap_bins_w, (size_t)c->n_sft * c->row)) != FSTAT_OK) return rc;
        if ((rc = grow(c, &c->d_floor, c->cap_floor, (size_t)c->n_sft * c->n_bins)) != FSTAT_OK) return rc;
        if ((rc = grow(c, &c->d_sbar, c->cap_sbar, (size_t)c->n_sft)) != FSTAT_OK) return rc;
        if ((rc = grow(c, &c->d_weight, c->cap_weight, (size_t)c->n_sft)) != FSTAT_OK) return rc;
        CUDA_TRY(c, launch_noise_floor(c->d_bins, c->row, c->n_sft, c->n_bins, c->nf_half, c->d_floor, c->d_bins_w,
                                       c->d_sbar, c->d_weight, s));
        c->launches += 2;
    }
    if (c->opts.bins_form == FSTAT_BINS_C64) {
        fill_kernel<<<64, 256, 0, s>>>(c->d_scale, c->n_sft, 1.0f);
        CUDA_TRY(c, cudaGetLastError());
    } else {
        CUDA_TRY(c, launch_quantize(work_bins(c), c->row, c->n_sft, c->n_bins, c->opts.bins_form, c->d_bins16,
                                    c->d_scale, s));
    }
    // the host vectors are copied asynchronously: wait before they go out of scope
    CUDA_TRY(c, cudaStreamSynchronize(s));
    c->sft_dirty = false;
    c->tab_dirty = true;
    return FSTAT_OK;
}

}  // namespace

extern "C" {

const char* fstat_version(void) { return "libfstat 0.1 (sm_103a)"; }

int fstat_create(fstat_ctx** out, int device, const fstat_opts* opts) {
    if (!out) return FSTAT_EINVAL;
    *out = nullptr;
    fstat_opts o{};
    o.dterms = 8;
    o.bins_form = FSTAT_BINS_C64;
    o.topk = 1000;
    if (opts) o = *opts;
    if (o.dterms < 1 || o.dterms > 64) return FSTAT_EINVAL;
    if (o.topk < 0 || o.topk > 16384) return FSTAT_EINVAL;
    if (o.bins_form < 0 || o.bins_form > 2) return FSTAT_EINVAL;
    if (o.tile_m < 0 || o.tile_warps < 0 || o.tile_warps > 11 || o.sft_chunk < 0 || o.sft_chunk > 64)
        return FSTAT_EINVAL;
    if (o.algo < FSTAT_ALGO_AUTO || o.algo > FSTAT_ALGO_SINCPAIRS) return FSTAT_EINVAL;
    if ((o.algo == FSTAT_ALGO_FARPOLY || o.algo == FSTAT_ALGO_SINCPOLY || o.algo == FSTAT_ALGO_SINCROWS ||
         o.algo == FSTAT_ALGO_SINCPAIRS) &&
        (o.dterms != 8 || o.kahan))
        return FSTAT_EINVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return FSTAT_ECUDA;
    fstat_ctx* c = new fstat_ctx();
    c->device = device;
    c->opts = o;
    c->gam = far_gamma();
    c->sgam = sinc_gamma();
    if (set_device(c) != FSTAT_OK) {
        delete c;
        return FSTAT_ECUDA;
    }
    if (cudaMalloc(&c->d_err, sizeof(int) * 4) != cudaSuccess) {
        delete c;
        return FSTAT_ENOMEM;
    }
    cudaMemset(c->d_err, 0, sizeof(int) * 4);
    for (int i = 0; i < kTimedRing; ++i) {
        cudaEventCreate(&c->ev_a[i]);
        cudaEventCreate(&c->ev_b[i]);
        cudaEventCreate(&c->ev_c[i]);
        cudaEventCreate(&c->ev_d[i]);
    }
    *out = c;
    return FSTAT_OK;
}

int fstat_batch_clear(fstat_ctx* c);

void fstat_destroy(fstat_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaDeviceSynchronize();
    fstat_batch_clear(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (cudaStream_t st : c->side_streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : c->side_events) cudaEventDestroy(ev);
    if (c->bev0) cudaEventDestroy(c->bev0);
    if (c->bev1) cudaEventDestroy(c->bev1);
    void* ptrs[] = {c->d_fstart, c->d_base, c->d_bins, c->d_bins16, c->d_scale, c->d_state, c->d_tstart, c->d_det_of, c->d_sky,
                    c->d_fdot, c->d_meta, c->d_kh0, c->d_ph0, c->d_abcd, c->d_comb, c->d_twoF, c->d_err,
                    c->tw.hist, c->tw.state, c->tw.tie_count, c->tw.cand_idx, c->tw.cand_val, c->tw.n_cand,
                    c->tw.out_idx, c->tw.out_val, c->d_inj_work, c->d_sig, c->d_ptab, c->d_pcoef,
                    c->d_bins_w, c->d_floor, c->d_sbar, c->d_weight, c->d_cov, c->d_comb_j, c->d_slide_seg, c->d_slide_A,
                    c->d_slide_B, c->d_slide_out, c->d_perm, c->d_rank};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int i = 0; i < kTimedRing; ++i) {
        cudaEventDestroy(c->ev_a[i]);
        cudaEventDestroy(c->ev_b[i]);
        cudaEventDestroy(c->ev_c[i]);
        cudaEventDestroy(c->ev_d[i]);
    }
    delete c;
}

const char* fstat_last_error(const fstat_ctx* c) { return c ? c->err.c_str() : ""; }

int fstat_set_coverage(fstat_ctx* c, const int32_t* j_lo, const int32_t* j_hi, int32_t n_sft) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!j_lo && !j_hi) {
        c->have_cov = false;
        c->plan_valid = false;
        c->computed = false;
        return FSTAT_OK;
    }
    if (!j_lo || !j_hi) return fail(c, FSTAT_EINVAL, "j_lo and j_hi must both be given or both be null");
    if (!c->have_sfts) return fail(c, FSTAT_ESTATE, "load SFTs first");
    if (n_sft != c->n_sft) return fail(c, FSTAT_EINVAL, "n_sft %d != loaded SFTs %d", n_sft, c->n_sft);
    std::vector<int2> h(n_sft);
    for (int i = 0; i < n_sft; ++i) {
        if (j_lo[i] > j_hi[i]) return fail(c, FSTAT_EINVAL, "SFT %d: j_lo > j_hi", i);
        h[i] = make_int2(j_lo[i], j_hi[i]);
    }
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    if (c->d_cov) cudaFree(c->d_cov);
    c->d_cov = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_cov, (size_t)n_sft * sizeof(int2)));
    CUDA_TRY(c, cudaMemcpy(c->d_cov, h.data(), (size_t)n_sft * sizeof(int2), cudaMemcpyHostToDevice));
    c->have_cov = true;
    c->plan_valid = false;
    c->computed = false;
    return FSTAT_OK;
}

int fstat_stackslide(fstat_ctx* const* seg, int32_t n_seg, double f0, double df, int32_t n_f, double t_ref,
                     float* out, int64_t* n_outside, void* cuda_stream) {
    if (!seg || n_seg < 1 || n_seg > FSTAT_SEMI_MAX_SEG || !seg[0]) return FSTAT_EINVAL;
    fstat_ctx* c = seg[0];
    c->err.clear();
    if (!out) return fail(c, FSTAT_EINVAL, "null output");
    if (n_f < 1) return fail(c, FSTAT_EINVAL, "n_f must be >= 1");
    if (!std::isfinite(f0) || !(df > 0) || !std::isfinite(df) || !std::isfinite(t_ref))
        return fail(c, FSTAT_EINVAL, "f0, df, t_ref must be finite and df > 0");
    std::vector<SlideSeg> h(n_seg);
    for (int s = 0; s < n_seg; ++s) {
        const fstat_ctx* g = seg[s];
        if (!g) return fail(c, FSTAT_EINVAL, "segment %d is null", s);
        if (g->device != c->device) return fail(c, FSTAT_EINVAL, "segment %d is on another device", s);
        if (!g->have_templates || !g->computed || !g->d_twoF)
            return fail(c, FSTAT_ESTATE, "segment %d has no computed 2F", s);
        if (g->n_sky != c->n_sky || g->h_sky != c->h_sky) return fail(c, FSTAT_EINVAL, "segment %d: other sky list", s);
        if (g->h_fdot != c->h_fdot) return fail(c, FSTAT_EINVAL, "segment %d: other spindown list", s);
        const double r = df / g->df;
        if (!(r >= 0x1p-20 && r <= 0x1p20)) return fail(c, FSTAT_EINVAL, "segment %d: df / df_s outside 2^-20..2^20", s);
        h[s] = SlideSeg{g->d_twoF, (long long)g->n_f, g->f0, g->df, g->t_ref};
    }
    // B = df / df_s rounds to exactly 1 on the device iff it does here (IEEE division)
    bool unit = true;
    for (int s = 0; s < n_seg; ++s) unit = unit && df / h[s].df == 1.0 && h[s].n_f < (1LL << 30);
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int rc;
    const int n_fdot = c->n_fdot;
    if ((rc = grow(c, &c->d_slide_seg, c->cap_slide_seg, (size_t)n_seg)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_slide_A, c->cap_slide_A, (size_t)n_seg * n_fdot)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_slide_B, c->cap_slide_B, (size_t)n_seg)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_slide_out, c->cap_slide_out, 1)) != FSTAT_OK) return rc;
    // the segment table and the fixed-point slide constants are rebuilt only
    // when the segments or the grid change
    bool same = c->slide_last.size() == h.size() && c->slide_grid[0] == f0 && c->slide_grid[1] == df &&
                c->slide_grid[2] == t_ref && c->slide_fdot == c->h_fdot && c->slide_A_at == c->d_slide_A;
    for (int s = 0; same && s < n_seg; ++s)
        same = h[s].twoF == c->slide_last[s].twoF && h[s].n_f == c->slide_last[s].n_f && h[s].f0 == c->slide_last[s].f0 &&
               h[s].df == c->slide_last[s].df && h[s].t == c->slide_last[s].t;
    if (!same) {
        c->slide_last.clear();   // invalid until the new table is in place
        CUDA_TRY(c, cudaMemcpyAsync(c->d_slide_seg, h.data(), (size_t)n_seg * sizeof(SlideSeg), cudaMemcpyHostToDevice,
                                    st));
    }
    if (n_outside) CUDA_TRY(c, cudaMemsetAsync(c->d_slide_out, 0, sizeof(unsigned long long), st));
    CUDA_TRY(c, launch_stackslide(c->d_slide_seg, n_seg, c->d_fdot, n_fdot, f0, df, t_ref, c->d_slide_A, c->d_slide_B,
                                  !same, unit, (long long)c->n_sky * n_fdot, n_f, out,
                                  n_outside ? c->d_slide_out : nullptr, st));
    c->launches += same ? 1 : 2;
    if (!same) {
        c->slide_last = h;
        c->slide_fdot = c->h_fdot;
        c->slide_A_at = c->d_slide_A;
        c->slide_grid[0] = f0;
        c->slide_grid[1] = df;
        c->slide_grid[2] = t_ref;
    }
    if (n_outside) {
        unsigned long long v = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&v, c->d_slide_out, sizeof(v), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(c, cudaStreamSynchronize(st));
        *n_outside = (int64_t)v;
    }
    return FSTAT_OK;
}

int fstat_set_sfts(fstat_ctx* c, int32_t det_index, const fstat_detector* det, double Tsft, int64_t k_lo,
                   int32_t n_bins, int32_t n_sft, const double* t_start, const float* bins, int32_t mem) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (det_index < 0 || det_index >= kMaxDet) return fail(c, FSTAT_EINVAL, "det_index %d out of 0..7", det_index);
    if (!det || !t_start || !bins) return fail(c, FSTAT_EINVAL, "null pointer argument");
    if (!(Tsft > 0) || !std::isfinite(Tsft)) return fail(c, FSTAT_EINVAL, "Tsft must be finite and > 0");
    if (n_bins < 2) return fail(c, FSTAT_EINVAL, "n_bins must be >= 2");
    if (n_sft < 1 || n_sft > 32768) return fail(c, FSTAT_EINVAL, "n_sft must be in 1..32768");
    if (mem != FSTAT_MEM_HOST && mem != FSTAT_MEM_DEVICE) return fail(c, FSTAT_EINVAL, "mem must be 0 or 1");
    if (!std::isfinite(det->lat_rad) || !std::isfinite(det->lon_rad) || !std::isfinite(det->xarm_az_rad))
        return fail(c, FSTAT_EINVAL, "non-finite detector geometry");
    if (!all_finite(t_start, n_sft)) return fail(c, FSTAT_EINVAL, "non-finite SFT start time");
    if (k_lo < 0 || k_lo > (1LL << 30)) return fail(c, FSTAT_EINVAL, "k_lo out of range");
    bool others = false;
    for (int d = 0; d < kMaxDet; ++d) others |= (d != det_index && c->det[d].set);
    if (others && (Tsft != c->T || k_lo != c->k_lo || n_bins != c->n_bins))
        return fail(c, FSTAT_EINVAL, "all detectors must share Tsft, k_lo and n_bins");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    if (n_bins > (1 << 24)) return fail(c, FSTAT_EINVAL, "n_bins too large");
    // new layout: detectors in index order, rows padded to 8 elements
    const long long row = ((long long)n_bins + 7) & ~7LL;
    int total = 0;
    int first_of[kMaxDet];
    for (int d = 0; d < kMaxDet; ++d) {
        first_of[d] = total;
        if (d == det_index) total += n_sft;
        else if (c->det[d].set) total += (int)c->det[d].t_start.size();
    }
    if (total > 65535) return fail(c, FSTAT_EINVAL, "more than 65535 SFTs in one context");
    // host staging for device input: validate values
    std::vector<float> hb;
    const float* src = bins;
    const size_t n_el = (size_t)n_sft * n_bins * 2;
    if (mem == FSTAT_MEM_HOST) {
        for (size_t i = 0; i < n_el; ++i)
            if (!std::isfinite(bins[i])) return fail(c, FSTAT_EINVAL, "non-finite SFT bin at %zu", i);
    }
    // new device store; copy kept detectors over
    float2* nb = nullptr;
    CUDA_TRY(c, cudaMalloc(&nb, (size_t)total * row * sizeof(float2)));
    CUDA_TRY(c, cudaMemsetAsync(nb, 0, (size_t)total * row * sizeof(float2), c->stream));
    int old_first = 0;
    for (int d = 0; d < kMaxDet; ++d) {
        const int n_old = c->det[d].set ? (int)c->det[d].t_start.size() : 0;
        if (d != det_index && n_old) {
            CUDA_TRY(c, cudaMemcpyAsync(nb + (size_t)first_of[d] * row, c->d_bins + (size_t)old_first * c->row,
                                        (size_t)n_old * row * sizeof(float2), cudaMemcpyDeviceToDevice, c->stream));
        }
        old_first += n_old;
    }
    CUDA_TRY(c, cudaMemcpy2DAsync(nb + (size_t)first_of[det_index] * row, row * sizeof(float2), src,
                                  (size_t)n_bins * sizeof(float2), (size_t)n_bins * sizeof(float2), n_sft,
                                  mem == FSTAT_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice,
                                  c->stream));
    if (mem == FSTAT_MEM_DEVICE) {
        int* bad = c->d_err + 3;
        CUDA_TRY(c, cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
        finite_check_kernel<<<256, 256, 0, c->stream>>>(bins, (long long)n_el, bad);
        CUDA_TRY(c, cudaGetLastError());
        c->launches += 1;
        int hbad = 0;
        CUDA_TRY(c, cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        if (hbad) {
            cudaFree(nb);
            return fail(c, FSTAT_EINVAL, "non-finite SFT bin in device input");
        }
    }
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (c->d_bins) cudaFree(c->d_bins);
    c->d_bins = nb;
    c->row = row;
    c->det[det_index].set = true;
    c->det[det_index].g = *det;
    c->det[det_index].t_start.assign(t_start, t_start + n_sft);
    c->n_sft = total;
    c->T = Tsft;
    c->k_lo = k_lo;
    c->n_bins = n_bins;
    // per-SFT buffers
    if (c->d_state) cudaFree(c->d_state);
    if (c->d_tstart) cudaFree(c->d_tstart);
    if (c->d_det_of) cudaFree(c->d_det_of);
    if (c->d_scale) cudaFree(c->d_scale);
    if (c->d_bins16) cudaFree(c->d_bins16);
    c->d_state = nullptr;
    c->d_tstart = nullptr;
    c->d_det_of = nullptr;
    c->d_scale = nullptr;
    c->d_bins16 = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_state, (size_t)total * sizeof(SftState)));
    CUDA_TRY(c, cudaMalloc(&c->d_tstart, (size_t)total * sizeof(double)));
    CUDA_TRY(c, cudaMalloc(&c->d_det_of, (size_t)total * sizeof(int)));
    CUDA_TRY(c, cudaMalloc(&c->d_scale, (size_t)total * sizeof(float)));
    if (c->opts.bins_form != FSTAT_BINS_C64)
        CUDA_TRY(c, cudaMalloc(&c->d_bins16, (size_t)total * row * 4));
    c->have_sfts = true;
    c->sft_dirty = true;
    c->plan_valid = false;
    c->computed = false;
    c->have_cov = false;   // coverage is per SFT index: a new SFT set clears it
    return FSTAT_OK;
}

int fstat_set_templates(fstat_ctx* c, const double* sky, int32_t n_sky, double f0, double df, int32_t n_f,
                        const double* fdot, int32_t n_fdot, double t_ref) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!sky || !fdot) return fail(c, FSTAT_EINVAL, "null pointer argument");
    if (n_sky < 1 || n_f < 1 || n_fdot < 1) return fail(c, FSTAT_EINVAL, "template counts must be >= 1");
    if (n_fdot > 64) return fail(c, FSTAT_EINVAL, "at most 64 spindowns per bank");
    if (!(df > 0) || !std::isfinite(df) || !std::isfinite(f0) || !(f0 > 0) || !std::isfinite(t_ref))
        return fail(c, FSTAT_EINVAL, "f0, df must be finite and > 0, t_ref finite");
    if (!all_finite(sky, 2 * (size_t)n_sky) || !all_finite(fdot, n_fdot))
        return fail(c, FSTAT_EINVAL, "non-finite sky position or spindown");
    const double nt = (double)n_sky * n_fdot * n_f;
    if (nt > (double)(1LL << 40)) return fail(c, FSTAT_EINVAL, "more than 2^40 templates");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    c->h_sky.assign(sky, sky + 2 * (size_t)n_sky);
    c->h_fdot.assign(fdot, fdot + n_fdot);
    c->h_order.clear();
    c->order_spread4 = -1.0;
    c->perm_on_device = false;
    if (c->d_sky) cudaFree(c->d_sky);
    if (c->d_fdot) cudaFree(c->d_fdot);
    c->d_sky = nullptr;
    c->d_fdot = nullptr;
    CUDA_TRY(c, cudaMalloc(&c->d_sky, 2 * (size_t)n_sky * sizeof(double)));
    CUDA_TRY(c, cudaMalloc(&c->d_fdot, (size_t)n_fdot * sizeof(double)));
    CUDA_TRY(c, cudaMemcpy(c->d_sky, sky, 2 * (size_t)n_sky * sizeof(double), cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(c->d_fdot, fdot, (size_t)n_fdot * sizeof(double), cudaMemcpyHostToDevice));
    c->n_sky = n_sky;
    c->n_f = n_f;
    c->n_fdot = n_fdot;
    // a uniform spindown grid gets compact per-(sky, SFT) bases
    c->dfdot = n_fdot > 1 ? (fdot[n_fdot - 1] - fdot[0]) / (n_fdot - 1) : 0.0;
    c->fdot_uniform = true;
    double fmax = 0.0;
    for (int d = 0; d < n_fdot; ++d) fmax = std::max(fmax, std::fabs(fdot[d]));
    for (int d = 0; d < n_fdot; ++d)
        if (std::fabs(fdot[d] - (fdot[0] + d * c->dfdot)) > 1e-12 * fmax) c->fdot_uniform = false;
    c->f0 = f0;
    c->df = df;
    c->t_ref = t_ref;
    c->have_templates = true;
    c->plan_valid = false;
    c->computed = false;
    return FSTAT_OK;
}

namespace {

// Refresh the per-SFT state, plan the tiles and size every buffer of one bank.
int ensure_tables(fstat_ctx* c, cudaStream_t s);

int prepare(fstat_ctx* c, cudaStream_t s) {
    int rc;
    if ((rc = refresh_sft_state(c, s)) != FSTAT_OK) return rc;
    if (!c->plan_valid) {
        if ((rc = make_plan(c, c->plan)) != FSTAT_OK) return rc;
        c->plan_valid = true;
    }
    const size_t n_meta = (size_t)c->n_sky * c->n_sft;
    const size_t n_base = n_meta * c->n_fdot;
    const size_t n_twoF = (size_t)c->n_sky * c->n_fdot * c->n_f;
    if ((rc = grow(c, &c->d_meta, c->cap_meta, n_meta)) != FSTAT_OK) return rc;
    if (c->fdot_uniform) {
        if ((rc = grow(c, &c->d_base, c->cap_base, n_meta)) != FSTAT_OK) return rc;
    } else {
        if ((rc = grow(c, &c->d_kh0, c->cap_kh0, n_base)) != FSTAT_OK) return rc;
        if ((rc = grow(c, &c->d_ph0, c->cap_ph0, n_base)) != FSTAT_OK) return rc;
    }
    if ((rc = grow(c, &c->d_abcd, c->cap_abcd, 4 * (size_t)c->n_sky)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_comb, c->cap_comb, (size_t)c->n_sky)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_twoF, c->cap_twoF, n_twoF)) != FSTAT_OK) return rc;
    if ((rc = ensure_topk(c)) != FSTAT_OK) return rc;
    if (c->have_cov) {
        if (c->n_f > kCovMaxF) return fail(c, FSTAT_EINVAL, "coverage supports at most %d frequencies", kCovMaxF);
        if ((rc = grow(c, &c->d_comb_j, c->cap_comb_j, (size_t)c->n_sky * c->n_f)) != FSTAT_OK) return rc;
    }
    return ensure_tables(c, s);
}

// The far-field or sinc tables for the current plan: their kind and extent
// follow the plan (form, window width), so a new plan may need a rebuild.
int ensure_tables(fstat_ctx* c, cudaStream_t s) {
    int rc;
    if (c->plan.sky_perm && !c->perm_on_device) {   // the neighbour order and its inverse
        const int n = c->n_sky;
        std::vector<int> rank(n);
        for (int i = 0; i < n; ++i) rank[c->h_order[i]] = i;
        if (c->d_perm) cudaFree(c->d_perm);
        if (c->d_rank) cudaFree(c->d_rank);
        c->d_perm = c->d_rank = nullptr;
        CUDA_TRY(c, cudaMalloc(&c->d_perm, (size_t)n * sizeof(int)));
        CUDA_TRY(c, cudaMalloc(&c->d_rank, (size_t)n * sizeof(int)));
        CUDA_TRY(c, cudaMemcpy(c->d_perm, c->h_order.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_rank, rank.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice));
        c->perm_on_device = true;
    }
    if (c->plan.far) far_extent(c, c->plan.w_pairs, &c->far_xoff, &c->n_pos);
    if (c->plan.far &&
        (c->tab_dirty || c->tab_npos != c->n_pos || c->tab_xoff != c->far_xoff || c->tab_sinc != c->plan.sinc ||
         (c->plan.sinc && c->tab_split != (c->plan.L == 2)))) {
        const size_t n_tab = (size_t)c->n_sft * c->n_pos;
        const void* bins = c->opts.bins_form == FSTAT_BINS_C64 ? (const void*)work_bins(c) : (const void*)c->d_bins16;
        if (c->plan.sinc) {
            if ((rc = grow(c, &c->d_pcoef, c->cap_pcoef, 6 * n_tab)) != FSTAT_OK) return rc;
            CUDA_TRY(c, launch_sinc_tables(bins, c->opts.bins_form, c->row, c->n_sft, c->n_bins, c->sgam, c->d_pcoef,
                                           c->n_pos, c->far_xoff, c->plan.L == 2, s));
        } else {
            if ((rc = grow(c, &c->d_ptab, c->cap_ptab, n_tab)) != FSTAT_OK) return rc;
            if ((rc = grow(c, &c->d_pcoef, c->cap_pcoef, 3 * n_tab)) != FSTAT_OK) return rc;
            CUDA_TRY(c, launch_far_tables(bins, c->opts.bins_form, c->row, c->n_sft, c->n_bins, c->gam, c->d_ptab,
                                          c->d_pcoef, c->n_pos, c->far_xoff, s));
        }
        c->launches += 1;
        c->tab_dirty = false;
        c->tab_npos = c->n_pos;
        c->tab_xoff = c->far_xoff;
        c->tab_sinc = c->plan.sinc;
        c->tab_split = c->plan.L == 2;
    }
    return FSTAT_OK;
}

TimingParams timing_params(const fstat_ctx* c, int n_sky) {
    TimingParams tp{};
    tp.st = c->d_state;
    tp.sky = c->d_sky;
    tp.fdot = c->d_fdot;
    tp.scale = c->d_scale;
    tp.weight = c->nf_half > 0 ? c->d_weight : nullptr;
    tp.n_sky = n_sky;
    tp.n_sft = c->n_sft;
    tp.n_fdot = c->n_fdot;
    tp.f0 = c->f0;
    tp.df = c->df;
    tp.T = c->T;
    tp.t_ref = c->t_ref;
    tp.P = c->plan.P;
    tp.L = c->plan.L;
    tp.M = c->plan.M;
    tp.uniform = c->fdot_uniform ? 1 : 0;
    tp.dfdot = c->dfdot;
    tp.meta = c->d_meta;
    tp.base = c->fdot_uniform ? c->d_base : nullptr;
    tp.sft_major = c->plan.sky_rows > 1 ? 1 : 0;   // blocks of several sky points read them SFT-major
    tp.sky_rank = c->plan.sky_perm ? c->d_rank : nullptr;
    tp.row_rot = (c->plan.rows || c->plan.two) ? 1 : 0;   // the row-tiled forms step the twiddle across rows
    tp.kh0 = c->fdot_uniform ? nullptr : c->d_kh0;
    tp.ph0 = c->fdot_uniform ? nullptr : c->d_ph0;
    tp.abcd = c->d_abcd;
    tp.comb = c->d_comb;
    tp.err = c->d_err;
    return tp;
}

DirichletParams dirichlet_params(const fstat_ctx* c) {
    const Plan& pl = c->plan;
    DirichletParams dp{};
    dp.bins = c->opts.bins_form == FSTAT_BINS_C64 ? (const void*)work_bins(c) : (const void*)c->d_bins16;
    dp.row = c->row;
    dp.k_lo = c->k_lo;
    dp.n_bins = c->n_bins;
    dp.n_sft = c->n_sft;
    dp.meta = c->d_meta;
    dp.base = c->fdot_uniform ? c->d_base : nullptr;
    dp.kh0 = c->fdot_uniform ? nullptr : c->d_kh0;
    dp.ph0 = c->fdot_uniform ? nullptr : c->d_ph0;
    dp.comb = c->d_comb;
    dp.sky_perm = pl.sky_perm ? c->d_perm : nullptr;
    dp.twoF = c->d_twoF;
    dp.n_sky = c->n_sky;
    dp.n_fdot = c->n_fdot;
    dp.n_f = c->n_f;
    dp.P = pl.P;
    dp.lg_row = pl.lg_row;
    dp.lg_cta = pl.lg_cta;
    dp.chunks_per_col = pl.chunks_per_col;
    dp.n_col = pl.n_col;
    dp.w_pairs = pl.w_pairs;
    dp.w_tab = pl.w_tab;
    dp.w_raw = pl.w_raw;
    dp.sft_chunk = pl.C;
    dp.err = c->d_err;
    dp.ring_stop = c->ring_stall;
    dp.cov = c->have_cov ? c->d_cov : nullptr;
    dp.comb_j = c->have_cov ? c->d_comb_j : nullptr;
    if (pl.far) {
        dp.ptab = c->d_ptab;
        dp.pcoef = c->d_pcoef;
        dp.n_pos = c->n_pos;
        dp.xoff = c->far_xoff;
    }
    return dp;
}

// True when the built tables are the ones the plan's kernel reads (kind and
// extent); the far-field and sinc kernels are never launched otherwise.
bool tables_match(const fstat_ctx* c, const Plan& pl) {
    if (!pl.far) return true;
    int xoff = 0, n_pos = 0;
    far_extent(c, pl.w_pairs, &xoff, &n_pos);
    return !c->tab_dirty && c->tab_sinc == pl.sinc && (!pl.sinc || c->tab_split == (pl.L == 2)) &&
           c->tab_npos == n_pos && c->tab_xoff == xoff &&
           c->n_pos == n_pos && c->far_xoff == xoff;
}

cudaError_t launch_dir(const fstat_ctx* c, const DirichletParams& dp, long long grid, cudaStream_t s) {
    const Plan& pl = c->plan;
    const int threads = pl.W * 32;
    if (pl.far) {
        if (!tables_match(c, pl)) return cudaErrorInvalidValue;
        return launch_dirichlet_far(pl.variant, dp, threads, pl.smem, grid, s);
    }
    if (c->opts.bins_form == FSTAT_BINS_C64)
        return launch_dirichlet_c64(pl.variant, dp, c->opts.dterms, threads, pl.smem, grid, s);
    if (c->opts.bins_form == FSTAT_BINS_F16)
        return launch_dirichlet_f16(pl.variant, dp, c->opts.dterms, threads, pl.smem, grid, s);
    return launch_dirichlet_bf16(pl.variant, dp, c->opts.dterms, threads, pl.smem, grid, s);
}

int enqueue_topk(fstat_ctx* c, cudaStream_t s) {
    const long long n = (long long)c->n_sky * c->n_fdot * c->n_f;
    const int k = (int)std::min<long long>(c->opts.topk, n);
    if (k > 0) {
        CUDA_TRY(c, launch_topk(c->d_twoF, n, k, c->tw, s));
        c->launches += 9;   // 3 histograms, 3 selections, collect, ties, sort
    }
    return FSTAT_OK;
}

}  // namespace

int fstat_compute(fstat_ctx* c, void* cuda_stream) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->have_sfts || !c->have_templates) return fail(c, FSTAT_ESTATE, "load SFTs and set templates first");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    c->stream = s;
    int rc;
    if ((rc = prepare(c, s)) != FSTAT_OK) return rc;
    CUDA_TRY(c, cudaMemsetAsync(c->d_err, 0, sizeof(int) * 3, s));
    const int slot = c->n_timed % kTimedRing;
    CUDA_TRY(c, cudaEventRecord(c->ev_a[slot], s));
    CUDA_TRY(c, launch_timing(timing_params(c, c->n_sky), s));
    if (c->have_cov) {
        CUDA_TRY(c, launch_coverage_comb(timing_params(c, c->n_sky), c->d_cov, c->n_f, c->d_comb_j, s));
        c->launches += 1;
    }
    CUDA_TRY(c, cudaEventRecord(c->ev_b[slot], s));
    cudaError_t e = launch_dir(c, dirichlet_params(c), c->plan.grid, s);
    if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "Dirichlet launch: %s", cudaGetErrorString(e));
    CUDA_TRY(c, cudaEventRecord(c->ev_c[slot], s));
    c->launches += 2;   // timing + Dirichlet
    if ((rc = enqueue_topk(c, s)) != FSTAT_OK) return rc;
    CUDA_TRY(c, cudaEventRecord(c->ev_d[slot], s));
    c->n_timed++;
    c->computed = true;
    return FSTAT_OK;
}

int fstat_get_2f(fstat_ctx* c, float* out, int64_t offset, int64_t count, int32_t mem) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->computed) return fail(c, FSTAT_ESTATE, "nothing computed");
    const long long n = (long long)c->n_sky * c->n_fdot * c->n_f;
    if (!out || offset < 0 || count < 0 || offset + count > n) return fail(c, FSTAT_EINVAL, "range out of bounds");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    CUDA_TRY(c, cudaMemcpyAsync(out, c->d_twoF + offset, (size_t)count * sizeof(float),
                                mem == FSTAT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                c->stream));
    const int rc = sync_ctx(c);
    return rc != FSTAT_OK ? rc : flag_status(c);
}

int fstat_get_toplist(fstat_ctx* c, int32_t k, int64_t* idx, float* twoF) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->computed) return fail(c, FSTAT_ESTATE, "nothing computed");
    const long long n = (long long)c->n_sky * c->n_fdot * c->n_f;
    const int kmax = (int)std::min<long long>(c->opts.topk, n);
    if (k < 0 || k > kmax || (k > 0 && (!idx || !twoF))) return fail(c, FSTAT_EINVAL, "k out of range 0..%d", kmax);
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    if (k > 0) {
        CUDA_TRY(c, cudaMemcpyAsync(idx, c->tw.out_idx, (size_t)k * sizeof(long long), cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(c, cudaMemcpyAsync(twoF, c->tw.out_val, (size_t)k * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    const int rc = sync_ctx(c);
    return rc != FSTAT_OK ? rc : flag_status(c);
}

int fstat_get_abcd(fstat_ctx* c, double* out) {
    if (!c || !out) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->computed) return fail(c, FSTAT_ESTATE, "nothing computed");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    CUDA_TRY(c, cudaMemcpyAsync(out, c->d_abcd, 4 * (size_t)c->n_sky * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return sync_ctx(c);
}

int fstat_get_sft_timing(fstat_ctx* c, int32_t sky, double* dtau, double* tdot, double* a, double* b) {
    if (!c || !dtau || !tdot || !a || !b) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->have_sfts || !c->have_templates) return fail(c, FSTAT_ESTATE, "load SFTs and set templates first");
    if (sky < 0 || sky >= c->n_sky) return fail(c, FSTAT_EINVAL, "sky index out of range");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int rc;
    if ((rc = refresh_sft_state(c, c->stream)) != FSTAT_OK) return rc;
    double* d_out = nullptr;
    CUDA_TRY(c, cudaMalloc(&d_out, 4 * (size_t)c->n_sft * sizeof(double)));
    cudaError_t e = launch_sft_timing_one(c->d_state, c->n_sft, c->h_sky[2 * sky], c->h_sky[2 * sky + 1], c->t_ref,
                                          d_out, c->stream);
    std::vector<double> h(4 * (size_t)c->n_sft);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_out);
    if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "sft timing: %s", cudaGetErrorString(e));
    const size_t n = c->n_sft;
    std::memcpy(dtau, h.data(), n * sizeof(double));
    std::memcpy(tdot, h.data() + n, n * sizeof(double));
    std::memcpy(a, h.data() + 2 * n, n * sizeof(double));
    std::memcpy(b, h.data() + 3 * n, n * sizeof(double));
    return FSTAT_OK;
}

int fstat_inject(fstat_ctx* c, const fstat_signal* sig, int32_t n_sig, double t_ref) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->have_sfts) return fail(c, FSTAT_ESTATE, "load SFTs first");
    if (n_sig < 0 || (n_sig > 0 && !sig) || !std::isfinite(t_ref)) return fail(c, FSTAT_EINVAL, "bad signal list");
    if (n_sig == 0) return FSTAT_OK;
    for (int i = 0; i < n_sig; ++i) {
        const double v[8] = {sig[i].alpha, sig[i].delta, sig[i].psi, sig[i].cosi, sig[i].phi0, sig[i].f, sig[i].fdot, sig[i].rho};
        if (!all_finite(v, 8) || !(sig[i].f > 0) || sig[i].rho < 0 || std::fabs(sig[i].cosi) > 1)
            return fail(c, FSTAT_EINVAL, "signal %d has invalid parameters", i);
    }
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int rc;
    if ((rc = refresh_sft_state(c, c->stream)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_sig, c->cap_sig, (size_t)n_sig)) != FSTAT_OK) return rc;
    if ((rc = grow(c, &c->d_inj_work, c->cap_inj, inject_work_doubles(n_sig, c->n_sft))) != FSTAT_OK) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_sig, sig, (size_t)n_sig * sizeof(fstat_signal), cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_inject(c->d_state, c->n_sft, c->d_sig, n_sig, c->T, t_ref, c->k_lo, c->n_bins, c->row,
                              c->d_bins, c->d_inj_work, c->stream));
    c->launches += 2;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    c->sft_dirty = true;   // 16-bit copies must be rebuilt
    c->computed = false;
    return FSTAT_OK;
}

int fstat_get_bins(fstat_ctx* c, int32_t det_index, float* out, int32_t mem) {
    if (!c || !out) return FSTAT_EINVAL;
    c->err.clear();
    if (det_index < 0 || det_index >= kMaxDet || !c->det[det_index].set)
        return fail(c, FSTAT_EINVAL, "detector %d not loaded", det_index);
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int first = 0;
    for (int d = 0; d < det_index; ++d)
        if (c->det[d].set) first += (int)c->det[d].t_start.size();
    const int n = (int)c->det[det_index].t_start.size();
    CUDA_TRY(c, cudaMemcpy2DAsync(out, (size_t)c->n_bins * sizeof(float2), c->d_bins + (size_t)first * c->row,
                                  c->row * sizeof(float2), (size_t)c->n_bins * sizeof(float2), n,
                                  mem == FSTAT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                  c->stream));
    return sync_ctx(c);
}

int fstat_get_error_flags(fstat_ctx* c, int32_t* flags) {
    if (!c || !flags) return FSTAT_EINVAL;
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int h[3] = {0, 0, 0};
    CUDA_TRY(c, cudaMemcpyAsync(h, c->d_err, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    int rc = sync_ctx(c);
    if (rc != FSTAT_OK) return rc;
    *flags = h[0];
    return FSTAT_OK;
}

int fstat_get_plan(fstat_ctx* c, int32_t* out) {
    if (!c || !out) return FSTAT_EINVAL;
    if (!c->have_sfts || !c->have_templates) return fail(c, FSTAT_ESTATE, "load SFTs and set templates first");
    if (!c->plan_valid) {
        int rc = make_plan(c, c->plan);
        if (rc != FSTAT_OK) return rc;
        c->plan_valid = true;
    }
    const Plan& p = c->plan;
    const int v[8] = {p.P, p.L, p.M, p.W, p.C, p.lg_row, p.w_pairs, p.far ? kFarIdBase + p.variant : p.variant};
    std::memcpy(out, v, sizeof(v));
    return FSTAT_OK;
}

int fstat_set_noise_floor(fstat_ctx* c, int32_t half_window) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (half_window < 0 || half_window > 64) return fail(c, FSTAT_EINVAL, "half window %d outside 0..64", half_window);
    if (half_window != c->nf_half) {
        c->nf_half = half_window;
        c->sft_dirty = true;
        c->computed = false;
    }
    return FSTAT_OK;
}

int fstat_get_noise(fstat_ctx* c, float* floor, double* weights, int32_t mem) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (c->nf_half <= 0) return fail(c, FSTAT_ESTATE, "noise floor is off");
    if (c->sft_dirty || !c->d_floor) return fail(c, FSTAT_ESTATE, "noise floor not computed yet (run fstat_compute)");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    const cudaMemcpyKind k = mem == FSTAT_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (floor) CUDA_TRY(c, cudaMemcpyAsync(floor, c->d_floor, sizeof(float) * (size_t)c->n_sft * c->n_bins, k, c->stream));
    if (weights) CUDA_TRY(c, cudaMemcpyAsync(weights, c->d_weight, sizeof(double) * (size_t)c->n_sft, k, c->stream));
    return sync_ctx(c);
}

int fstat_test_ring_stall(fstat_ctx* c, int32_t after_sft) {
    if (!c) return FSTAT_EINVAL;
    c->ring_stall = after_sft < 0 ? -1 : after_sft;
    return FSTAT_OK;
}

int fstat_get_launch_count(fstat_ctx* c, int64_t* n_launches) {
    if (!c || !n_launches) return FSTAT_EINVAL;
    *n_launches = c->launches;
    return FSTAT_OK;
}

int fstat_take_kernel_time(fstat_ctx* c, double* ms_dirichlet, double* ms_total, int32_t* n_calls) {
    if (!c || !ms_dirichlet || !ms_total || !n_calls) return FSTAT_EINVAL;
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    const int n = std::min(c->n_timed, kTimedRing);
    double sb = 0.0, st = 0.0;
    for (int i = 0; i < n; ++i) {
        CUDA_TRY(c, cudaEventSynchronize(c->ev_d[i]));
        float mb = 0.f, mt = 0.f;
        CUDA_TRY(c, cudaEventElapsedTime(&mb, c->ev_b[i], c->ev_c[i]));
        CUDA_TRY(c, cudaEventElapsedTime(&mt, c->ev_a[i], c->ev_d[i]));
        sb += mb;
        st += mt;
    }
    *n_calls = n;
    *ms_dirichlet = n ? sb / n : 0.0;
    *ms_total = n ? st / n : 0.0;
    c->n_timed = 0;
    return FSTAT_OK;
}


int fstat_autotune(fstat_ctx* c, void* cuda_stream, int32_t* out) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    // a context holding only workunits tunes on its largest one and applies its
    // templates per thread to all; each workunit keeps the planner's stage count,
    // which follows its own table width and residency (one stage count for all
    // cost up to 60 % on workunits whose stages then left one block per SM)
    if ((!c->have_sfts || !c->have_templates) && !c->wus.empty()) {
        fstat_ctx* big = c->wus[0];
        for (fstat_ctx* w : c->wus)
            if ((double)w->n_sky * w->n_f * w->n_fdot * w->n_sft > (double)big->n_sky * big->n_f * big->n_fdot * big->n_sft)
                big = w;
        int32_t o[4];
        int rc = fstat_autotune(big, cuda_stream, o);
        if (rc != FSTAT_OK) return fail(c, rc, "autotune: %s", big->err.c_str());
        for (fstat_ctx* w : c->wus) {   // the tuned workunit too returns to the caller's stage count
            w->opts.tile_m = o[0];
            w->opts.sft_chunk = c->opts.sft_chunk;
            w->plan_valid = false;
        }
        c->opts.tile_m = o[0];
        c->graph_valid = false;
        if (out) std::memcpy(out, o, sizeof(o));
        return FSTAT_OK;
    }
    if (!c->have_sfts || !c->have_templates) return fail(c, FSTAT_ESTATE, "load SFTs and set templates first");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    c->stream = s;
    const fstat_opts saved = c->opts;
    // candidate (M, SFT round) pairs for this bank's thread layout
    c->opts.tile_m = 0;
    c->opts.sft_chunk = 0;
    c->plan_valid = false;
    int rc = prepare(c, s);
    if (rc != FSTAT_OK) {
        c->opts = saved;
        return rc;
    }
    std::vector<int> Ms;   // 0: the planner's own choice of form (the rows form where it applies)
    if (c->plan.rows) Ms = {0, 5, 7};
    else if (c->plan.two) Ms = {5, 3};
    else if (c->plan.M == 1) Ms = {1};
    else if (c->opts.kahan) Ms = {5};
    else if (c->plan.L == 2 || c->plan.far) Ms = {5, 7, 9};
    else Ms = {7, 9};
    std::vector<int> Cs = {6, 8, 10};
    if (c->plan.ring) Cs = {4, 6, 8};
    else if (c->plan.far) Cs = {2, 3, 4};
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int bestM = c->plan.M, bestC = c->plan.C, bestW = c->plan.W;
    for (int M : Ms) {
        for (int C : Cs) {
            c->opts.tile_m = M;
            c->opts.sft_chunk = C;
            c->plan_valid = false;
            if (make_plan(c, c->plan) != FSTAT_OK) continue;
            c->plan_valid = true;
            if (c->plan.C != C) continue;   // round size capped by shared memory
            if (c->plan.sky_perm) continue;   // the slice takes the first sky points, not an order's groups
            if (ensure_tables(c, s) != FSTAT_OK) continue;   // tables for this plan's form and width
            // a slice of the bank: the first sky points, about four waves of blocks
            const long long per_sky = (long long)c->plan.n_col * c->plan.chunks_per_col;
            int occ = 2;
            const long long want = 4LL * occ * current_sm_count();
            const int n_sky_sub = (int)std::min<long long>(c->n_sky, std::max<long long>(1, (want + per_sky - 1) / per_sky));
            if (launch_timing(timing_params(c, n_sky_sub), s) != cudaSuccess) continue;
            DirichletParams dp = dirichlet_params(c);
            dp.n_sky = n_sky_sub;   // the far-field form orders blocks sky-fastest
            const int sr = c->plan.sky_rows;
            const long long grid = (long long)((n_sky_sub + sr - 1) / sr) * per_sky;
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                cudaEventRecord(e0, s);
                cudaError_t e = launch_dir(c, dp, grid, s);
                cudaEventRecord(e1, s);
                if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rep > 0) t = std::min(t, ms);   // first run warms up
            }
            c->launches += 4;
            if (t < best) {
                best = t;
                bestM = M;
                bestC = C;
                bestW = c->plan.W;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->opts = saved;
    c->opts.tile_m = bestM;
    c->opts.sft_chunk = bestC;
    c->plan_valid = false;
    c->computed = false;
    if (out) {
        out[0] = bestM;
        out[1] = bestC;
        out[2] = bestW;
        out[3] = (int32_t)std::min(best * 1000.f, 2.0e9f);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "autotune: %s", cudaGetErrorString(e));
    return FSTAT_OK;
}

int fstat_batch_add(fstat_ctx* c, const fstat_workunit* wu, int32_t* wu_id) {
    if (!c || !wu) return FSTAT_EINVAL;
    c->err.clear();
    if (wu->n_det < 1 || wu->n_det > kMaxDet || !wu->det || !wu->n_sft || !wu->t_start || !wu->bins)
        return fail(c, FSTAT_EINVAL, "workunit needs 1..8 detectors with SFTs");
    fstat_ctx* w = nullptr;
    int rc = fstat_create(&w, c->device, &c->opts);
    if (rc != FSTAT_OK) return fail(c, rc, "workunit context creation failed");
    w->batch_member = true;
    for (int d = 0; d < wu->n_det; ++d) {
        rc = fstat_set_sfts(w, d, &wu->det[d], wu->Tsft, wu->k_lo, wu->n_bins, wu->n_sft[d], wu->t_start[d],
                            wu->bins[d], FSTAT_MEM_HOST);
        if (rc != FSTAT_OK) {
            fail(c, rc, "workunit detector %d: %s", d, w->err.c_str());
            fstat_destroy(w);
            return rc;
        }
    }
    rc = fstat_set_templates(w, wu->sky, wu->n_sky, wu->f0, wu->df, wu->n_f, wu->fdot, wu->n_fdot, wu->t_ref);
    if (rc != FSTAT_OK) {
        fail(c, rc, "workunit bank: %s", w->err.c_str());
        fstat_destroy(w);
        return rc;
    }
    // the persistent kernels exist for the direct and the ring forms: a workunit
    // the far-field form would stage in rounds runs the direct form, alone or batched
    Plan pl;
    if (make_plan(w, pl) == FSTAT_OK && (pl.rows || pl.two)) {   // no persistent form of these: the one-row ring
        w->opts.algo = FSTAT_ALGO_SINCPOLY;
        if (make_plan(w, pl) != FSTAT_OK) pl = Plan{};
    }
    if (pl.far && (!pl.ring || pl.L != 2)) w->opts.algo = FSTAT_ALGO_DIRECT;
    w->plan_valid = false;
    w->err.clear();
    c->wus.push_back(w);
    c->graph_valid = false;
    c->batch_ran = false;
    if (wu_id) *wu_id = (int32_t)c->wus.size() - 1;
    return FSTAT_OK;
}

int fstat_batch_inject(fstat_ctx* c, int32_t wu, const fstat_signal* sig, int32_t n_sig, double t_ref) {
    if (!c) return FSTAT_EINVAL;
    if (wu < 0 || wu >= (int)c->wus.size()) return fail(c, FSTAT_EINVAL, "no workunit %d", wu);
    int rc = fstat_inject(c->wus[wu], sig, n_sig, t_ref);
    if (rc != FSTAT_OK) return fail(c, rc, "%s", c->wus[wu]->err.c_str());
    c->graph_valid = false;
    c->batch_ran = false;
    return FSTAT_OK;
}

int fstat_batch_clear(fstat_ctx* c) {
    if (!c) return FSTAT_EINVAL;
    cudaSetDevice(c->device);
    if (!c->wus.empty()) cudaDeviceSynchronize();
    for (fstat_ctx* w : c->wus) fstat_destroy(w);
    c->wus.clear();
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    c->graph_exec = nullptr;
    c->graph = nullptr;
    void* ptrs[] = {c->d_banks, c->d_prefix, c->d_rem_init, c->d_rem, c->d_queue, c->d_done};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c->d_banks = nullptr;
    c->d_prefix = nullptr;
    c->d_rem_init = nullptr;
    c->d_rem = nullptr;
    c->d_queue = nullptr;
    c->d_done = nullptr;
    c->graph_valid = false;
    c->batch_ran = false;
    return FSTAT_OK;
}

int fstat_batch_size(fstat_ctx* c, int32_t* n_wu) {
    if (!c || !n_wu) return FSTAT_EINVAL;
    *n_wu = (int32_t)c->wus.size();
    return FSTAT_OK;
}

}  // extern "C"

namespace {

__global__ void stamp_kernel(unsigned long long* t) {
    unsigned long long v;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(v));
    *t = v;
}

// Groups of workunits sharing a kernel (direct or far-field ring), variant and block size.
struct BatchGroup {
    int variant, W, form;
    size_t smem;
    int first, count;   // range in the sorted workunit order
    bool ring;
};

// Enqueue the whole batch on stream s (also used inside graph capture).
int enqueue_batch(fstat_ctx* c, const std::vector<int>& order, const std::vector<BatchGroup>& groups,
                  cudaStream_t s) {
    const int n = (int)c->wus.size();
    stamp_kernel<<<1, 1, 0, s>>>(c->d_done + n);
    CUDA_TRY(c, cudaGetLastError());
    c->launches += 1;
    for (fstat_ctx* w : c->wus) {
        CUDA_TRY(c, cudaMemsetAsync(w->d_err, 0, sizeof(int) * 3, s));
        CUDA_TRY(c, launch_timing(timing_params(w, w->n_sky), s));
        w->launches += 1;
    }
    CUDA_TRY(c, cudaMemcpyAsync(c->d_rem, c->d_rem_init, sizeof(int) * n, cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(c, cudaMemsetAsync(c->d_queue, 0, sizeof(unsigned long long) * groups.size(), s));
    const int dev_sms = current_sm_count();
    const size_t n_side = groups.empty() ? 0 : groups.size() - 1;
    while (c->side_streams.size() < n_side) {
        cudaStream_t st;
        CUDA_TRY(c, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        c->side_streams.push_back(st);
    }
    while (c->side_events.size() < n_side + 1) {
        cudaEvent_t ev;
        CUDA_TRY(c, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        c->side_events.push_back(ev);
    }
    if (n_side) CUDA_TRY(c, cudaEventRecord(c->side_events[0], s));
    for (size_t g = 0; g < groups.size(); ++g) {
        const BatchGroup& G = groups[g];
        cudaStream_t gs = s;   // the group's stream
        if (g > 0) {
            gs = c->side_streams[g - 1];
            CUDA_TRY(c, cudaStreamWaitEvent(gs, c->side_events[0], 0));
        }
        DirichletBatch b{};
        b.banks = c->d_banks + G.first;
        b.item_prefix = c->d_prefix + G.first + g;   // each group's prefix has count + 1 entries
        b.n_wu = G.count;
        b.queue = c->d_queue + g;
        b.remaining = c->d_rem + G.first;
        b.done_ns = c->d_done + G.first;
        int occ = 1;
        cudaError_t e;
        if (G.ring) {
            e = dirichlet_far_batch_occupancy(G.variant, G.W * 32, G.smem, &occ);
            if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "occupancy: %s", cudaGetErrorString(e));
            e = launch_dirichlet_far_batch(G.variant, b, G.W * 32, G.smem, std::max(1, occ) * dev_sms, gs);
            if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "batch Dirichlet launch: %s", cudaGetErrorString(e));
            c->launches += 1;
            if (g > 0) CUDA_TRY(c, cudaEventRecord(c->side_events[g], gs));
            continue;
        }
        if (G.form == FSTAT_BINS_C64) e = dirichlet_occupancy_c64(G.variant, G.W * 32, G.smem, &occ);
        else if (G.form == FSTAT_BINS_F16) e = dirichlet_occupancy_f16(G.variant, G.W * 32, G.smem, &occ);
        else e = dirichlet_occupancy_bf16(G.variant, G.W * 32, G.smem, &occ);
        if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "occupancy: %s", cudaGetErrorString(e));
        const int grid = std::max(1, occ) * dev_sms;
        if (G.form == FSTAT_BINS_C64) e = launch_dirichlet_batch_c64(G.variant, b, c->opts.dterms, G.W * 32, G.smem, grid, gs);
        else if (G.form == FSTAT_BINS_F16) e = launch_dirichlet_batch_f16(G.variant, b, c->opts.dterms, G.W * 32, G.smem, grid, gs);
        else e = launch_dirichlet_batch_bf16(G.variant, b, c->opts.dterms, G.W * 32, G.smem, grid, gs);
        if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "batch Dirichlet launch: %s", cudaGetErrorString(e));
        c->launches += 1;
        if (g > 0) CUDA_TRY(c, cudaEventRecord(c->side_events[g], gs));
    }
    for (size_t g = 1; g < groups.size(); ++g) CUDA_TRY(c, cudaStreamWaitEvent(s, c->side_events[g], 0));
    for (fstat_ctx* w : c->wus) {
        int rc = enqueue_topk(w, s);
        if (rc != FSTAT_OK) return fail(c, rc, "%s", w->err.c_str());
    }
    (void)order;
    return FSTAT_OK;
}

}  // namespace

extern "C" {

int fstat_batch_compute(fstat_ctx* c, void* cuda_stream) {
    if (!c) return FSTAT_EINVAL;
    c->err.clear();
    if (c->wus.empty()) return fail(c, FSTAT_ESTATE, "no workunits in the batch");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    c->stream = s;
    const int n = (int)c->wus.size();
    for (fstat_ctx* w : c->wus) {
        w->stream = s;
        int rc = prepare(w, s);
        if (rc != FSTAT_OK) return fail(c, rc, "workunit: %s", w->err.c_str());
        if (w->plan.far && (!w->plan.ring || w->plan.L != 2 || w->plan.rows || w->plan.two)) {   // persistent: direct, one-row L = 2 ring
            w->opts.algo = FSTAT_ALGO_DIRECT;
            w->plan_valid = false;
            c->graph_valid = false;
            if ((rc = prepare(w, s)) != FSTAT_OK) return fail(c, rc, "workunit: %s", w->err.c_str());
        }
    }
    if (!c->bev0) {
        cudaEventCreate(&c->bev0);
        cudaEventCreate(&c->bev1);
    }
    // group workunits by kernel variant, block size and blocks resident per SM
    // (the persistent launch of a group takes its largest shared-memory need,
    // so a workunit with wide stages must not set the residency of small ones)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto key = [&](int i) {
        const Plan& pl = c->wus[i]->plan;
        const int resident = (int)std::min<size_t>(15, (227 * 1024) / (pl.smem + 1024));
        return (pl.ring ? 1 << 20 : 0) + pl.variant * 1024 + pl.W * 16 + resident;
    };
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return key(a) < key(b); });
    if (!c->graph_valid) {
        // device tables in grouped order
        std::vector<BatchGroup> groups;
        std::vector<DirichletParams> banks(n);
        std::vector<long long> prefix;
        std::vector<int> rem(n);
        for (int k = 0; k < n; ++k) {
            fstat_ctx* w = c->wus[order[k]];
            if (groups.empty() || key(order[groups.back().first]) != key(order[k])) {
                groups.push_back(BatchGroup{w->plan.variant, w->plan.W, w->opts.bins_form, 0, k, 0, w->plan.ring});
                prefix.push_back(0);
            }
            BatchGroup& G = groups.back();
            G.count++;
            G.smem = std::max(G.smem, w->plan.smem);
            banks[k] = dirichlet_params(w);
            rem[k] = (int)w->plan.grid;
            prefix.push_back(prefix.back() + w->plan.grid);
        }
        if (c->d_banks) cudaFree(c->d_banks);
        if (c->d_prefix) cudaFree(c->d_prefix);
        if (c->d_rem_init) cudaFree(c->d_rem_init);
        if (c->d_rem) cudaFree(c->d_rem);
        if (c->d_queue) cudaFree(c->d_queue);
        if (c->d_done) cudaFree(c->d_done);
        CUDA_TRY(c, cudaMalloc(&c->d_banks, sizeof(DirichletParams) * n));
        CUDA_TRY(c, cudaMalloc(&c->d_prefix, sizeof(long long) * prefix.size()));
        CUDA_TRY(c, cudaMalloc(&c->d_rem_init, sizeof(int) * n));
        CUDA_TRY(c, cudaMalloc(&c->d_rem, sizeof(int) * n));
        CUDA_TRY(c, cudaMalloc(&c->d_queue, sizeof(unsigned long long) * groups.size()));
        CUDA_TRY(c, cudaMalloc(&c->d_done, sizeof(unsigned long long) * (n + 1)));
        CUDA_TRY(c, cudaMemcpy(c->d_banks, banks.data(), sizeof(DirichletParams) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_prefix, prefix.data(), sizeof(long long) * prefix.size(), cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemcpy(c->d_rem_init, rem.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
        CUDA_TRY(c, cudaMemset(c->d_done, 0, sizeof(unsigned long long) * (n + 1)));
        // first run without a graph (sets kernel attributes), then capture the same sequence
        CUDA_TRY(c, cudaEventRecord(c->bev0, s));
        int rc = enqueue_batch(c, order, groups, s);
        if (rc != FSTAT_OK) return rc;
        CUDA_TRY(c, cudaEventRecord(c->bev1, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        if (!c->cap_stream) CUDA_TRY(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
        if (c->graph) cudaGraphDestroy(c->graph);
        c->graph_exec = nullptr;
        c->graph = nullptr;
        const long long launches_before = c->launches;
        CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
        rc = enqueue_batch(c, order, groups, c->cap_stream);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (rc != FSTAT_OK) return rc;
        if (e != cudaSuccess) return fail(c, FSTAT_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        c->graph = g;
        CUDA_TRY(c, cudaGraphInstantiate(&c->graph_exec, g, 0));
        c->launches_per_graph = c->launches - launches_before;
        c->batch_order = order;
        c->launches = launches_before;
        c->graph_valid = true;
    } else {
        CUDA_TRY(c, cudaEventRecord(c->bev0, s));
        CUDA_TRY(c, cudaGraphLaunch(c->graph_exec, s));
        CUDA_TRY(c, cudaEventRecord(c->bev1, s));
        c->launches += c->launches_per_graph;
    }
    for (fstat_ctx* w : c->wus) w->computed = true;
    return FSTAT_OK;
}

int fstat_batch_compute_one(fstat_ctx* c, int32_t wu, void* cuda_stream) {
    if (!c) return FSTAT_EINVAL;
    if (wu < 0 || wu >= (int)c->wus.size()) return fail(c, FSTAT_EINVAL, "no workunit %d", wu);
    int rc = fstat_compute(c->wus[wu], cuda_stream);
    if (rc != FSTAT_OK) return fail(c, rc, "%s", c->wus[wu]->err.c_str());
    return FSTAT_OK;
}

int fstat_batch_get_toplist(fstat_ctx* c, int32_t wu, int32_t k, int64_t* idx, float* twoF) {
    if (!c) return FSTAT_EINVAL;
    if (wu < 0 || wu >= (int)c->wus.size()) return fail(c, FSTAT_EINVAL, "no workunit %d", wu);
    int rc = fstat_get_toplist(c->wus[wu], k, idx, twoF);
    if (rc != FSTAT_OK) return fail(c, rc, "%s", c->wus[wu]->err.c_str());
    return FSTAT_OK;
}

int fstat_batch_get_2f(fstat_ctx* c, int32_t wu, float* out, int64_t offset, int64_t count, int32_t mem) {
    if (!c) return FSTAT_EINVAL;
    if (wu < 0 || wu >= (int)c->wus.size()) return fail(c, FSTAT_EINVAL, "no workunit %d", wu);
    int rc = fstat_get_2f(c->wus[wu], out, offset, count, mem);
    if (rc != FSTAT_OK) return fail(c, rc, "%s", c->wus[wu]->err.c_str());
    return FSTAT_OK;
}

int fstat_batch_get_plan(fstat_ctx* c, int32_t wu, int32_t* out) {
    if (!c || !out) return FSTAT_EINVAL;
    c->err.clear();
    if (wu < 0 || wu >= (int)c->wus.size()) return fail(c, FSTAT_EINVAL, "no workunit %d", wu);
    const int rc = fstat_get_plan(c->wus[wu], out);
    if (rc != FSTAT_OK) return fail(c, rc, "%s", c->wus[wu]->err.c_str());
    return FSTAT_OK;
}

int fstat_batch_get_times(fstat_ctx* c, double* wu_done_ms, double* total_ms) {
    if (!c || !total_ms) return FSTAT_EINVAL;
    if (c->wus.empty() || !c->bev1) return fail(c, FSTAT_ESTATE, "no batch computed");
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    CUDA_TRY(c, cudaEventSynchronize(c->bev1));
    float ms = 0.f;
    CUDA_TRY(c, cudaEventElapsedTime(&ms, c->bev0, c->bev1));
    *total_ms = ms;
    if (wu_done_ms) {
        const int n = (int)c->wus.size();
        std::vector<unsigned long long> t(n + 1);
        CUDA_TRY(c, cudaMemcpy(t.data(), c->d_done, sizeof(unsigned long long) * (n + 1), cudaMemcpyDeviceToHost));
        for (int k = 0; k < n; ++k) {
            const int i = k < (int)c->batch_order.size() ? c->batch_order[k] : k;
            wu_done_ms[i] = t[k] >= t[n] ? (double)(t[k] - t[n]) * 1e-6 : 0.0;
        }
    }
    return FSTAT_OK;
}


int fstat_extract_patches(fstat_ctx* c, int32_t n_a, int32_t n_d, int32_t s_a, int32_t s_d, int32_t n_fp,
                          const int32_t* f_start, int32_t n_q, float shift, float scale, uint16_t* out) {
    if (!c || !f_start || !out) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->computed) return fail(c, FSTAT_ESTATE, "nothing computed");
    if (c->n_fdot != 1) return fail(c, FSTAT_EINVAL, "patches need a bank with one spindown");
    if (n_a < 1 || n_d < 1 || s_a < 1 || s_d < 1 || n_a % s_a || n_d % s_d || (long long)n_a * n_d != c->n_sky)
        return fail(c, FSTAT_EINVAL, "sky grid %d x %d does not tile the bank's %d sky points", n_a, n_d, c->n_sky);
    if (n_fp < 1 || n_q < 1) return fail(c, FSTAT_EINVAL, "empty patch");
    for (int q = 0; q < n_q; ++q)
        if (f_start[q] < 0 || f_start[q] + n_fp > c->n_f) return fail(c, FSTAT_EINVAL, "frequency patch %d outside the band", q);
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int rc = grow(c, &c->d_fstart, c->cap_fstart, (size_t)n_q);
    if (rc != FSTAT_OK) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_fstart, f_start, sizeof(int) * n_q, cudaMemcpyHostToDevice, c->stream));
    const int n_pd = n_d / s_d;
    const int n_patches = (n_a / s_a) * n_pd * n_q;
    CUDA_TRY(c, launch_patches(c->d_twoF, c->n_f, n_d, s_a, s_d, n_fp, c->d_fstart, n_q, n_patches, n_pd, shift, scale,
                               out, c->stream));
    c->launches += 1;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // f_start is a caller buffer
    return FSTAT_OK;
}

int fstat_extract_windows(fstat_ctx* c, int32_t n_a, int32_t n_d, int32_t s_a, int32_t s_d, int32_t n_fp,
                          const int32_t* origin, int32_t n_w, float shift, float scale, uint16_t* out) {
    if (!c || !origin || !out) return FSTAT_EINVAL;
    c->err.clear();
    if (!c->computed) return fail(c, FSTAT_ESTATE, "nothing computed");
    if (c->n_fdot != 1) return fail(c, FSTAT_EINVAL, "windows need a bank with one spindown");
    if (n_a < 1 || n_d < 1 || (long long)n_a * n_d != c->n_sky)
        return fail(c, FSTAT_EINVAL, "sky grid %d x %d does not match the bank's %d sky points", n_a, n_d, c->n_sky);
    if (s_a < 1 || s_d < 1 || n_fp < 1 || s_a > n_a || s_d > n_d || n_fp > c->n_f || n_w < 1)
        return fail(c, FSTAT_EINVAL, "empty or oversized window");
    for (int w = 0; w < n_w; ++w) {
        const int32_t a0 = origin[3 * w], d0 = origin[3 * w + 1], f0 = origin[3 * w + 2];
        if (a0 < 0 || a0 >= n_a || d0 < 0 || d0 + s_d > n_d || f0 < 0 || f0 + n_fp > c->n_f)
            return fail(c, FSTAT_EINVAL, "window %d origin (%d, %d, %d) outside the grid", w, a0, d0, f0);
    }
    if (set_device(c) != FSTAT_OK) return FSTAT_ECUDA;
    int rc = grow(c, &c->d_fstart, c->cap_fstart, (size_t)3 * n_w);
    if (rc != FSTAT_OK) return rc;
    CUDA_TRY(c, cudaMemcpyAsync(c->d_fstart, origin, sizeof(int) * 3 * (size_t)n_w, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(c, launch_windows(c->d_twoF, c->n_f, n_a, n_d, s_a, s_d, n_fp, c->d_fstart, n_w, shift, scale, out,
                               c->stream));
    c->launches += 1;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));   // origin is a caller buffer
    return FSTAT_OK;
}

}  // extern "C"
