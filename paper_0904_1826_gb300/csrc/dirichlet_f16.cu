// Dirichlet kernel instantiations for one SFT storage form.
#include "dirichlet.cuh"

namespace fs {
cudaError_t launch_dirichlet_f16(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                               long long grid, cudaStream_t s) {
    return launch_dirichlet_form<FSTAT_BINS_F16>(v, p, d_rt, threads, smem, grid, s);
}
cudaError_t launch_dirichlet_batch_f16(int v, const DirichletBatch& b, int d_rt, int threads, size_t smem,
                                     int grid, cudaStream_t s) {
    return launch_dirichlet_batch_form<FSTAT_BINS_F16>(v, b, d_rt, threads, smem, grid, s);
}
cudaError_t dirichlet_occupancy_f16(int v, int threads, size_t smem, int* blocks_per_sm) {
    return dirichlet_occupancy_form<FSTAT_BINS_F16>(v, threads, smem, blocks_per_sm);
}
}  // namespace fs
