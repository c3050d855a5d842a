// Dirichlet kernel instantiations for one SFT storage form.
#include "dirichlet.cuh"

namespace fs {
cudaError_t launch_dirichlet_f16(int v, const DirichletParams& p, int d_rt, int threads, size_t smem,
                               long long grid, cudaStream_t s) {
    return launch_dirichlet_form<FSTAT_BINS_F16>(v, p, d_rt, threads, smem, grid, s);
}
}  // namespace fs
