// etd_ensemble_f64_2d.cu -- persistent ensemble step kernels, double, 2D.
#include "etd_ensemble.cuh"

namespace etd {

cudaError_t launch_ensemble_2d(const EnsArgs<double> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident) {
  return ensemble_any<double, 2>(E, nspecies, L0, LS, nthreads, smem, grid, s, resident);
}

}  // namespace etd
