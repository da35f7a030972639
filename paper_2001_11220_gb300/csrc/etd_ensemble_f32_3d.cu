// etd_ensemble_f32_3d.cu -- persistent ensemble step kernels, float, 3D.
#include "etd_ensemble.cuh"

namespace etd {

cudaError_t launch_ensemble_3d(const EnsArgs<float> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident) {
  return ensemble_any<float, 3>(E, nspecies, L0, LS, nthreads, smem, grid, s, resident);
}

}  // namespace etd
