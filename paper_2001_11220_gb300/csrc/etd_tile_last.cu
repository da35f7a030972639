// etd_tile_last.cu -- FP32 tile kernels of the LAST (strided) sweep.
#include "etd_tile_launch.cuh"

namespace etd {

cudaError_t launch_tile_last(const SweepArgs<float> &a, int nspecies, int L, int NLB, int pk, int nthreads,
                             size_t smem, cudaStream_t s) {
  if (pk == 2) {
    ETD_TILE_DISPATCH(SWEEP_LAST, 2)
  }
  ETD_TILE_DISPATCH(SWEEP_LAST, 1)
}

}  // namespace etd
