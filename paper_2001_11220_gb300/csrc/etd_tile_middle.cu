// etd_tile_middle.cu -- FP32 tile kernels of the MIDDLE (y-axis, 3D) sweep.
#include "etd_tile_launch.cuh"

namespace etd {

cudaError_t launch_tile_middle(const SweepArgs<float> &a, int nspecies, int L, int NLB, int pk, int nthreads,
                               size_t smem, cudaStream_t s) {
  if (pk == 2) {
    ETD_TILE_DISPATCH(SWEEP_MIDDLE, 2)
  }
  ETD_TILE_DISPATCH(SWEEP_MIDDLE, 1)
}

}  // namespace etd
