// etd_tile_first.cu -- FP32 tile kernels of the FIRST (x-axis) sweep.
#include "etd_tile_launch.cuh"

namespace etd {

cudaError_t launch_tile_first(const SweepArgs<float> &a, int nspecies, int L, int NLB, int nthreads, size_t smem,
                              cudaStream_t s) {
  ETD_TILE_DISPATCH(SWEEP_FIRST, 1)
}

// every tile launch goes through here: one entry point for the host code
cudaError_t launch_tile(const SweepArgs<float> &a, int nspecies, int L, int NLB, int kind, int pk, int nthreads,
                        size_t smem, cudaStream_t s) {
  if (kind == SWEEP_FIRST) return pk == 1 ? launch_tile_first(a, nspecies, L, NLB, nthreads, smem, s)
                                          : cudaErrorInvalidValue;
  if (kind == SWEEP_MIDDLE) return launch_tile_middle(a, nspecies, L, NLB, pk, nthreads, smem, s);
  return launch_tile_last(a, nspecies, L, NLB, pk, nthreads, smem, s);
}

}  // namespace etd
