// etd_adjoint_circ_f32.cu -- adjoint sweeps of periodic axes on the circulant
// factorisation, float (chunk length 8).
#include "etd_adjoint_launch.cuh"

namespace etd {

cudaError_t launch_adjoint_circ(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                cudaStream_t s) {
  if (L != 8) return cudaErrorInvalidValue;
  switch (nspecies * 10 + kind) {
    case 10: return launch_adj_one<float, 1, 8, ADJ_FIRST, true>(a, nthreads, smem, s);
    case 11: return launch_adj_one<float, 1, 8, ADJ_MIDDLE, true>(a, nthreads, smem, s);
    case 12: return launch_adj_one<float, 1, 8, ADJ_LAST, true>(a, nthreads, smem, s);
    case 20: return launch_adj_one<float, 2, 8, ADJ_FIRST, true>(a, nthreads, smem, s);
    case 21: return launch_adj_one<float, 2, 8, ADJ_MIDDLE, true>(a, nthreads, smem, s);
    case 22: return launch_adj_one<float, 2, 8, ADJ_LAST, true>(a, nthreads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace etd
