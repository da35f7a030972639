// etd_adjoint_circ_f64.cu -- adjoint sweeps of periodic axes on the circulant
// factorisation, double (chunk length 4).
#include "etd_adjoint_launch.cuh"

namespace etd {

cudaError_t launch_adjoint_circ(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                cudaStream_t s) {
  if (L != 4) return cudaErrorInvalidValue;
  switch (nspecies * 10 + kind) {
    case 10: return launch_adj_one<double, 1, 4, ADJ_FIRST, true>(a, nthreads, smem, s);
    case 11: return launch_adj_one<double, 1, 4, ADJ_MIDDLE, true>(a, nthreads, smem, s);
    case 12: return launch_adj_one<double, 1, 4, ADJ_LAST, true>(a, nthreads, smem, s);
    case 20: return launch_adj_one<double, 2, 4, ADJ_FIRST, true>(a, nthreads, smem, s);
    case 21: return launch_adj_one<double, 2, 4, ADJ_MIDDLE, true>(a, nthreads, smem, s);
    case 22: return launch_adj_one<double, 2, 4, ADJ_LAST, true>(a, nthreads, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace etd
