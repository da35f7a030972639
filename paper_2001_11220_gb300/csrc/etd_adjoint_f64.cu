// etd_adjoint_f64.cu -- adjoint sweep kernels and launchers for double.
#include "etd_adjoint_launch.cuh"

namespace etd {

int loss_blocks(long long n) { return misfit_blocks(n); }

cudaError_t launch_adjoint(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                           cudaStream_t s) {
  if (a.circ_adj) return launch_adjoint_circ(a, nspecies, L, kind, nthreads, smem, s);
#define CALL(S_, L_, K_) launch_adj_one<double, S_, L_, K_>(a, nthreads, smem, s)
  ETD_ADJ_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_loss(const double *U, const double *target, double *Ubar, long long n, double *loss, double *part,
                        cudaStream_t s) {
  return launch_misfit<double>(U, target, Ubar, n, loss, part, s);
}

}  // namespace etd
