// etd_sweep_f64.cu -- sweep kernels and launchers for double.
#include "etd_sweep_launch.cuh"

namespace etd {

cudaError_t launch_sweep(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                         cudaStream_t s) {
  if (a.segphase == SEG_CLUSTER) return launch_sweep_cluster(a, nspecies, L, kind, nthreads, smem, s);
#define CALL(S_, L_, K_) launch_one<double, S_, L_, K_>(a, nthreads, smem, s)
  ETD_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_sweep_batched(const SweepArgs<double> *args, const int *bs, int ninst, int total, int nspecies,
                                 int L, int kind, int nthreads, size_t smem, cudaStream_t s, double t_eval) {
#define CALL(S_, L_, K_) launch_one_batched<double, S_, L_, K_>(args, bs, ninst, total, nthreads, smem, s, t_eval)
  ETD_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_seg_carry(const SweepArgs<double> &a, int nspecies, int kind, int q0, int nq, cudaStream_t s) {
  return launch_seg_carry_t<double>(a, nspecies, kind, q0, nq, s);
}

}  // namespace etd
