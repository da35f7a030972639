// etd_sweep_f32.cu -- sweep kernels and launchers for float.
#include "etd_sweep_launch.cuh"

namespace etd {

cudaError_t launch_sweep(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                         cudaStream_t s) {
  if (a.segphase == SEG_CLUSTER) return launch_sweep_cluster(a, nspecies, L, kind, nthreads, smem, s);
  if (a.sp.staged == 2) return launch_tile(a, nspecies, L, a.nlb * a.pk, kind, a.pk, nthreads, a.sp.bytes, s);
#define CALL(S_, L_, K_) launch_one<float, S_, L_, K_>(a, nthreads, smem, s)
  ETD_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_sweep_batched(const SweepArgs<float> *args, const int *bs, int ninst, int total, int nspecies,
                                 int L, int kind, int nthreads, size_t smem, cudaStream_t s, double t_eval) {
#define CALL(S_, L_, K_) launch_one_batched<float, S_, L_, K_>(args, bs, ninst, total, nthreads, smem, s, t_eval)
  ETD_DISPATCH(CALL)
#undef CALL
}

cudaError_t launch_seg_carry(const SweepArgs<float> &a, int nspecies, int kind, int q0, int nq, cudaStream_t s) {
  return launch_seg_carry_t<float>(a, nspecies, kind, q0, nq, s);
}

}  // namespace etd
