// etd_circ_rk_first.cu -- first-axis circulant kernels with the reaction
// fixed at compile time (FP32, two species: Brusselator, Schnakenberg,
// Gray-Scott); the per-position reaction then needs no dispatch.
#include "etd_circ.cuh"

namespace etd {

CircKernel<float> circ_first_kernel_rk(int L, int nthreads, int rkind) {
  if (nthreads != 256 && nthreads != 512) return nullptr;
  const bool big = nthreads == 512;
#define ETD_FIRST_RK(L_, K_) \
  (big ? circ_first_kernel<float, 2, L_, 512, K_> : circ_first_kernel<float, 2, L_, 256, K_>)
  switch (L * 10 + rkind) {
    case 82: return ETD_FIRST_RK(8, 2);
    case 83: return ETD_FIRST_RK(8, 3);
    case 84: return ETD_FIRST_RK(8, 4);
    case 162: return ETD_FIRST_RK(16, 2);
    case 163: return ETD_FIRST_RK(16, 3);
    case 164: return ETD_FIRST_RK(16, 4);
    default: return nullptr;
  }
#undef ETD_FIRST_RK
}

int circ_take_status_rk_first() { return take_status_here(); }

}  // namespace etd
