// etd_circ_rk_strided.cu -- strided-axis circulant kernels with the reaction
// fixed at compile time (FP32, two species: Brusselator, Schnakenberg,
// Gray-Scott), for the block shapes 16 x 32 and 16 x 16 (chunks x lines).
#include "etd_circ.cuh"

namespace etd {

CircKernel<float> circ_strided_kernel_rk(int kind, int wb, int nc, int rkind) {
  if (rkind < 2 || rkind > 4 || (kind != SWEEP_MIDDLE && kind != SWEEP_LAST)) return nullptr;
#define ETD_STRIDED_RK(WB_, NC_)                                                                        \
  if (wb == WB_ && nc == NC_) {                                                                         \
    const bool last = kind == SWEEP_LAST;                                                               \
    switch (rkind) {                                                                                    \
      case 2: return last ? circ_strided_kernel<float, 2, 16, SWEEP_LAST, WB_, NC_, 2>                  \
                          : circ_strided_kernel<float, 2, 16, SWEEP_MIDDLE, WB_, NC_, 2>;               \
      case 3: return last ? circ_strided_kernel<float, 2, 16, SWEEP_LAST, WB_, NC_, 3>                  \
                          : circ_strided_kernel<float, 2, 16, SWEEP_MIDDLE, WB_, NC_, 3>;               \
      default: return last ? circ_strided_kernel<float, 2, 16, SWEEP_LAST, WB_, NC_, 4>                 \
                           : circ_strided_kernel<float, 2, 16, SWEEP_MIDDLE, WB_, NC_, 4>;              \
    }                                                                                                   \
  }
  ETD_STRIDED_RK(16, 32)
  ETD_STRIDED_RK(16, 16)
#undef ETD_STRIDED_RK
  return nullptr;
}

int circ_take_status_rk_strided() { return take_status_here(); }

}  // namespace etd
