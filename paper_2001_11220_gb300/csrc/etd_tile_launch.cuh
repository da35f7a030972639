// etd_tile_launch.cuh -- host launchers of the FP32 tile kernels, one
// translation unit per sweep kind (etd_tile_first.cu, _middle.cu, _last.cu).
#pragma once

#include "etd_sweep_launch.cuh"
#include "etd_tile.cuh"

namespace etd {

template <int S, int L, int NLB, int KIND, int PK>
cudaError_t launch_tile_one(const SweepArgs<float> &a, int nthreads, size_t smem, cudaStream_t s) {
  auto fn = sweep_tile_kernel<S, L, NLB, KIND, PK>;
  cudaError_t e = ensure_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<a.nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

// nspecies in {1, 2} x L in {8, 16} x NLB in {16, 32}
#define ETD_TILE_DISPATCH(KIND_, PK_)                                              \
  switch (nspecies * 10000 + L * 100 + NLB) {                                      \
    case 10816: return launch_tile_one<1, 8, 16, KIND_, PK_>(a, nthreads, smem, s); \
    case 10832: return launch_tile_one<1, 8, 32, KIND_, PK_>(a, nthreads, smem, s); \
    case 11616: return launch_tile_one<1, 16, 16, KIND_, PK_>(a, nthreads, smem, s); \
    case 11632: return launch_tile_one<1, 16, 32, KIND_, PK_>(a, nthreads, smem, s); \
    case 20816: return launch_tile_one<2, 8, 16, KIND_, PK_>(a, nthreads, smem, s); \
    case 20832: return launch_tile_one<2, 8, 32, KIND_, PK_>(a, nthreads, smem, s); \
    case 21616: return launch_tile_one<2, 16, 16, KIND_, PK_>(a, nthreads, smem, s); \
    case 21632: return launch_tile_one<2, 16, 32, KIND_, PK_>(a, nthreads, smem, s); \
    default: return cudaErrorInvalidValue;                                         \
  }

}  // namespace etd
