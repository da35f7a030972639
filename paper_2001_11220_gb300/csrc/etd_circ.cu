// etd_circ.cu -- launchers of the circulant sweeps of periodic axes.
#include <cuda_runtime.h>

#include "etd_circ.cuh"

namespace etd {

namespace {

template <typename K>
cudaError_t ensure_dyn_smem(K fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R, int S, int L>
cudaError_t launch_first(const CircArgs<R> &a, int nthreads, size_t smem, int nblocks, cudaStream_t s) {
  auto fn = circ_first_kernel<R, S, L>;
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_any(const CircArgs<R> &a, int nspecies, int L, int kind, int nthreads, size_t smem, int nblocks,
                       cudaStream_t s) {
  if (kind != SWEEP_FIRST) return cudaErrorNotSupported;
  const int key = nspecies * 100 + L;
  if constexpr (sizeof(R) == 4) {
    switch (key) {
      case 108: return launch_first<R, 1, 8>(a, nthreads, smem, nblocks, s);
      case 116: return launch_first<R, 1, 16>(a, nthreads, smem, nblocks, s);
      case 208: return launch_first<R, 2, 8>(a, nthreads, smem, nblocks, s);
      case 216: return launch_first<R, 2, 16>(a, nthreads, smem, nblocks, s);
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (key) {
      case 104: return launch_first<R, 1, 4>(a, nthreads, smem, nblocks, s);
      case 108: return launch_first<R, 1, 8>(a, nthreads, smem, nblocks, s);
      case 204: return launch_first<R, 2, 4>(a, nthreads, smem, nblocks, s);
      case 208: return launch_first<R, 2, 8>(a, nthreads, smem, nblocks, s);
      default: return cudaErrorInvalidValue;
    }
  }
}

}  // namespace

cudaError_t launch_circ(const CircArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                        int nblocks, cudaStream_t s) {
  return launch_any<float>(a, nspecies, L, kind, nthreads, smem, nblocks, s);
}
cudaError_t launch_circ(const CircArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                        int nblocks, cudaStream_t s) {
  return launch_any<double>(a, nspecies, L, kind, nthreads, smem, nblocks, s);
}

}  // namespace etd
