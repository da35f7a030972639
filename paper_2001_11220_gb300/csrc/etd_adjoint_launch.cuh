// etd_adjoint_launch.cuh -- launchers of the adjoint sweeps for one element type.
#pragma once

#include "etd_adjoint.cuh"
#include "etd_sweep_launch.cuh"

namespace etd {

template <typename R, int S, int L, int KIND>
cudaError_t launch_adj_one(const SweepArgs<R> &a, int nthreads, size_t smem, cudaStream_t s) {
  constexpr bool CONTIG = (KIND == ADJ_FIRST);
  auto fn = adjoint_kernel<R, S, L, CONTIG, KIND>;
  cudaError_t e = ensure_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<a.nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

#define ETD_ADJ_DISPATCH(CALL)                  \
  switch (nspecies * 1000 + L * 10 + kind) {    \
    case 1040: return CALL(1, 4, ADJ_FIRST);    \
    case 1041: return CALL(1, 4, ADJ_MIDDLE);   \
    case 1042: return CALL(1, 4, ADJ_LAST);     \
    case 1080: return CALL(1, 8, ADJ_FIRST);    \
    case 1081: return CALL(1, 8, ADJ_MIDDLE);   \
    case 1082: return CALL(1, 8, ADJ_LAST);     \
    case 2040: return CALL(2, 4, ADJ_FIRST);    \
    case 2041: return CALL(2, 4, ADJ_MIDDLE);   \
    case 2042: return CALL(2, 4, ADJ_LAST);     \
    case 2080: return CALL(2, 8, ADJ_FIRST);    \
    case 2081: return CALL(2, 8, ADJ_MIDDLE);   \
    case 2082: return CALL(2, 8, ADJ_LAST);     \
    default: return cudaErrorInvalidValue;      \
  }

template <typename R>
cudaError_t launch_misfit(const R *U, const R *T, R *Ub, long long n, double *loss, cudaStream_t s) {
  const int threads = 256;
  long long blocks = (n + threads - 1) / threads;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  misfit_kernel<R><<<(int)blocks, threads, 0, s>>>(U, T, Ub, n, loss);
  return cudaGetLastError();
}

}  // namespace etd
