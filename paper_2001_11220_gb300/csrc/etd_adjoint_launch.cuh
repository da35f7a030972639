// etd_adjoint_launch.cuh -- launchers of the adjoint sweeps for one element type.
#pragma once

#include "etd_adjoint.cuh"
#include "etd_sweep_launch.cuh"

namespace etd {

template <typename R, int S, int L, int KIND, bool CIRC = false>
cudaError_t launch_adj_one(const SweepArgs<R> &a, int nthreads, size_t smem, cudaStream_t s) {
  constexpr bool CONTIG = (KIND == ADJ_FIRST);
  auto fn = adjoint_kernel<R, S, L, CONTIG, KIND, CIRC>;
  cudaError_t e = ensure_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<a.nblocks, nthreads, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_partials_kernel<<<1, 32 * (MAX_SPECIES + 8), 0, s>>>(a.part, a.nblocks, MAX_SPECIES + 8, a.acc);
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

inline int misfit_blocks(long long n) {
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  return blocks < 1 ? 1 : (int)blocks;
}

template <typename R>
cudaError_t launch_misfit(const R *U, const R *T, R *Ub, long long n, double *loss, double *part, cudaStream_t s) {
  const int blocks = misfit_blocks(n);
  misfit_kernel<R><<<blocks, 256, 0, s>>>(U, T, Ub, n, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  reduce_partials_kernel<<<1, 32, 0, s>>>(part, blocks, 1, loss);
  return cudaGetLastError();
}

}  // namespace etd
