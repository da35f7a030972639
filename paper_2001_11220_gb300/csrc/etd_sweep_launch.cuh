// etd_sweep_launch.cuh -- host launchers for the sweep kernels of one element
// type; included once per element type by etd_sweep_f32.cu / etd_sweep_f64.cu.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>
#include <unordered_map>

#include "etd_sweep_smem.cuh"

namespace etd {

// raise the dynamic shared-memory limit of a kernel once per requested size
inline cudaError_t ensure_smem(const void *fn, size_t smem) {
  static std::mutex mu;
  static std::unordered_map<const void *, size_t> done;
  if (smem <= 48 * 1024) return cudaSuccess;
  std::lock_guard<std::mutex> g(mu);
  auto it = done.find(fn);
  if (it != done.end() && it->second >= smem) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done[fn] = smem;
  return e;
}

// resident blocks per SM of a kernel configuration times the SM count (cached)
inline cudaError_t persistent_grid(const void *fn, int nthreads, size_t smem, int ntiles, int &grid) {
  static std::mutex mu;
  static std::unordered_map<std::string, int> cache;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  char key[96];
  snprintf(key, sizeof(key), "%p/%d/%zu/%d", fn, nthreads, smem, dev);
  int per_sm = 0, nsm = 0;
  {
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
      grid = std::min(ntiles, it->second);
      return cudaSuccess;
    }
  }
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nthreads, smem);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int resident = std::max(1, per_sm) * nsm;
  {
    std::lock_guard<std::mutex> g(mu);
    cache[key] = resident;
  }
  grid = std::min(ntiles, resident);
  return cudaSuccess;
}

template <typename R>
inline cudaError_t launch_register(void (*fn)(const SweepArgs<R>), const SweepArgs<R> &a, int nthreads, size_t smem,
                                   cudaStream_t s) {
  cudaError_t e = ensure_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<a.nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R, int S, int L, int KIND>
cudaError_t launch_one(const SweepArgs<R> &a, int nthreads, size_t smem, cudaStream_t s) {
  constexpr bool CONTIG = (KIND == SWEEP_FIRST);
  if (a.sp.staged == 2) return cudaErrorInvalidValue;  // tile kernels: launch_tile
  if (a.sp.staged) {
    auto fn = sweep_staged_kernel<R, S, L, CONTIG, KIND>;
    cudaError_t e = ensure_smem((const void *)fn, a.sp.bytes);
    if (e != cudaSuccess) return e;
    int grid = 0;
    e = persistent_grid((const void *)fn, nthreads, a.sp.bytes, a.sp.ntiles, grid);
    if (e != cudaSuccess) return e;
    fn<<<grid, nthreads, a.sp.bytes, s>>>(a);
    return cudaGetLastError();
  }
  if constexpr (sizeof(R) == 4 && !CONTIG && L == 8) {
    if (a.pk == 2) return launch_register<R>(sweep_kernel<R, S, L, false, KIND, 2>, a, nthreads, smem, s);
  }
  if (a.pk != 1) return cudaErrorInvalidValue;
  return launch_register<R>(sweep_kernel<R, S, L, CONTIG, KIND>, a, nthreads, smem, s);
}

template <typename R, int S, int L, int KIND>
cudaError_t launch_one_batched(const SweepArgs<R> *args, const int *bs, int ninst, int total, int nthreads,
                               size_t smem, cudaStream_t s, double t_eval) {
  constexpr bool CONTIG = (KIND == SWEEP_FIRST);
  auto fn = sweep_kernel_batched<R, S, L, CONTIG, KIND>;
  cudaError_t e = ensure_smem((const void *)fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<total, nthreads, smem, s>>>(args, bs, ninst, t_eval, (R)std::exp(-t_eval));
  return cudaGetLastError();
}

template <typename R, int S, int KIND>
cudaError_t launch_seg_carry_one(const SweepArgs<R> &a, int q0, int nq, cudaStream_t s) {
  const long long work = (long long)nq * a.nlines;
  const int threads = 256;
  const int blocks = (int)std::min<long long>((work + threads - 1) / threads, 152LL * 16);
  seg_carry_kernel<R, S, KIND><<<std::max(blocks, 1), threads, 0, s>>>(a, q0, nq);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_seg_carry_t(const SweepArgs<R> &a, int nspecies, int kind, int q0, int nq, cudaStream_t s) {
  switch (nspecies * 10 + kind) {
    case 10: return launch_seg_carry_one<R, 1, SWEEP_FIRST>(a, q0, nq, s);
    case 11: return launch_seg_carry_one<R, 1, SWEEP_MIDDLE>(a, q0, nq, s);
    case 12: return launch_seg_carry_one<R, 1, SWEEP_LAST>(a, q0, nq, s);
    case 20: return launch_seg_carry_one<R, 2, SWEEP_FIRST>(a, q0, nq, s);
    case 21: return launch_seg_carry_one<R, 2, SWEEP_MIDDLE>(a, q0, nq, s);
    case 22: return launch_seg_carry_one<R, 2, SWEEP_LAST>(a, q0, nq, s);
    default: return cudaErrorInvalidValue;
  }
}

#define ETD_DISPATCH(CALL)                                                        \
  switch (nspecies * 1000 + L * 10 + kind) {                                      \
    case 1040: return CALL(1, 4, SWEEP_FIRST);                                    \
    case 1041: return CALL(1, 4, SWEEP_MIDDLE);                                   \
    case 1042: return CALL(1, 4, SWEEP_LAST);                                     \
    case 1080: return CALL(1, 8, SWEEP_FIRST);                                    \
    case 1081: return CALL(1, 8, SWEEP_MIDDLE);                                   \
    case 1082: return CALL(1, 8, SWEEP_LAST);                                     \
    case 1160: return CALL(1, 16, SWEEP_FIRST);                                   \
    case 1161: return CALL(1, 16, SWEEP_MIDDLE);                                  \
    case 1162: return CALL(1, 16, SWEEP_LAST);                                    \
    case 2040: return CALL(2, 4, SWEEP_FIRST);                                    \
    case 2041: return CALL(2, 4, SWEEP_MIDDLE);                                   \
    case 2042: return CALL(2, 4, SWEEP_LAST);                                     \
    case 2080: return CALL(2, 8, SWEEP_FIRST);                                    \
    case 2081: return CALL(2, 8, SWEEP_MIDDLE);                                   \
    case 2082: return CALL(2, 8, SWEEP_LAST);                                     \
    case 2160: return CALL(2, 16, SWEEP_FIRST);                                   \
    case 2161: return CALL(2, 16, SWEEP_MIDDLE);                                  \
    case 2162: return CALL(2, 16, SWEEP_LAST);                                    \
    default: return cudaErrorInvalidValue;                                        \
  }

}  // namespace etd
