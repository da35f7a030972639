// etd_circ.cu -- launchers of the circulant sweeps of periodic axes.
#include <cuda_runtime.h>

#include "etd_circ.cuh"

namespace etd {

namespace {

template <typename R>
cudaError_t ensure_dyn_smem(CircKernel<R> fn, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

template <typename R>
cudaError_t launch_first(CircKernel<R> fn, const CircArgs<R> &a, int nthreads, size_t smem, int nblocks,
                         cudaStream_t s) {
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

// capacity != nullptr: only report the clusters (cs > 1) or blocks per SM
// (cs = 1) that fit at once
template <typename R>
cudaError_t launch_strided(CircKernel<R> fn, const CircArgs<R> &a, size_t smem, int nblocks, cudaStream_t s,
                           int *capacity) {
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblocks, 1, 1);
  cfg.blockDim = dim3((unsigned)(a.wb * a.ncol), 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (a.cs > 1) {
    if (a.cs > 8) {
      e = cudaFuncSetAttribute((const void *)fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) return e;
    }
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)a.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  if (capacity) {
    *capacity = 0;
    cfg.gridDim = dim3((unsigned)(a.cs > 1 ? a.cs : 1), 1, 1);
    if (a.cs <= 1) {
      int per_sm = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, a.wb * a.ncol, smem);
      *capacity = per_sm;
      return e;
    }
    return cudaOccupancyMaxActiveClusters(capacity, fn, &cfg);
  }
  e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// strided kernels, (chunks, lines) per block: FP32 (L = 16) 16 x 16, 16 x 32,
// 8 x 32, 32 x 16; FP64 (L = 8) 8 x 32, 16 x 16.  A kernel with the reaction
// fixed at compile time where one is compiled (FP32, two species), else the
// generic one.
template <typename R>
CircKernel<R> strided_kernel(int nspecies, int L, int kind, int wb, int nc, int rkind) {
  constexpr int LL = sizeof(R) == 4 ? 16 : 8;
  if (L != LL) return nullptr;
  if constexpr (sizeof(R) == 4) {
    if (nspecies == 2)
      if (CircKernel<float> k = circ_strided_kernel_rk(kind, wb, nc, rkind)) return k;
  }
  const int key = (wb * 100 + nc) * 100 + nspecies * 10 + kind;
#define ETD_CIRC_STRIDED(WB_, NC_)                                                             \
  case (WB_ * 100 + NC_) * 100 + 11: return circ_strided_kernel<R, 1, LL, SWEEP_MIDDLE, WB_, NC_>; \
  case (WB_ * 100 + NC_) * 100 + 12: return circ_strided_kernel<R, 1, LL, SWEEP_LAST, WB_, NC_>;   \
  case (WB_ * 100 + NC_) * 100 + 21: return circ_strided_kernel<R, 2, LL, SWEEP_MIDDLE, WB_, NC_>; \
  case (WB_ * 100 + NC_) * 100 + 22: return circ_strided_kernel<R, 2, LL, SWEEP_LAST, WB_, NC_>;
  if constexpr (sizeof(R) == 4) {
    switch (key) {
      ETD_CIRC_STRIDED(16, 16)
      ETD_CIRC_STRIDED(16, 32)
      ETD_CIRC_STRIDED(8, 32)
      ETD_CIRC_STRIDED(32, 16)
      default: break;
    }
  } else {
    switch (key) {
      ETD_CIRC_STRIDED(8, 32)
      ETD_CIRC_STRIDED(16, 16)
      default: break;
    }
  }
#undef ETD_CIRC_STRIDED
  return nullptr;
}

// first-axis kernels: FP32 L = 8, 16; FP64 L = 4, 8; 256 or 512 threads
template <typename R>
CircKernel<R> first_kernel(int nspecies, int L, int nthreads, int rkind) {
  if constexpr (sizeof(R) == 4) {
    if (nspecies == 2)
      if (CircKernel<float> k = circ_first_kernel_rk(L, nthreads, rkind)) return k;
  }
  const bool big = nthreads == 512;
  const int key = nspecies * 100 + L;
#define ETD_FIRST_FN(S_, L_) (big ? circ_first_kernel<R, S_, L_, 512> : circ_first_kernel<R, S_, L_, 256>)
  if constexpr (sizeof(R) == 4) {
    switch (key) {
      case 108: return ETD_FIRST_FN(1, 8);
      case 116: return ETD_FIRST_FN(1, 16);
      case 208: return ETD_FIRST_FN(2, 8);
      case 216: return ETD_FIRST_FN(2, 16);
      default: return nullptr;
    }
  } else {
    switch (key) {
      case 104: return ETD_FIRST_FN(1, 4);
      case 108: return ETD_FIRST_FN(1, 8);
      case 204: return ETD_FIRST_FN(2, 4);
      case 208: return ETD_FIRST_FN(2, 8);
      default: return nullptr;
    }
  }
#undef ETD_FIRST_FN
}

template <typename R>
cudaError_t launch_any(const CircArgs<R> &a, int nspecies, int L, int kind, int nthreads, size_t smem, int nblocks,
                       cudaStream_t s) {
  if (kind != SWEEP_FIRST) {
    CircKernel<R> fn = strided_kernel<R>(nspecies, L, kind, a.wb, a.ncol, a.rkind);
    return fn ? launch_strided<R>(fn, a, smem, nblocks, s, nullptr) : cudaErrorInvalidValue;
  }
  CircKernel<R> fn = first_kernel<R>(nspecies, L, nthreads, a.rkind);
  return fn ? launch_first<R>(fn, a, nthreads, smem, nblocks, s) : cudaErrorInvalidValue;
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

cudaError_t circ_cluster_capacity(const CircArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters) {
  (void)nthreads;
  CircKernel<float> fn = strided_kernel<float>(nspecies, L, kind, a.wb, a.ncol, a.rkind);
  return fn ? launch_strided<float>(fn, a, smem, 1, nullptr, &nclusters) : cudaErrorInvalidValue;
}
cudaError_t circ_cluster_capacity(const CircArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters) {
  (void)nthreads;
  CircKernel<double> fn = strided_kernel<double>(nspecies, L, kind, a.wb, a.ncol, a.rkind);
  return fn ? launch_strided<double>(fn, a, smem, 1, nullptr, &nclusters) : cudaErrorInvalidValue;
}

cudaError_t circ_first_capacity(int real_bytes, int nspecies, int L, int nthreads, int rkind, size_t smem,
                                int &blocks_per_sm) {
  blocks_per_sm = 0;
  const void *fn = real_bytes == 4 ? (const void *)first_kernel<float>(nspecies, L, nthreads, rkind)
                                   : (const void *)first_kernel<double>(nspecies, L, nthreads, rkind);
  if (!fn) return cudaErrorInvalidValue;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, fn, nthreads, smem);
}

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiled)p;
    else
      cudaGetLastError();
  }
  return fn;
}

template <typename R>
bool encode_maps(CircArgs<R> &a, int nspecies, int rows) {
  EncodeTiled enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)a.st, (cuuint64_t)(a.N / a.st), (cuuint64_t)nspecies};
  const cuuint64_t strides[2] = {(cuuint64_t)a.st * sizeof(R), (cuuint64_t)a.N * sizeof(R)};
  const cuuint32_t box[3] = {32u, (cuuint32_t)rows, 1u};
  const cuuint32_t estr[3] = {1u, 1u, 1u};
  const CUtensorMapDataType dt = sizeof(R) == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
  for (int f = 0; f < 3; ++f) {
    if (!a.in[f]) return false;
    if (enc(&a.tmap[f], dt, 3, (void *)a.in[f], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

}  // namespace

bool circ_encode_maps(CircArgs<float> &a, int nspecies, int rows) { return encode_maps<float>(a, nspecies, rows); }
bool circ_encode_maps(CircArgs<double> &a, int nspecies, int rows) { return encode_maps<double>(a, nspecies, rows); }

int circ_take_status() {
  return take_status_here() | circ_take_status_rk_first() | circ_take_status_rk_strided();
}

}  // namespace etd
