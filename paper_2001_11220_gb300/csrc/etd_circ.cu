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
  auto fn = nthreads == 512 ? circ_first_kernel<R, S, L, 512> : circ_first_kernel<R, S, L, 256>;
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
  fn<<<nblocks, nthreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename R, int S, int L, int KIND, int WB, int NC>
cudaError_t launch_strided(const CircArgs<R> &a, size_t smem, int nblocks, cudaStream_t s, int *capacity) {
  auto fn = circ_strided_kernel<R, S, L, KIND, WB, NC>;
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)nblocks, 1, 1);
  cfg.blockDim = dim3(WB * NC, 1, 1);
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
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, WB * NC, smem);
      *capacity = per_sm;
      return e;
    }
    return cudaOccupancyMaxActiveClusters(capacity, fn, &cfg);
  }
  e = cudaLaunchKernelEx(&cfg, fn, a);
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

// strided sweeps, (chunks, lines) per block: FP32 (L = 16) 16 x 16, 16 x 32,
// 8 x 32, 32 x 16; FP64 (L = 8) 8 x 32, 16 x 16
template <typename R>
cudaError_t strided_any(const CircArgs<R> &a, int nspecies, int L, int kind, size_t smem, int nblocks,
                        cudaStream_t s, int *capacity) {
  constexpr int LL = sizeof(R) == 4 ? 16 : 8;
  if (L != LL) return cudaErrorInvalidValue;
  const int key = (a.wb * 100 + a.ncol) * 100 + nspecies * 10 + kind;
#define ETD_CIRC_STRIDED(WB_, NC_)                                                                         \
  case (WB_ * 100 + NC_) * 100 + 11: return launch_strided<R, 1, LL, SWEEP_MIDDLE, WB_, NC_>(a, smem, nblocks, s, capacity); \
  case (WB_ * 100 + NC_) * 100 + 12: return launch_strided<R, 1, LL, SWEEP_LAST, WB_, NC_>(a, smem, nblocks, s, capacity);   \
  case (WB_ * 100 + NC_) * 100 + 21: return launch_strided<R, 2, LL, SWEEP_MIDDLE, WB_, NC_>(a, smem, nblocks, s, capacity); \
  case (WB_ * 100 + NC_) * 100 + 22: return launch_strided<R, 2, LL, SWEEP_LAST, WB_, NC_>(a, smem, nblocks, s, capacity);
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
  return cudaErrorInvalidValue;
}

template <typename R>
cudaError_t launch_any(const CircArgs<R> &a, int nspecies, int L, int kind, int nthreads, size_t smem, int nblocks,
                       cudaStream_t s) {
  if (kind != SWEEP_FIRST) return strided_any<R>(a, nspecies, L, kind, smem, nblocks, s, nullptr);
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

cudaError_t circ_cluster_capacity(const CircArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters) {
  (void)nthreads;
  return strided_any<float>(a, nspecies, L, kind, smem, 1, nullptr, &nclusters);
}
cudaError_t circ_cluster_capacity(const CircArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters) {
  (void)nthreads;
  return strided_any<double>(a, nspecies, L, kind, smem, 1, nullptr, &nclusters);
}

cudaError_t circ_first_capacity(int real_bytes, int nspecies, int L, int nthreads, size_t smem, int &blocks_per_sm) {
  blocks_per_sm = 0;
  const void *fn = nullptr;
  const int key = nspecies * 100 + L;
  const bool big = nthreads == 512;
#define ETD_FIRST_FN(R_, S_, L_) \
  (big ? (const void *)circ_first_kernel<R_, S_, L_, 512> : (const void *)circ_first_kernel<R_, S_, L_, 256>)
  if (real_bytes == 4) {
    switch (key) {
      case 108: fn = ETD_FIRST_FN(float, 1, 8); break;
      case 116: fn = ETD_FIRST_FN(float, 1, 16); break;
      case 208: fn = ETD_FIRST_FN(float, 2, 8); break;
      case 216: fn = ETD_FIRST_FN(float, 2, 16); break;
      default: return cudaErrorInvalidValue;
    }
  } else {
    switch (key) {
      case 104: fn = ETD_FIRST_FN(double, 1, 4); break;
      case 108: fn = ETD_FIRST_FN(double, 1, 8); break;
      case 204: fn = ETD_FIRST_FN(double, 2, 4); break;
      case 208: fn = ETD_FIRST_FN(double, 2, 8); break;
      default: return cudaErrorInvalidValue;
    }
  }
#undef ETD_FIRST_FN
  cudaError_t e = ensure_dyn_smem(fn, smem);
  if (e != cudaSuccess) return e;
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
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_circ_status, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  if (v) {
    const int zero = 0;
    cudaMemcpyToSymbol(g_circ_status, &zero, sizeof(int));
  }
  return v;
}

}  // namespace etd
