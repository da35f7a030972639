// etd_sweep_cluster.cu -- cluster-segmented register sweeps (both element
// types): the nseg blocks that hold the segments of a group of long lines run
// as one thread-block cluster and exchange their segment summaries through
// distributed shared memory, so a sweep is a single launch.
#include "etd_sweep_launch.cuh"

namespace etd {

namespace {

// launch configuration: the nseg blocks of every line group (consecutive
// block indices) form one cluster
template <typename R>
cudaError_t cluster_config(const void *fn, const SweepArgs<R> &a, int nthreads, size_t smem, cudaStream_t s,
                           cudaLaunchConfig_t &cfg, cudaLaunchAttribute *attr) {
  if (a.segphase != SEG_CLUSTER || a.nseg < 2 || a.nseg > ETD_MAX_CLUSTER || a.nblocks % a.nseg != 0)
    return cudaErrorInvalidValue;
  cudaError_t e = ensure_smem(fn, smem);
  if (e != cudaSuccess) return e;
  if (a.nseg > 8) {
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cfg = cudaLaunchConfig_t{};
  cfg.gridDim = dim3((unsigned)a.nblocks);
  cfg.blockDim = dim3((unsigned)nthreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.nseg;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaSuccess;
}

// register kernels on single lines with L = 8 or 16 (FP32) / 4 or 8 (FP64)
template <typename R, int L>
constexpr bool cluster_shape() {
  return sizeof(R) == 4 ? (L == 8 || L == 16) : (L == 4 || L == 8);
}

template <typename R, int S, int L, int KIND>
cudaError_t cluster_one(const SweepArgs<R> &a, int nthreads, size_t smem, cudaStream_t s, int *capacity) {
  if constexpr (!cluster_shape<R, L>()) {
    return cudaErrorInvalidValue;
  } else {
    constexpr bool CONTIG = (KIND == SWEEP_FIRST);
    if (a.pk != 1 || a.sp.staged) return cudaErrorInvalidValue;
    auto fn = sweep_kernel<R, S, L, CONTIG, KIND, 1, true>;
    cudaLaunchConfig_t cfg;
    cudaLaunchAttribute attr[1];
    cudaError_t e = cluster_config<R>((const void *)fn, a, nthreads, smem, s, cfg, attr);
    if (e != cudaSuccess) return e;
    if (capacity) return cudaOccupancyMaxActiveClusters(capacity, (const void *)fn, &cfg);
    return cudaLaunchKernelEx(&cfg, fn, a);
  }
}

template <typename R>
cudaError_t cluster_dispatch(const SweepArgs<R> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                             cudaStream_t s, int *capacity) {
#define CALL(S_, L_, K_) cluster_one<R, S_, L_, K_>(a, nthreads, smem, s, capacity)
  ETD_DISPATCH(CALL)
#undef CALL
}

}  // namespace

cudaError_t launch_sweep_cluster(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                 cudaStream_t s) {
  return cluster_dispatch<float>(a, nspecies, L, kind, nthreads, smem, s, nullptr);
}
cudaError_t launch_sweep_cluster(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads,
                                 size_t smem, cudaStream_t s) {
  return cluster_dispatch<double>(a, nspecies, L, kind, nthreads, smem, s, nullptr);
}

cudaError_t sweep_cluster_capacity(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads,
                                   size_t smem, int &nclusters) {
  nclusters = 0;
  return cluster_dispatch<float>(a, nspecies, L, kind, nthreads, smem, nullptr, &nclusters);
}
cudaError_t sweep_cluster_capacity(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads,
                                   size_t smem, int &nclusters) {
  nclusters = 0;
  return cluster_dispatch<double>(a, nspecies, L, kind, nthreads, smem, nullptr, &nclusters);
}

}  // namespace etd
