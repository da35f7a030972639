// etd_context.h -- the opaque etd_ctx and per-instance state of libetdrdpif.
#pragma once

#include <cuda_runtime.h>

#include <cstdlib>
#include <cstring>
#include <list>
#include <string>
#include <utility>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_circ.h"
#include "etd_cplx.h"
#include "etd_internal.h"

#define ETD_MAX_BLOCK_THREADS 512

namespace etd {

// device memory of an instance's tables: 256-byte aligned pieces carved
// from blocks of at least 1 MiB
struct DeviceArena {
  std::vector<void *> blocks;
  size_t used = 0, cap = 0;
  void *put(const void *host, size_t bytes, cudaError_t &err) {
    if (err != cudaSuccess) return nullptr;
    const size_t need = (bytes + 255) & ~(size_t)255;
    if (blocks.empty() || used + need > cap) {
      void *d = nullptr;
      const size_t sz = need > ((size_t)1 << 20) ? need : ((size_t)1 << 20);
      err = cudaMalloc(&d, sz);
      if (err != cudaSuccess) return nullptr;
      blocks.push_back(d);
      used = 0;
      cap = sz;
    }
    void *p = (unsigned char *)blocks.back() + used;
    used += need;
    err = cudaMemcpy(p, host, bytes, cudaMemcpyHostToDevice);
    return p;
  }
  void release() {
    for (void *p : blocks) cudaFree(p);
    blocks.clear();
    used = cap = 0;
  }
};

// launch plan of one axis sweep
struct AxisPlan {
  int kind = 0;        // SweepKind
  int L = 8;           // chunk length (elements per thread)
  int m = 1;           // chunks per line
  int nlb = 1;         // lines per block
  int pitch = 1;       // shared-memory pitch
  int nthreads = 1;    // nlb * m
  int nlo_blocks = 1;  // strided sweeps: blocks along the contiguous line index
  int nblocks = 1;
  long long st = 1;    // element stride of the axis
  long long nlines = 1;
  size_t smem = 0;     // register kernel: shared memory bytes
  int pk = 1;          // 2: register kernel on FP32 line pairs (nlb counts pairs)
  int mx = 1;          // chunks per block along the line (= m unless segmented)
  int nseg = 1;        // segments per line (> 1: segmented sweep, see SegPhase)
  bool cluster = false;  // segmented in one launch: the segments of a line group form a cluster
  void *seg_buf = nullptr;  // segmented sweeps: summaries, carries, scalars (owned)
  size_t seg_bytes = 0;
  StagePlan sp{};      // staged (persistent) kernel plan; sp.staged = 0 -> register kernel
  bool circ = false;   // periodic axis solved by the circulant kernels (etd_circ.cuh); nlb = lines per block
  bool circ_lean = false;  // strided circulant plan with its exchange tables in global memory (2 blocks per SM)
};

// one problem: grid, coefficients, tables, plans and scratch
struct Instance {
  int dim = 2, S = 1, real_bytes = 8;
  long long n[3] = {1, 1, 1};
  int bc[3] = {0, 0, 0};
  double length[3] = {1, 1, 1};
  long long N = 1;
  double D[MAX_SPECIES] = {0, 0};
  double k = 0;
  int rkind = 0;
  double rp[8] = {0};
  bool has_source = false;
  double src_lf = 0;
  void *phi[3] = {nullptr, nullptr, nullptr};
  AxisPlan plan[3];
  // [transpose][axis][species][gamma index: 0 -> 1, 1 -> 3, 2 -> 4]
  MatTab<float> tab32[2][3][MAX_SPECIES][3];
  MatTab<double> tab64[2][3][MAX_SPECIES][3];
  void *scratch[3] = {nullptr, nullptr, nullptr};  // c_U, c_f, w
  // adjoint: launch plans and line tables at the adjoint chunk length
  bool adj_ready = false;
  AxisPlan aplan[3];
  MatTab<float> atab32[2][3][MAX_SPECIES][3];
  MatTab<double> atab64[2][3][MAX_SPECIES][3];
  // adjoint on the circulant factorisation (periodic axes with n a multiple of the chunk length)
  bool acirc[3] = {false, false, false};
  SweepArgs<float>::CircLine acl32[3][MAX_SPECIES][3];
  SweepArgs<double>::CircLine acl64[3][MAX_SPECIES][3];
  DeviceArena arena;                               // source tables, adjoint tables
  void *axis_tables[3] = {nullptr, nullptr, nullptr};  // forward line tables of each axis (one block)
  // circulant plans: kernel arguments with every coefficient filled in (only
  // the field pointers change per launch) and their device power tables
  CircArgs<float> circ32[3];
  CircArgs<double> circ64[3];
  void *circ_tables[3] = {nullptr, nullptr, nullptr};
  // coupled two-species diffusion Dm = [[dcp, -dcq], [dcq, dcp]] (complex p + i q): complex line kernels
  bool coupled = false;
  double dcp = 0, dcq = 0;
  CplxAxis cax[3];
  std::vector<void *> owned;  // cudaMalloc'ed buffers freed by etd_destroy
};

// one sweep of axis a (segmented plans: all of its launches), stream-ordered
template <typename R>
cudaError_t run_sweep(const Instance &I, int a, SweepArgs<R> &A, cudaStream_t s);

struct GraphKey {
  const void *U;
  const void *U2;
  double t0;
  int64_t nsteps;
  bool operator==(const GraphKey &o) const {
    return U == o.U && U2 == o.U2 && t0 == o.t0 && nsteps == o.nsteps;
  }
};

}  // namespace etd

struct etd_ctx {
  cudaStream_t stream = nullptr;
  int32_t precision = 0;
  bool batched = false;
  std::vector<etd::Instance> inst;
  std::string err = "no error";
  void *host_state = nullptr;           // device copy used by etd_run_host
  std::vector<void *> owned;            // context-level device buffers
  void *finite_word = nullptr;          // etd_check_finite: smallest non-finite index (owned)
  std::list<std::pair<etd::GraphKey, cudaGraphExec_t>> graphs;  // captured multi-step runs
  // batched launch data: per axis, SweepArgs<R>[ninst] and block prefix sums on the device
  void *batch_args[3] = {nullptr, nullptr, nullptr};
  int *batch_block_start[3] = {nullptr, nullptr, nullptr};
  int batch_total_blocks[3] = {0, 0, 0};
  int batch_threads[3] = {0, 0, 0};
  size_t batch_smem[3] = {0, 0, 0};
  int batch_L[3] = {0, 0, 0};
  std::vector<void *> batch_states;  // state pointers the device args were built for
  void *batch_scratch = nullptr;     // scratch of every instance, one allocation
  // persistent ensemble step (one launch per step): work list, counters, status
  bool ens_on = false;               // else one launch per sweep kind
  bool ens_circ = true;              // periodic whole-chunk lines on the circulant factorisation
  int2 *ens_items = nullptr;         // (axis << 24 | instance, block), dependencies first
  int ens_nitems = 0;
  unsigned *ens_queue = nullptr;     // [2], reset by each launch's last block
  int *ens_done = nullptr;           // [dim - 1][ninst] finished blocks, reset likewise
  int *ens_status = nullptr;         // ENS_STATUS_WORDS
  int ens_threads = 0;
  size_t ens_smem = 0;
  int ens_grid = 0;
  int ens_max_threads = 256;         // largest block of the persistent step (2 resident per SM)
  double ens_wait_s = 1.0;           // limit of one dependency wait
  double ens_window_mb = 0.0;        // scratch MB per instance group of the interleaved order (0: by axis)
  // per-sweep profiling (etd_profile)
  bool profiling = false;
  std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
  std::vector<cudaEvent_t> prof_pool;
  // adjoint / gradient workspace (allocated on first use)
  void *adj_ws = nullptr;         // 9 carried fields: forward axis-0 outputs, axis-1 outputs, adjoint fields
  void *adj_ubar[2] = {nullptr, nullptr};
  double *adj_acc = nullptr;      // dL/dD[2], dL/dparams[8], loss
  double *adj_part = nullptr;     // per-block partial sums of the adjoint sweeps and the misfit
  void *ckpt = nullptr;           // checkpoint states
  size_t ckpt_states = 0;
  void *seg = nullptr;            // states of one recomputed segment
  size_t seg_states = 0;
  void *seg_mid = nullptr;        // first (and middle) sweep outputs of every step of the segment
  size_t seg_mid_steps = 0;
};

namespace etd {

etd_status fail(etd_ctx *ctx, etd_status st, const char *fmt, ...);
etd_status cuda_fail(etd_ctx *ctx, cudaError_t e, const char *what);
cudaError_t forward_step(const Instance &I, void *U, double t, cudaStream_t s, etd_ctx *prof = nullptr);
cudaError_t prof_begin(etd_ctx *ctx, cudaStream_t s, cudaEvent_t &ev);
cudaError_t prof_end(etd_ctx *ctx, cudaStream_t s, int kind, cudaEvent_t ev0);
template <typename R> void fill_args(const Instance &I, int a, int transpose, SweepArgs<R> &A);

// Destroys every cached executable graph of the context (they hold the old
// plans, streams or state pointers) and empties the cache.
inline void drop_graphs(etd_ctx *ctx) {
  for (auto &kv : ctx->graphs) cudaGraphExecDestroy(kv.second);
  ctx->graphs.clear();
}

// Enqueue nsteps steps with enqueue(stream, step_index).  Runs of two or more
// steps on a non-legacy stream are captured once into a CUDA graph (cached
// by key) and replayed; otherwise kernels are launched directly.
template <typename F>
etd_status run_steps(etd_ctx *ctx, F enqueue, GraphKey key, int64_t nsteps) {
  cudaStream_t s = ctx->stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  bool graphs = nsteps >= 2 && s != nullptr && !ctx->profiling && std::getenv("ETD_NO_GRAPHS") == nullptr;
  if (graphs && cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) graphs = false;
  if (!graphs) {
    for (int64_t n = 0; n < nsteps; ++n) {
      cudaError_t e = enqueue(s, n);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    }
    return ETD_OK;
  }
  for (auto it = ctx->graphs.begin(); it != ctx->graphs.end(); ++it)
    if (it->first == key) {
      cudaError_t e = cudaGraphLaunch(it->second, s);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
      ctx->graphs.splice(ctx->graphs.begin(), ctx->graphs, it);
      return ETD_OK;
    }
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "begin capture");
  cudaError_t le = cudaSuccess;
  for (int64_t n = 0; n < nsteps && le == cudaSuccess; ++n) le = enqueue(s, n);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(s, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(ctx, le, "step launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
  ctx->graphs.emplace_front(key, ex);
  while (ctx->graphs.size() > 4) {
    cudaGraphExecDestroy(ctx->graphs.back().second);
    ctx->graphs.pop_back();
  }
  e = cudaGraphLaunch(ex, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "graph launch");
  return ETD_OK;
}

}  // namespace etd
