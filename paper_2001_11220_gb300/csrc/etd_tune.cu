// etd_tune.cu -- tile-shape autotuner: for every axis, time each candidate
// (chunk length L, lines per tile, staged or register kernel, one line or a
// line pair per thread) on the context's stream with CUDA events and keep
// the fastest.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_context.h"

namespace etd {
bool plan_axis_ex(Instance &I, int a, int L, int max_threads, int nlb_force, bool reg_force, int pack);
bool plan_axis_tile(Instance &I, int a, int L, int NLB, int pk);
bool plan_axis_seg(Instance &I, int a, int L, int nlb, int mx, bool cluster);
bool cluster_plan_fits(const Instance &I, int a);
bool plan_axis_circ(Instance &I, int a, int L, int wb, int nc);
etd_status build_axis_tables(etd_ctx *ctx, Instance &I, int a);
}  // namespace etd

using namespace etd;

namespace {

struct Cand {
  int L, nlb;
  bool reg;
  int pack;
  bool tile = false;  // FP32 tile kernel with nlb lines per block
  int seg = 0;        // > 0: segmented register kernel with seg chunks per segment
  bool cluster = false;  // segmented as one cluster launch
  bool circ = false;     // circulant kernel of a periodic axis
};

bool plan_cand(Instance &I, int a, const Cand &c) {
  if (c.circ) return plan_axis_circ(I, a, c.L, c.nlb, c.pack);
  if (c.seg) return plan_axis_seg(I, a, c.L, c.nlb, c.seg, c.cluster) && cluster_plan_fits(I, a);
  if (c.tile) return plan_axis_tile(I, a, c.L, c.nlb, c.pack);
  return plan_axis_ex(I, a, c.L, ETD_MAX_BLOCK_THREADS, c.nlb, c.reg, c.pack);
}

// device time of axis a's sweep, averaged over `reps` steps
etd_status time_axis(etd_ctx *ctx, Instance &I, int a, void *U, int reps, double &ms) {
  const bool was = ctx->profiling;
  ctx->profiling = false;
  for (int r = 0; r < 2; ++r) {
    cudaError_t e = forward_step(I, U, 0.0, ctx->stream, nullptr);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune warm-up");
  }
  ctx->profiling = true;
  double acc[3] = {0, 0, 0};
  int64_t cnt[3] = {0, 0, 0};
  etd_profile_read(ctx, acc, cnt);  // drop stale records
  acc[0] = acc[1] = acc[2] = 0;
  cnt[0] = cnt[1] = cnt[2] = 0;
  for (int r = 0; r < reps; ++r) {
    cudaError_t e = forward_step(I, U, 0.0, ctx->stream, ctx);
    if (e != cudaSuccess) {
      ctx->profiling = was;
      return cuda_fail(ctx, e, "autotune step");
    }
  }
  etd_status st = etd_profile_read(ctx, acc, cnt);
  ctx->profiling = was;
  if (st != ETD_OK) return st;
  const int kind = I.plan[a].kind;
  ms = cnt[kind] ? acc[kind] / cnt[kind] : 1e30;
  return ETD_OK;
}

}  // namespace

extern "C" etd_status etd_autotune(etd_ctx *ctx, void *U_work) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_autotune on a batched context");
  if (!U_work) return fail(ctx, ETD_ERR_INVALID_ARG, "U_work is NULL");
  Instance &I = ctx->inst[0];
  if (I.coupled) return fail(ctx, ETD_ERR_UNSUPPORTED, "coupled contexts have one complex line kernel plan");
  drop_graphs(ctx);
  const int Ls32[] = {4, 8, 16}, Ls64[] = {4, 8};
  const int nlbs[] = {4, 8, 16, 32, 64};
  for (int a = 0; a < I.dim; ++a) {
    std::vector<Cand> cands;
    const int nL = I.real_bytes == 4 ? 3 : 2;
    for (int li = 0; li < nL; ++li) {
      const int L = I.real_bytes == 4 ? Ls32[li] : Ls64[li];
      for (int nlb : nlbs) cands.push_back({L, nlb, false, 1});
      cands.push_back({L, 0, true, 1});
      for (int nlb : {8, 16}) cands.push_back({L, nlb, true, 1});
      if (L == 8)
        for (int nlb : {0, 8, 16, 32}) cands.push_back({L, nlb, true, 2});  // line pairs (planner checks)
      if (I.real_bytes == 4 && L >= 8)
        for (int nlb : {16, 32})
          for (int pk : {1, 2}) cands.push_back({L, nlb, false, pk, true});  // tile kernels
      if (I.bc[a] == 2)  // periodic axis: circulant kernels (planner checks the shape; nlb = chunks per block)
        for (int wb : {8, 16, 32})
          for (int nc : {16, 32}) {  // chunks and lines per block (first axis: one shape)
            if (a == 0 && (wb != 16 || nc != 32)) continue;
            if (wb * nc > 512) continue;
            Cand c{L, wb, true, nc};
            c.circ = true;
            cands.push_back(c);
          }
      if ((I.n[a] + L - 1) / L > 32)  // long lines: segmented blocks (planner checks the shape)
        for (int mx : {16, 32})
          for (int nlb : {8, 16, 32})
            for (bool cl : {false, true}) cands.push_back({L, nlb, true, 1, false, mx, cl});
    }
    const AxisPlan keep = I.plan[a];
    double best = 1e30;
    Cand pick{keep.L, keep.sp.staged || keep.pk == 2 ? keep.nlb : 0, !keep.sp.staged, keep.pk,
              keep.sp.staged == 2, keep.nseg > 1 ? keep.mx : 0, keep.cluster, keep.circ};
    if (pick.tile) pick.nlb = keep.nlb * keep.pk;
    if (pick.seg) pick.nlb = keep.nlb;
    if (pick.circ) {  // circulant plans: chunks and lines per block
      pick.nlb = keep.mx;
      pick.pack = keep.nlb;
    }
    for (const Cand &c : cands) {
      if (!plan_cand(I, a, c)) continue;
      if (c.reg && I.plan[a].sp.staged) continue;
      etd_status st = build_axis_tables(ctx, I, a);
      if (st != ETD_OK) return st;
      double ms = 0;
      st = time_axis(ctx, I, a, U_work, 5, ms);
      if (st != ETD_OK) return st;
      if (std::getenv("ETD_TUNE_VERBOSE"))
        fprintf(stderr, "etd_autotune axis %d: L=%d nlb=%d mx=%d %s%s -> %.4f ms\n", a, c.L, I.plan[a].nlb, I.plan[a].mx,
                I.plan[a].circ ? "circulant" : I.plan[a].nseg > 1 ? (I.plan[a].cluster ? "cluster-segmented" : "segmented")
                : I.plan[a].sp.staged == 2 ? "tile"
                                                 : (I.plan[a].sp.staged ? "staged" : "register"),
                I.plan[a].pk == 2 ? " pairs" : "", ms);
      if (ms < best) {
        best = ms;
        pick = c;
      }
    }
    if (!plan_cand(I, a, pick))
      return fail(ctx, ETD_ERR_CUDA, "autotune: best candidate of axis %d no longer plans", a);
    etd_status st = build_axis_tables(ctx, I, a);
    if (st != ETD_OK) return st;
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "autotune synchronize");
  return ETD_OK;
}
