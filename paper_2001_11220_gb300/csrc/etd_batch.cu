// etd_batch.cu -- batched ensemble: many independent problems of uneven size
// advanced together, one kernel launch per sweep kind covering every
// instance (blocks find their instance by a prefix sum over block counts);
// multi-step runs are captured into a CUDA graph.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_context.h"
#include "etd_internal.h"
#include "etd_circ.h"
#include "etd_tables.h"

namespace etd {
etd_status validate_problem(const etd_grid *grid, const double *D, const etd_reaction *rx, double k,
                            int32_t precision);
bool plan_axis_ex(Instance &I, int a, int L, int max_threads, int nlb_force, bool reg_force, int pack);
etd_status build_axis_tables(etd_ctx *ctx, Instance &I, int a);
etd_status init_instance(etd_ctx *ctx, Instance &I, const etd_grid *grid, const double *D, const etd_reaction *rx,
                         double k, int32_t precision, bool with_scratch);
}  // namespace etd

using namespace etd;

namespace {

template <typename R>
etd_status upload_batch_args(etd_ctx *ctx, void *const *U) {
  const int ninst = (int)ctx->inst.size();
  const int dim = ctx->inst[0].dim;
  std::vector<SweepArgs<R>> args(ninst);
  for (int a = 0; a < dim; ++a) {
    for (int i = 0; i < ninst; ++i) {
      const Instance &I = ctx->inst[i];
      SweepArgs<R> &A = args[i];
      fill_args<R>(I, a, 0, A);
      // persistent step: periodic lines of whole chunks on the circulant
      // factorisation (ETD_ENSEMBLE_CIRC=0 keeps the tables)
      const AxisPlan &P = I.plan[a];
      if (ctx->ens_on && ctx->ens_circ && I.bc[a] == BC_PERIODIC && P.nseg == 1 && P.pk == 1 &&
          I.n[a] % P.L == 0) {
        static const double gammas[3] = {1.0, 3.0, 4.0};
        const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
        for (int s = 0; s < I.S; ++s)
          for (int g = 0; g < 3; ++g) {
            CircHost H;
            circ_coeffs((I.k / gammas[g]) * I.D[s] / (h * h), (int)I.n[a], P.L, H);
            auto &C = A.cl[s][g];
            C.lam = (R)H.lam;
            C.lamL = (R)H.lamL;
            C.kap = (R)H.kap;
            C.inv1m = (R)H.inv1m;
            C.ialpha = (R)(1.0 / H.alpha);
            for (int t = 0; t < 16; ++t) C.pw[t] = (R)H.pw[t];
          }
        A.circ_fwd = 1;
      }
      R *cu = (R *)I.scratch[0], *cf = (R *)I.scratch[1], *w = (R *)I.scratch[2];
      const int kind = I.plan[a].kind;
      if (kind == SWEEP_FIRST) {
        A.in[0] = (const R *)U[i];
        A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
      } else if (kind == SWEEP_MIDDLE) {
        A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
        A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
      } else {
        A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
        A.out[0] = (R *)U[i];
      }
    }
    // ordered on the context's stream: launches still in flight keep reading the old arguments
    cudaError_t e = cudaMemcpyAsync(ctx->batch_args[a], args.data(), sizeof(SweepArgs<R>) * ninst,
                                    cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // host buffer must outlive the copy
    if (e != cudaSuccess) return cuda_fail(ctx, e, "batch argument upload");
  }
  return ETD_OK;
}

template <typename R>
cudaError_t ensemble_launch(etd_ctx *ctx, const EnsArgs<R> &E, cudaStream_t s, int *resident) {
  const Instance &I0 = ctx->inst[0];
  const int LS = I0.dim > 1 ? ctx->batch_L[1] : ctx->batch_L[0];
  if (I0.dim == 2)
    return launch_ensemble_2d(E, I0.S, ctx->batch_L[0], LS, ctx->ens_threads, ctx->ens_smem, ctx->ens_grid, s,
                              resident);
  return launch_ensemble_3d(E, I0.S, ctx->batch_L[0], LS, ctx->ens_threads, ctx->ens_smem, ctx->ens_grid, s,
                            resident);
}

// Work list of the persistent step.  Instances are taken in groups whose
// scratch (3 fields) adds up to about ens_window_mb; group g's sweep a is
// queued in round g + a, after the first sweep of group g + a, so every item
// comes after the items it depends on (sweep a - 1 of its instance, one round
// earlier) and the scratch a group writes is read back while it may still be
// in L2.  ens_window_mb = 0: one group (every instance's sweep 0, then 1, ...).
etd_status plan_ensemble_step(etd_ctx *ctx) {
  const int ninst = (int)ctx->inst.size();
  const int dim = ctx->inst[0].dim;
  std::vector<int> gstart(1, 0);
  if (ctx->ens_window_mb > 0) {
    const double win = ctx->ens_window_mb * 1048576.0;
    double acc = 0;
    for (int i = 0; i < ninst; ++i) {
      const Instance &I = ctx->inst[i];
      const double b = 3.0 * I.S * (double)I.N * I.real_bytes;
      if (acc > 0 && acc + b > win) {
        gstart.push_back(i);
        acc = 0;
      }
      acc += b;
    }
  }
  gstart.push_back(ninst);
  const int G = (int)gstart.size() - 1;
  std::vector<int2> items;
  for (int r = 0; r < G + dim - 1; ++r)
    for (int a = 0; a < dim; ++a) {
      const int g = r - a;
      if (g < 0 || g >= G) continue;
      for (int i = gstart[g]; i < gstart[g + 1]; ++i)
        for (int b = 0; b < ctx->inst[i].plan[a].nblocks; ++b) items.push_back(make_int2((a << 24) | i, b));
    }
  if (ninst >= (1 << 24)) return fail(ctx, ETD_ERR_UNSUPPORTED, "more than 2^24 instances");
  if (ctx->ens_items && (int)items.size() != ctx->ens_nitems) {
    cudaFree(ctx->ens_items);
    ctx->ens_items = nullptr;
  }
  if (!ctx->ens_items && cudaMalloc((void **)&ctx->ens_items, sizeof(int2) * items.size()) != cudaSuccess)
    return fail(ctx, ETD_ERR_OOM, "ensemble work list");
  ctx->ens_nitems = (int)items.size();
  if (cudaMemcpy(ctx->ens_items, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(ctx, ETD_ERR_CUDA, "ensemble work list upload");
  if (!ctx->ens_queue) {
    if (cudaMalloc((void **)&ctx->ens_queue, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMalloc((void **)&ctx->ens_done, sizeof(int) * (size_t)std::max(1, dim - 1) * ninst) != cudaSuccess ||
        cudaMalloc((void **)&ctx->ens_status, sizeof(int) * ENS_STATUS_WORDS) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "ensemble counters");
    if (cudaMemset(ctx->ens_queue, 0, 2 * sizeof(unsigned)) != cudaSuccess ||
        cudaMemset(ctx->ens_done, 0, sizeof(int) * (size_t)std::max(1, dim - 1) * ninst) != cudaSuccess ||
        cudaMemset(ctx->ens_status, 0, sizeof(int) * ENS_STATUS_WORDS) != cudaSuccess)
      return fail(ctx, ETD_ERR_CUDA, "ensemble counters");
  }
  int thr = 0;
  size_t smem = 0;
  for (int a = 0; a < dim; ++a) {
    thr = std::max(thr, ctx->batch_threads[a]);
    smem = std::max(smem, ctx->batch_smem[a]);
  }
  ctx->ens_threads = (thr + 31) / 32 * 32;
  ctx->ens_smem = smem;
  int resident = 0;
  cudaError_t e;
  if (ctx->precision == ETD_FP64) e = ensemble_launch<double>(ctx, EnsArgs<double>{}, nullptr, &resident);
  else e = ensemble_launch<float>(ctx, EnsArgs<float>{}, nullptr, &resident);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ensemble step kernel occupancy");
  if (resident < 1) return fail(ctx, ETD_ERR_UNSUPPORTED, "ensemble step kernel does not fit an SM");
  ctx->ens_grid = std::min(resident, ctx->ens_nitems);
  return ETD_OK;
}

// Plan every instance's sweeps with chunk length Lax[a] on axis a, rebuild
// their line tables, let instances fill the common block size with more
// lines, and (re)build the block prefix sums of the launches.
etd_status plan_batch(etd_ctx *ctx, const int *Lax) {
  const int ninst = (int)ctx->inst.size();
  const int dim = ctx->inst[0].dim;
  const int rb = ctx->inst[0].real_bytes;
  if (ctx->ens_on && dim == 3 && Lax[1] != Lax[2])
    return fail(ctx, ETD_ERR_UNSUPPORTED, "persistent ensemble step: axes 1 and 2 share one chunk length");
  for (int i = 0; i < ninst; ++i) {
    Instance &I = ctx->inst[i];
    for (int a = 0; a < dim; ++a) {
      if (!plan_axis_ex(I, a, Lax[a], ctx->ens_on ? ctx->ens_max_threads : ETD_MAX_BLOCK_THREADS, 0, true, 1))
        return fail(ctx, ETD_ERR_UNSUPPORTED, "instance %d axis %d does not fit one block", i, a);
    }
  }
  // Blocks are as large as the largest instance needs; give every instance as
  // many lines per block as fit that size (small instances would otherwise
  // leave most of each block idle)
  const char *nofill = std::getenv("ETD_BATCH_NOFILL");
  // (persistent step: one block size for every axis)
  int Tall = 0;
  for (int a = 0; a < dim; ++a)
    for (int i = 0; i < ninst; ++i) Tall = std::max(Tall, ctx->inst[i].plan[a].nthreads);
  for (int a = 0; a < dim && !(nofill && nofill[0] == '1'); ++a) {
    int T = 0;
    for (int i = 0; i < ninst; ++i) T = std::max(T, ctx->inst[i].plan[a].nthreads);
    if (ctx->ens_on) T = Tall;
    for (int i = 0; i < ninst; ++i) {
      Instance &I = ctx->inst[i];
      AxisPlan &P = I.plan[a];
      const long long avail = (a == 0) ? P.nlines : P.st;
      int nlb = P.nlb;
      while (nlb * 2 * P.m <= T && nlb * 2 <= avail &&
             sweep_smem_bytes(P.kind, I.S, nlb * 2, P.pitch, I.real_bytes) <= 200 * 1024)
        nlb *= 2;
      if (nlb == P.nlb) continue;
      P.nlb = nlb;
      P.nthreads = nlb * P.m;
      P.smem = sweep_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes);
      if (a == 0) {
        P.nblocks = (int)((P.nlines + nlb - 1) / nlb);
      } else {
        P.nlo_blocks = (int)((P.st + nlb - 1) / nlb);
        P.nblocks = (int)((long long)P.nlo_blocks * (I.N / (P.st * I.n[a])));
      }
    }
  }
  for (int i = 0; i < ninst; ++i)
    for (int a = 0; a < dim; ++a) {
      etd_status st = build_axis_tables(ctx, ctx->inst[i], a);
      if (st != ETD_OK) return st;
    }
  for (int a = 0; a < dim; ++a) {
    std::vector<int> bs(ninst + 1, 0);
    int thr = 0;
    size_t smem = 0;
    for (int i = 0; i < ninst; ++i) {
      const AxisPlan &P = ctx->inst[i].plan[a];
      bs[i + 1] = bs[i] + P.nblocks;
      thr = std::max(thr, P.nthreads);
      smem = std::max(smem, P.smem);
    }
    ctx->batch_total_blocks[a] = bs[ninst];
    ctx->batch_threads[a] = thr;
    ctx->batch_smem[a] = smem;
    ctx->batch_L[a] = Lax[a];
    const size_t argb = (rb == 8 ? sizeof(SweepArgs<double>) : sizeof(SweepArgs<float>)) * ninst;
    if (!ctx->batch_args[a] && cudaMalloc(&ctx->batch_args[a], argb) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "ensemble launch tables");
    if (!ctx->batch_block_start[a] && cudaMalloc((void **)&ctx->batch_block_start[a], sizeof(int) * (ninst + 1)) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "ensemble launch tables");
    if (cudaMemcpy(ctx->batch_block_start[a], bs.data(), sizeof(int) * (ninst + 1), cudaMemcpyHostToDevice) !=
        cudaSuccess)
      return fail(ctx, ETD_ERR_CUDA, "ensemble launch tables upload");
  }
  if (ctx->ens_on) {
    etd_status st = plan_ensemble_step(ctx);
    if (st != ETD_OK) return st;
  }
  // arguments and captured graphs refer to the old plan: rebuild on the next run
  drop_graphs(ctx);
  ctx->batch_states.clear();
  return ETD_OK;
}

}  // namespace

extern "C" {

etd_status etd_batch_create(int32_t ninst, const etd_grid *grids, const double *D, const etd_reaction *reactions,
                            double k, int32_t precision, void *stream, etd_ctx **out) {
  if (!out) return fail(nullptr, ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (ninst < 1 || !grids || !D || !reactions) return fail(nullptr, ETD_ERR_INVALID_ARG, "empty or null ensemble");
  const int S = reactions[0].nspecies;
  for (int i = 0; i < ninst; ++i) {
    etd_status st = validate_problem(&grids[i], D + (size_t)i * S, &reactions[i], k, precision);
    if (st != ETD_OK) return st;
    if (grids[i].dim != grids[0].dim || reactions[i].nspecies != S)
      return fail(nullptr, ETD_ERR_INVALID_ARG, "instance %d: every instance needs the same dim and nspecies", i);
  }
  etd_ctx *ctx = new (std::nothrow) etd_ctx();
  if (!ctx) return fail(nullptr, ETD_ERR_OOM, "host allocation failed");
  ctx->stream = (cudaStream_t)stream;
  ctx->precision = precision;
  ctx->batched = true;
  // one persistent launch per step unless ETD_ENSEMBLE_PERSISTENT=0 (one launch per sweep kind)
  const char *pe = std::getenv("ETD_ENSEMBLE_PERSISTENT");
  ctx->ens_on = !(pe && pe[0] == '0');
  const char *ec = std::getenv("ETD_ENSEMBLE_CIRC");
  ctx->ens_circ = !(ec && ec[0] == '0');
  if (const char *w = std::getenv("ETD_ENSEMBLE_WINDOW_MB")) ctx->ens_window_mb = std::max(0.0, atof(w));
  if (const char *t = std::getenv("ETD_ENSEMBLE_THREADS")) {
    const int v = atoi(t);
    if (v == 128 || v == 256 || v == 512) ctx->ens_max_threads = v;
  }
  ctx->inst.resize(ninst);
  const int dim = grids[0].dim;
  const int rb = precision == ETD_FP64 ? 8 : 4;
  auto abort_create = [&](etd_status st) {
    std::string msg = ctx->err;
    etd_destroy(ctx);
    return fail(nullptr, st, "%s", msg.c_str());
  };
  // common chunk length per axis (kernel template parameter), per-instance tiles
  int Lax[3];
  // FP32: 16 positions per thread on every axis (measured fastest for the 64..512 ensemble)
  for (int a = 0; a < dim; ++a) Lax[a] = (rb == 4) ? 16 : (a == 0 ? 4 : 8);
  // ETD_BATCH_CHUNK="L0,L1[,L2]" forces the chunk lengths (to compare shapes)
  if (const char *f = std::getenv("ETD_BATCH_CHUNK")) {
    int v[3] = {0, 0, 0};
    if (sscanf(f, "%d,%d,%d", &v[0], &v[1], &v[2]) >= dim)
      for (int a = 0; a < dim; ++a)
        if (v[a] == 4 || v[a] == 8 || v[a] == 16) Lax[a] = v[a];
  }
  size_t scratch_elems = 0;
  for (int i = 0; i < ninst; ++i) {
    Instance &I = ctx->inst[i];
    etd_status st = init_instance(ctx, I, &grids[i], D + (size_t)i * S, &reactions[i], k, precision, false);
    if (st != ETD_OK) return abort_create(st);
    scratch_elems += (size_t)3 * I.S * I.N;
  }
  if (cudaMalloc(&ctx->batch_scratch, scratch_elems * rb) != cudaSuccess) {
    fail(ctx, ETD_ERR_OOM, "ensemble scratch of %zu bytes", scratch_elems * rb);
    return abort_create(ETD_ERR_OOM);
  }
  size_t off = 0;
  for (Instance &I : ctx->inst) {
    const size_t F = (size_t)I.S * I.N;
    for (int f = 0; f < 3; ++f) I.scratch[f] = (unsigned char *)ctx->batch_scratch + (off + f * F) * rb;
    off += 3 * F;
  }
  etd_status st = plan_batch(ctx, Lax);
  if (st != ETD_OK) return abort_create(st);
  *out = ctx;
  return ETD_OK;
}

etd_status etd_batch_run(etd_ctx *ctx, void *const *U, double t0, int64_t nsteps) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_batch_run on a single-problem context");
  if (!U) return fail(ctx, ETD_ERR_INVALID_ARG, "U is NULL");
  if (nsteps < 0 || !std::isfinite(t0)) return fail(ctx, ETD_ERR_INVALID_ARG, "bad nsteps or t0");
  const int ninst = (int)ctx->inst.size();
  for (int i = 0; i < ninst; ++i)
    if (!U[i]) return fail(ctx, ETD_ERR_INVALID_ARG, "U[%d] is NULL", i);
  std::vector<void *> now(U, U + ninst);
  if (now != ctx->batch_states) {
    // the device arguments hold the state pointers: rebuild them, drop graphs built on the old ones
    etd_status st = ctx->precision == ETD_FP64 ? upload_batch_args<double>(ctx, U) : upload_batch_args<float>(ctx, U);
    if (st != ETD_OK) return st;
    ctx->batch_states = now;
    drop_graphs(ctx);
  }
  const Instance &I0 = ctx->inst[0];
  const double k = I0.k;
  if (ctx->ens_on) {
    auto enqueue_ens = [&](cudaStream_t s, int64_t n) -> cudaError_t {
      const double t = t0 + (double)n * k;
      auto fill = [&](auto &E) {
        using R = std::remove_reference_t<decltype(E.exp_mt[0])>;
        for (int a = 0; a < 3; ++a) {
          E.args[a] = a < I0.dim ? (const SweepArgs<R> *)ctx->batch_args[a] : nullptr;
          E.t_eval[a] = a == I0.dim - 1 ? t + k : t;
          E.exp_mt[a] = (R)std::exp(-E.t_eval[a]);
        }
        E.items = ctx->ens_items;
        E.nitems = ctx->ens_nitems;
        E.ninst = ninst;
        E.queue = ctx->ens_queue;
        E.done = ctx->ens_done;
        E.status = ctx->ens_status;
        E.wait_ns = (long long)(ctx->ens_wait_s * 1e9);
      };
      if (ctx->precision == ETD_FP64) {
        EnsArgs<double> E{};
        fill(E);
        return ensemble_launch<double>(ctx, E, s, nullptr);
      }
      EnsArgs<float> E{};
      fill(E);
      return ensemble_launch<float>(ctx, E, s, nullptr);
    };
    etd_status st = run_steps(ctx, enqueue_ens, GraphKey{ctx->batch_states.data(), nullptr, t0, nsteps}, nsteps);
    if (st != ETD_OK) return st;
    // the waits' status: ETD_ERR_TIMEOUT if one gave up (the steps after it are skipped)
    int status[ENS_STATUS_WORDS] = {0, 0, 0, 0};
    cudaError_t e = cudaMemcpyAsync(status, ctx->ens_status, sizeof(status), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ensemble step status");
    if (status[0]) {
      cudaMemsetAsync(ctx->ens_status, 0, sizeof(int) * ENS_STATUS_WORDS, ctx->stream);
      cudaStreamSynchronize(ctx->stream);
      return fail(ctx, ETD_ERR_TIMEOUT,
                  "ensemble step: the wait of instance %d axis %d for sweep %d gave up after %g s; the run is "
                  "incomplete",
                  status[1], status[2], status[2] - 1, ctx->ens_wait_s);
    }
    return ETD_OK;
  }
  auto enqueue = [&](cudaStream_t s, int64_t n) -> cudaError_t {
    const double t = t0 + (double)n * k;
    for (int a = 0; a < I0.dim; ++a) {
      const int kind = I0.plan[a].kind;
      const double te = kind == SWEEP_LAST ? t + k : t;
      cudaError_t e;
      if (ctx->precision == ETD_FP64)
        e = launch_sweep_batched((const SweepArgs<double> *)ctx->batch_args[a], ctx->batch_block_start[a], ninst,
                                 ctx->batch_total_blocks[a], I0.S, ctx->batch_L[a], kind, ctx->batch_threads[a],
                                 ctx->batch_smem[a], s, te);
      else
        e = launch_sweep_batched((const SweepArgs<float> *)ctx->batch_args[a], ctx->batch_block_start[a], ninst,
                                 ctx->batch_total_blocks[a], I0.S, ctx->batch_L[a], kind, ctx->batch_threads[a],
                                 ctx->batch_smem[a], s, te);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  };
  return run_steps(ctx, enqueue, GraphKey{ctx->batch_states.data(), nullptr, t0, nsteps}, nsteps);
}

etd_status etd_batch_autotune(etd_ctx *ctx, void *const *U_work) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_batch_autotune on a single-problem context");
  if (!U_work) return fail(ctx, ETD_ERR_INVALID_ARG, "U_work is NULL");
  const int ninst = (int)ctx->inst.size();
  for (int i = 0; i < ninst; ++i)
    if (!U_work[i]) return fail(ctx, ETD_ERR_INVALID_ARG, "U_work[%d] is NULL", i);
  const int dim = ctx->inst[0].dim;
  const bool fp32 = ctx->precision != ETD_FP64;
  const int choices[2] = {fp32 ? 8 : 4, fp32 ? 16 : 8};
  int keep[3] = {ctx->batch_L[0], ctx->batch_L[1], ctx->batch_L[2]};
  int best[3] = {keep[0], keep[1], keep[2]};
  double best_ms = 1e30;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(ctx, ETD_ERR_CUDA, "autotune events");
  etd_status st = ETD_OK;
  for (int c = 0; c < (1 << dim) && st == ETD_OK; ++c) {
    int Lax[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) Lax[a] = choices[(c >> a) & 1];
    if (ctx->ens_on && dim == 3 && Lax[1] != Lax[2]) continue;  // one chunk length on axes 1 and 2
    if (plan_batch(ctx, Lax) != ETD_OK) continue;  // this shape does not fit every instance
    st = etd_batch_run(ctx, U_work, 0.0, 2);       // warm-up (arguments, graph)
    if (st != ETD_OK) break;
    cudaEventRecord(e0, ctx->stream);
    st = etd_batch_run(ctx, U_work, 0.0, 2);
    cudaEventRecord(e1, ctx->stream);
    if (st != ETD_OK || cudaEventSynchronize(e1) != cudaSuccess) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (std::getenv("ETD_TUNE_VERBOSE"))
      fprintf(stderr, "etd_batch_autotune L = %d,%d,%d -> %.4f ms/step\n", Lax[0], Lax[1], Lax[2], ms / 2);
    if (ms < best_ms) {
      best_ms = ms;
      for (int a = 0; a < 3; ++a) best[a] = Lax[a];
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != ETD_OK) return st;
  return plan_batch(ctx, best_ms < 1e30 ? best : keep);
}

etd_status etd_batch_set_wait_limit(etd_ctx *ctx, double seconds) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_batch_set_wait_limit on a single-problem context");
  if (!(seconds > 0.0) || !(seconds <= 60.0))
    return fail(ctx, ETD_ERR_INVALID_ARG, "wait limit %g s outside (0, 60]", seconds);
  ctx->ens_wait_s = seconds;
  drop_graphs(ctx);  // the limit is a launch argument of the captured steps
  return ETD_OK;
}

etd_status etd_batch_debug_hold(etd_ctx *ctx, int32_t instance, int32_t axis) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (!ctx->batched || !ctx->ens_on)
    return fail(ctx, ETD_ERR_INVALID_ARG, "etd_batch_debug_hold needs a batched context with the persistent step");
  const int ninst = (int)ctx->inst.size();
  const int dim = ctx->inst[0].dim;
  if (instance < 0 || instance >= ninst || axis < 0 || axis > dim - 2)
    return fail(ctx, ETD_ERR_INVALID_ARG, "instance %d axis %d out of range", instance, axis);
  // a counter this far below zero cannot reach its target (the blocks of one sweep) in a launch
  const int seed = -(1 << 30);
  cudaError_t e = cudaMemcpyAsync(ctx->ens_done + (size_t)axis * ninst + instance, &seed, sizeof(int),
                                  cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);  // host value must outlive the copy
  if (e != cudaSuccess) return cuda_fail(ctx, e, "ensemble counter seed");
  return ETD_OK;
}

}  // extern "C"
