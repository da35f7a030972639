// etd_grad.cu -- reverse mode: one adjoint step (etd_step_adjoint) and the
// checkpointed gradient of a final-state misfit (etd_grad).
//
// Adjoint of one step n: recompute the forward sweeps' intermediates of step
// n from U_n (axis-0 outputs; in 3D also the axis-1 outputs, kept out of
// place), then run the adjoint sweeps in reverse axis order (last, middle,
// first).  etd_grad stores U every ckpt steps on the forward pass; in the
// reverse pass each segment is recomputed from its checkpoint and walked
// backwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <type_traits>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_context.h"
#include "etd_internal.h"
#include "etd_tables.h"
#include "etd_circ.h"

namespace etd {
bool plan_axis(Instance &I, int a, int L, int max_threads);
}

using namespace etd;

namespace {

int pow2_floor_i(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}

bool plan_adjoint_axis(Instance &I, int a, int L, int nlb_force = 0) {
  AxisPlan &P = I.aplan[a];
  const long long n = I.n[a];
  P.L = L;
  P.m = (int)((n + L - 1) / L);
  if (P.m > ETD_MAX_BLOCK_THREADS) return false;
  P.kind = (a == 0) ? ADJ_FIRST : (a == I.dim - 1 ? ADJ_LAST : ADJ_MIDDLE);
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  P.st = st;
  P.nlines = I.N / n;
  P.pitch = exchange_pitch(P.m);
  const long long avail = (a == 0) ? P.nlines : st;
  // ETD_ADJ_THREADS=256|128 caps the block (more resident blocks per SM, same 128 registers)
  int maxt = ETD_MAX_BLOCK_THREADS;
  if (const char *t = std::getenv("ETD_ADJ_THREADS")) {
    const int v = atoi(t);
    if ((v == 128 || v == 256) && P.m <= v) maxt = v;
  }
  int nlb = pow2_floor_i(std::min<long long>(32, maxt / P.m));
  if (nlb_force > 0 && nlb_force <= nlb) nlb = nlb_force;
  while (nlb > 1 && nlb / 2 >= avail) nlb /= 2;
  while (nlb > 1 && adjoint_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes) > 200 * 1024) nlb /= 2;
  P.nlb = nlb;
  P.nthreads = nlb * P.m;
  P.smem = adjoint_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes);
  if (a == 0) {
    P.nlo_blocks = 1;
    P.nblocks = (int)((P.nlines + nlb - 1) / nlb);
  } else {
    P.nlo_blocks = (int)((st + nlb - 1) / nlb);
    P.nblocks = (int)(P.nlo_blocks * (I.N / (st * n)));
  }
  P.sp = StagePlan{};
  return P.smem <= 200 * 1024;
}

template <typename R>
void upload(DeviceArena &arena, const HostTab &T, MatTab<R> &M, cudaError_t &err) {
  std::vector<R> pos(T.pos.begin(), T.pos.end()), sum(T.sum.begin(), T.sum.end()), ch(T.chunk.begin(), T.chunk.end());
  M.pos = (const typename V4T<R>::T *)arena.put(pos.data(), pos.size() * sizeof(R), err);
  M.sum = (const typename V2T<R>::T *)arena.put(sum.data(), sum.size() * sizeof(R), err);
  M.chunk = (const typename V4T<R>::T *)arena.put(ch.data(), ch.size() * sizeof(R), err);
  std::vector<R> e1(T.e1.begin(), T.e1.end()), v1(T.v1.begin(), T.v1.end()), w1(T.w1.begin(), T.w1.end()),
      z1(T.z1.begin(), T.z1.end());
  M.e1 = (const R *)arena.put(e1.data(), e1.size() * sizeof(R), err);
  M.v1 = (const R *)arena.put(v1.data(), v1.size() * sizeof(R), err);
  M.w1 = (const R *)arena.put(w1.data(), w1.size() * sizeof(R), err);
  M.z1 = (const R *)arena.put(z1.data(), z1.size() * sizeof(R), err);
  M.rows1 = nullptr;
  M.rows2 = nullptr;  // adjoint sweeps run one line per thread
  M.segc = nullptr;
  if constexpr (sizeof(R) == 4) {
    const std::vector<float> r1 = fp32_rows(T);
    M.rows1 = (const float *)arena.put(r1.data(), r1.size() * sizeof(float), err);
  }
  M.r = T.r;
  M.sm_c = T.sm_c;
  M.sm_inv = T.sm_inv;
}

etd_status prepare_adjoint(etd_ctx *ctx, Instance &I) {
  if (!I.adj_ready) {
    static const double gammas[3] = {1.0, 3.0, 4.0};
    // ETD_ADJ_TILES="L:nlb,..." (one entry per axis) forces the adjoint chunk
    // length and lines per block, e.g. to compare shapes in a profiler run
    const char *forced = std::getenv("ETD_ADJ_TILES");
    for (int a = 0; a < I.dim; ++a) {
      // FP32: 8 positions per thread (32 chunks on 256-node lines: the serial carry chain, measured
      // faster than 4 with the warp scan); FP64: 4 (register pressure)
      int L = (I.real_bytes == 4) ? 8 : 4;
      int fl = 0, fn = 0;
      if (forced) {
        const char *p = forced;
        for (int b = 0; b < a && p; ++b) {
          p = strchr(p, ',');
          if (p) ++p;
        }
        if (p && sscanf(p, "%d:%d", &fl, &fn) >= 1 && (fl == 4 || fl == 8) && plan_adjoint_axis(I, a, fl, fn)) L = fl;
      }
      if (L != fl) {
        fn = 0;
        while (!plan_adjoint_axis(I, a, L) && L < 8) L *= 2;
      }
      if (!plan_adjoint_axis(I, a, L, fn))
        return fail(ctx, ETD_ERR_UNSUPPORTED, "adjoint: axis %d with n = %lld does not fit one block", a,
                    (long long)I.n[a]);
      const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
      // periodic axes whose lines are whole chunks run the circulant adjoint
      // (ETD_ADJ_CIRC=0 keeps the tables)
      const char *ac = std::getenv("ETD_ADJ_CIRC");
      I.acirc[a] = !(ac && ac[0] == '0') && I.bc[a] == BC_PERIODIC && I.n[a] % L == 0 &&
                   L == (I.real_bytes == 4 ? 8 : 4);
      if (I.acirc[a])
        for (int s = 0; s < I.S; ++s)
          for (int g = 0; g < 3; ++g) {
            CircHost H;
            circ_coeffs((I.k / gammas[g]) * I.D[s] / (h * h), (int)I.n[a], L, H);
            auto fill = [&](auto &C) {
              using RR = std::remove_reference_t<decltype(C.lam)>;
              C.lam = (RR)H.lam;
              C.lamL = (RR)H.lamL;
              C.kap = (RR)H.kap;
              C.inv1m = (RR)H.inv1m;
              C.ialpha = (RR)(1.0 / H.alpha);
              for (int t = 0; t < 16; ++t) C.pw[t] = (RR)H.pw[t];
            };
            fill(I.acl32[a][s][g]);
            fill(I.acl64[a][s][g]);
          }
      cudaError_t err = cudaSuccess;
      for (int s = 0; s < I.S; ++s)
        for (int g = 0; g < 3; ++g)
          for (int tr = 0; tr < 2; ++tr) {
            HostTab T;
            build_tab((int)I.n[a], I.bc[a], (I.k / gammas[g]) * I.D[s] / (h * h), tr != 0, L, T);
            if (I.real_bytes == 8) upload<double>(I.arena, T, I.atab64[tr][a][s][g], err);
            else upload<float>(I.arena, T, I.atab32[tr][a][s][g], err);
            if (err != cudaSuccess) return cuda_fail(ctx, err, "adjoint tables");
          }
    }
    I.adj_ready = true;
  }
  const size_t field = (size_t)I.S * I.N * I.real_bytes;
  if (!ctx->adj_ws) {
    if (cudaMalloc(&ctx->adj_ws, 9 * field) != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "adjoint workspace");
    if (cudaMalloc(&ctx->adj_ubar[0], field) != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "adjoint workspace");
    if (cudaMalloc(&ctx->adj_ubar[1], field) != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "adjoint workspace");
    if (cudaMalloc((void **)&ctx->adj_acc, 16 * sizeof(double)) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "adjoint accumulators");
    size_t np = (size_t)loss_blocks((long long)I.S * I.N);
    for (int a = 0; a < I.dim; ++a) np = std::max(np, (size_t)I.aplan[a].nblocks * (MAX_SPECIES + 8));
    if (cudaMalloc((void **)&ctx->adj_part, np * sizeof(double)) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "adjoint partial sums");
  }
  return ETD_OK;
}

template <typename R>
void geometry(const AxisPlan &P, const Instance &I, int a, SweepArgs<R> &A) {
  memset(&A, 0, sizeof(A));
  A.N = I.N;
  A.st = P.st;
  A.nlines = P.nlines;
  A.n = (int)I.n[a];
  A.nlo_blocks = P.nlo_blocks;
  A.m = P.m;
  A.mx = P.m;  // adjoint sweeps keep whole lines in one block
  A.nseg = 1;
  A.nlb = P.nlb;
  A.pitch = P.pitch;
  A.nblocks = P.nblocks;
  A.k = I.k;
  A.kR = (R)I.k;
  A.rkind = I.rkind;
  for (int j = 0; j < 8; ++j) {
    A.rp[j] = I.rp[j];
    A.rpR[j] = (R)I.rp[j];
  }
  for (int b = 0; b < 3; ++b) A.phi[b] = (const R *)I.phi[b];
  A.nx = (int)I.n[0];
  A.ny = (int)I.n[1];
  A.src_lf = I.src_lf;
  A.src_lfR = (R)I.src_lf;
  A.axis = a;
}

// forward sweeps of step n up to (not including) the last axis: axis-0
// outputs to fa, axis-1 outputs (3D) to fb
template <typename R>
cudaError_t forward_intermediates(const Instance &I, const R *Un, double t, R *fa, R *fb, cudaStream_t s) {
  const size_t F = (size_t)I.S * I.N;
  for (int a = 0; a < I.dim - 1; ++a) {
    SweepArgs<R> A;
    fill_args<R>(I, a, 0, A);
    if (a == 0) {
      A.in[0] = Un;
    } else {
      A.in[0] = fa;
      A.in[1] = fa + F;
      A.in[2] = fa + 2 * F;
    }
    R *o = (a == 0) ? fa : fb;
    A.out[0] = o;
    A.out[1] = o + F;
    A.out[2] = o + 2 * F;
    A.t_eval = t;
    A.exp_mt = std::exp(-t);
    A.exp_mtR = (R)A.exp_mt;
    cudaError_t e = run_sweep<R>(I, a, A, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One forward step U_{n+1} = step(U_n) out of place, keeping the first
// sweep's outputs in fa and (3D) the middle sweep's in fb: the inputs of the
// step's later sweeps, which its adjoint reads.
template <typename R>
cudaError_t step_keep_t(const Instance &I, const R *Un, R *Unext, double t, R *fa, R *fb, cudaStream_t s) {
  cudaError_t e = forward_intermediates<R>(I, Un, t, fa, fb, s);
  if (e != cudaSuccess) return e;
  const size_t F = (size_t)I.S * I.N;
  const R *z = (I.dim == 3) ? fb : fa;
  const int a = I.dim - 1;
  SweepArgs<R> A;
  fill_args<R>(I, a, 0, A);
  A.in[0] = z;
  A.in[1] = z + F;
  A.in[2] = z + 2 * F;
  A.out[0] = Unext;
  A.t_eval = t + I.k;
  A.exp_mt = std::exp(-A.t_eval);
  A.exp_mtR = (R)A.exp_mt;
  return run_sweep<R>(I, a, A, s);
}

// The adjoint sweeps of step n from the kept intermediates fa, fb of U_n.
template <typename R>
cudaError_t adjoint_sweeps_t(etd_ctx *ctx, const Instance &I, const R *Un, double t, const R *ubar_next, R *ubar_out,
                             const R *fa, const R *fb) {
  cudaStream_t s = ctx->stream;
  const size_t F = (size_t)I.S * I.N;
  R *cb = (R *)ctx->adj_ws + 6 * F;
  cudaError_t e = cudaSuccess;
  const R *z = (I.dim == 3) ? fb : fa;  // inputs of the last forward sweep
  for (int a = I.dim - 1; a >= 0; --a) {
    const AxisPlan &P = I.aplan[a];
    SweepArgs<R> A;
    geometry<R>(P, I, a, A);
    for (int sp = 0; sp < I.S; ++sp) {
      for (int g = 0; g < 3; ++g) {
        if constexpr (sizeof(R) == 8) {
          A.mat[sp][g] = I.atab64[0][a][sp][g];
          A.matT[sp][g] = I.atab64[1][a][sp][g];
        } else {
          A.mat[sp][g] = I.atab32[0][a][sp][g];
          A.matT[sp][g] = I.atab32[1][a][sp][g];
        }
      }
      A.invD[sp] = 1.0 / I.D[sp];
      for (int g = 0; g < 3; ++g) {
        if constexpr (sizeof(R) == 8) A.cl[sp][g] = I.acl64[a][sp][g];
        else A.cl[sp][g] = I.acl32[a][sp][g];
      }
    }
    A.circ_adj = I.acirc[a] ? 1 : 0;
    A.acc = ctx->adj_acc;
    A.part = ctx->adj_part;
    if (P.kind == ADJ_LAST) {
      A.in[0] = ubar_next;
      A.fin[0] = z;
      A.fin[1] = z + F;
      A.fin[2] = z + 2 * F;
      A.t_eval = t + I.k;
    } else {
      A.in[0] = cb;
      A.in[1] = cb + F;
      A.in[2] = cb + 2 * F;
      A.t_eval = t;
      if (P.kind == ADJ_MIDDLE) {
        A.fin[0] = fa;
        A.fin[1] = fa + F;
        A.fin[2] = fa + 2 * F;
      } else {
        A.fin[0] = Un;
      }
    }
    if (P.kind == ADJ_FIRST) {
      A.out[0] = ubar_out;
    } else {
      A.out[0] = cb;
      A.out[1] = cb + F;
      A.out[2] = cb + 2 * F;
    }
    A.exp_mt = std::exp(-A.t_eval);
    A.exp_mtR = (R)A.exp_mt;
    e = launch_adjoint(A, I.S, P.L, P.kind, P.nthreads, P.smem, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t adjoint_step_t(etd_ctx *ctx, const Instance &I, const R *Un, double t, const R *ubar_next, R *ubar_out) {
  const size_t F = (size_t)I.S * I.N;
  R *ws = (R *)ctx->adj_ws;
  R *fa = ws, *fb = ws + 3 * F;
  cudaError_t e = forward_intermediates<R>(I, Un, t, fa, fb, ctx->stream);
  if (e != cudaSuccess) return e;
  return adjoint_sweeps_t<R>(ctx, I, Un, t, ubar_next, ubar_out, fa, fb);
}

cudaError_t step_keep(const Instance &I, const void *Un, void *Unext, double t, void *fa, void *fb, cudaStream_t s) {
  if (I.real_bytes == 8)
    return step_keep_t<double>(I, (const double *)Un, (double *)Unext, t, (double *)fa, (double *)fb, s);
  return step_keep_t<float>(I, (const float *)Un, (float *)Unext, t, (float *)fa, (float *)fb, s);
}
cudaError_t keep_intermediates(const Instance &I, const void *Un, double t, void *fa, void *fb, cudaStream_t s) {
  if (I.real_bytes == 8) return forward_intermediates<double>(I, (const double *)Un, t, (double *)fa, (double *)fb, s);
  return forward_intermediates<float>(I, (const float *)Un, t, (float *)fa, (float *)fb, s);
}
cudaError_t adjoint_sweeps(etd_ctx *ctx, const Instance &I, const void *Un, double t, const void *ub_next,
                           void *ub_out, const void *fa, const void *fb) {
  if (I.real_bytes == 8)
    return adjoint_sweeps_t<double>(ctx, I, (const double *)Un, t, (const double *)ub_next, (double *)ub_out,
                                    (const double *)fa, (const double *)fb);
  return adjoint_sweeps_t<float>(ctx, I, (const float *)Un, t, (const float *)ub_next, (float *)ub_out,
                                 (const float *)fa, (const float *)fb);
}
cudaError_t adjoint_step(etd_ctx *ctx, const Instance &I, const void *Un, double t, const void *ub_next, void *ub_out) {
  if (I.real_bytes == 8)
    return adjoint_step_t<double>(ctx, I, (const double *)Un, t, (const double *)ub_next, (double *)ub_out);
  return adjoint_step_t<float>(ctx, I, (const float *)Un, t, (const float *)ub_next, (float *)ub_out);
}

etd_status check_grad_ctx(etd_ctx *ctx) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "gradients of batched contexts are not supported");
  const Instance &I = ctx->inst[0];
  if (I.coupled) return fail(ctx, ETD_ERR_UNSUPPORTED, "gradients of coupled (complex-diffusion) contexts are not built");
  for (int s = 0; s < I.S; ++s)
    if (!(I.D[s] > 0))
      return fail(ctx, ETD_ERR_UNSUPPORTED, "the adjoint needs D_s > 0 (D[%d] = %g): dL/dD is formed as "
                                            "<lambda, b - x> / D_s", s, I.D[s]);
  return ETD_OK;
}

}  // namespace

extern "C" {

etd_status etd_step_adjoint(etd_ctx *ctx, const void *Un, double t_n, const void *Ubar_next, void *Ubar_n,
                            double *dD, double *dparams) {
  etd_status st = check_grad_ctx(ctx);
  if (st != ETD_OK) return st;
  if (!Un || !Ubar_next || !Ubar_n) return fail(ctx, ETD_ERR_INVALID_ARG, "null state pointer");
  if (!std::isfinite(t_n)) return fail(ctx, ETD_ERR_INVALID_ARG, "t_n not finite");
  Instance &I = ctx->inst[0];
  st = prepare_adjoint(ctx, I);
  if (st != ETD_OK) return st;
  cudaError_t e = cudaMemsetAsync(ctx->adj_acc, 0, 16 * sizeof(double), ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "accumulator reset");
  e = adjoint_step(ctx, I, Un, t_n, Ubar_next, Ubar_n);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint step launch");
  double acc[16];
  e = cudaMemcpyAsync(acc, ctx->adj_acc, sizeof(acc), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint accumulators");
  if (dD)
    for (int s = 0; s < I.S; ++s) dD[s] += acc[s];
  if (dparams)
    for (int j = 0; j < 8; ++j) dparams[j] += acc[MAX_SPECIES + j];
  return ETD_OK;
}

}  // extern "C"

namespace {

// forward pass with checkpoints, then either the misfit (target != NULL) or a
// given cotangent ubarN of U_N, then the reverse pass
etd_status grad_core(etd_ctx *ctx, const void *U0, double t0, const void *target, const void *ubarN, int64_t nsteps,
                     int64_t ckpt_every, double *loss, void *dU0, double *dD, double *dparams) {
  etd_status st = check_grad_ctx(ctx);
  if (st != ETD_OK) return st;
  if (!U0 || !dU0 || (!target && !ubarN)) return fail(ctx, ETD_ERR_INVALID_ARG, "null argument");
  if (target && !loss) return fail(ctx, ETD_ERR_INVALID_ARG, "loss is NULL");
  if (nsteps < 0 || ckpt_every < 1) return fail(ctx, ETD_ERR_INVALID_ARG, "nsteps < 0 or ckpt_every < 1");
  if (!std::isfinite(t0)) return fail(ctx, ETD_ERR_INVALID_ARG, "t0 not finite");
  Instance &I = ctx->inst[0];
  st = prepare_adjoint(ctx, I);
  if (st != ETD_OK) return st;
  cudaStream_t s = ctx->stream;
  const size_t bytes = (size_t)I.S * I.N * I.real_bytes;
  const int64_t nseg = nsteps == 0 ? 1 : (nsteps + ckpt_every - 1) / ckpt_every;
  const int64_t seglen = std::min<int64_t>(ckpt_every, std::max<int64_t>(nsteps, 1));
  if (ctx->ckpt_states < (size_t)nseg) {
    if (ctx->ckpt) cudaFree(ctx->ckpt);
    ctx->ckpt = nullptr;
    ctx->ckpt_states = 0;
    if (cudaMalloc(&ctx->ckpt, bytes * nseg) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "checkpoint storage (%lld states)", (long long)nseg);
    ctx->ckpt_states = nseg;
  }
  if (ctx->seg_states < (size_t)(seglen + 1)) {
    if (ctx->seg) cudaFree(ctx->seg);
    ctx->seg = nullptr;
    ctx->seg_states = 0;
    if (cudaMalloc(&ctx->seg, bytes * (seglen + 1)) != cudaSuccess)
      return fail(ctx, ETD_ERR_OOM, "segment storage (%lld states)", (long long)seglen + 1);
    ctx->seg_states = seglen + 1;
  }
  unsigned char *ck = (unsigned char *)ctx->ckpt, *sg = (unsigned char *)ctx->seg;
  unsigned char *run = sg + bytes * seglen;  // running state of the forward pass
  cudaError_t e = cudaMemsetAsync(ctx->adj_acc, 0, 16 * sizeof(double), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(run, U0, bytes, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "grad setup");
  // Intermediates kept during the segment recompute (the first sweep's outputs
  // and, in 3D, the middle sweep's of every step of the segment), when they
  // fit in device memory: the reverse steps then read them instead of running
  // those sweeps again.  ETD_GRAD_KEEP=0 recomputes them (less memory).
  const size_t mid_bytes = bytes * 3 * (size_t)(I.dim - 1);
  const char *kv = std::getenv("ETD_GRAD_KEEP");
  bool keep = !(kv && kv[0] == '0');
  if (keep && ctx->seg_mid_steps < (size_t)seglen) {
    if (ctx->seg_mid) cudaFree(ctx->seg_mid);
    ctx->seg_mid = nullptr;
    ctx->seg_mid_steps = 0;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) == cudaSuccess && mid_bytes * seglen + ((size_t)1 << 30) <= fr &&
        cudaMalloc(&ctx->seg_mid, mid_bytes * seglen) == cudaSuccess)
      ctx->seg_mid_steps = seglen;
    else
      cudaGetLastError();
  }
  keep = keep && ctx->seg_mid_steps >= (size_t)seglen;
  unsigned char *mid = (unsigned char *)ctx->seg_mid;
  // forward pass with checkpoints (U_{g ckpt} for every segment g); the last
  // segment keeps its states and intermediates right away, so the reverse
  // pass does not recompute it
  for (int64_t g = 0; g < nseg; ++g) {
    e = cudaMemcpyAsync(ck + bytes * g, run, bytes, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "checkpoint copy");
    const int64_t s0 = g * ckpt_every, len = std::min<int64_t>(ckpt_every, nsteps - s0);
    if (keep && g == nseg - 1) {
      e = cudaMemcpyAsync(sg, run, bytes, cudaMemcpyDeviceToDevice, s);
      for (int64_t i = 0; i < len && e == cudaSuccess; ++i) {
        unsigned char *fa = mid + mid_bytes * i, *fb = fa + 3 * bytes;
        e = step_keep(I, sg + bytes * i, i + 1 < len ? sg + bytes * (i + 1) : run, t0 + (double)(s0 + i) * I.k, fa,
                      fb, s);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "forward step");
      continue;
    }
    for (int64_t i = 0; i < len; ++i) {
      e = forward_step(I, run, t0 + (double)(s0 + i) * I.k, s, nullptr);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "forward step");
    }
  }
  // cotangent of U_N: misfit gradient U_N - target, or the caller's
  void *ub = ctx->adj_ubar[0], *ub2 = ctx->adj_ubar[1];
  if (target) {
    if (I.real_bytes == 8)
      e = launch_loss((const double *)run, (const double *)target, (double *)ub, (long long)I.S * I.N,
                      ctx->adj_acc + 10, ctx->adj_part, s);
    else
      e = launch_loss((const float *)run, (const float *)target, (float *)ub, (long long)I.S * I.N,
                      ctx->adj_acc + 10, ctx->adj_part, s);
  } else {
    e = cudaMemcpyAsync(ub, ubarN, bytes, cudaMemcpyDeviceToDevice, s);
  }
  if (e != cudaSuccess) return cuda_fail(ctx, e, "final cotangent");
  // reverse pass, segment by segment: recompute the segment's states from its
  // checkpoint, then walk its steps backwards
  for (int64_t g = nseg - 1; g >= 0 && nsteps > 0; --g) {
    const int64_t s0 = g * ckpt_every, len = std::min<int64_t>(ckpt_every, nsteps - s0);
    e = cudaSuccess;
    if (keep && g == nseg - 1) {
      // kept by the forward pass
    } else if (keep) {
      e = cudaMemcpyAsync(sg, ck + bytes * g, bytes, cudaMemcpyDeviceToDevice, s);
      for (int64_t i = 0; i < len && e == cudaSuccess; ++i) {
        unsigned char *fa = mid + mid_bytes * i, *fb = fa + 3 * bytes;
        const double ti = t0 + (double)(s0 + i) * I.k;
        if (i + 1 < len) e = step_keep(I, sg + bytes * i, sg + bytes * (i + 1), ti, fa, fb, s);
        else e = keep_intermediates(I, sg + bytes * i, ti, fa, fb, s);
      }
    } else {
      e = cudaMemcpyAsync(sg, ck + bytes * g, bytes, cudaMemcpyDeviceToDevice, s);
      for (int64_t i = 1; i < len && e == cudaSuccess; ++i) {
        e = cudaMemcpyAsync(sg + bytes * i, sg + bytes * (i - 1), bytes, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = forward_step(I, sg + bytes * i, t0 + (double)(s0 + i - 1) * I.k, s, nullptr);
      }
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "segment recompute");
    for (int64_t i = len - 1; i >= 0; --i) {
      const double ti = t0 + (double)(s0 + i) * I.k;
      if (keep) {
        unsigned char *fa = mid + mid_bytes * i, *fb = fa + 3 * bytes;
        e = adjoint_sweeps(ctx, I, sg + bytes * i, ti, ub, ub2, fa, fb);
      } else {
        e = adjoint_step(ctx, I, sg + bytes * i, ti, ub, ub2);
      }
      if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint step");
      std::swap(ub, ub2);
    }
  }
  e = cudaMemcpyAsync(dU0, ub, bytes, cudaMemcpyDeviceToDevice, s);
  double acc[16];
  if (e == cudaSuccess) e = cudaMemcpyAsync(acc, ctx->adj_acc, sizeof(acc), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "gradient read-back");
  if (loss) *loss = target ? acc[10] : 0.0;
  if (dD)
    for (int sp = 0; sp < I.S; ++sp) dD[sp] = acc[sp];
  if (dparams)
    for (int j = 0; j < 8; ++j) dparams[j] = acc[MAX_SPECIES + j];
  return ETD_OK;
}

}  // namespace

extern "C" {

etd_status etd_grad(etd_ctx *ctx, const void *U0, double t0, const void *target, int64_t nsteps, int64_t ckpt_every,
                    double *loss, void *dU0, double *dD, double *dparams) {
  if (!target) return fail(ctx, ETD_ERR_INVALID_ARG, "target is NULL");
  return grad_core(ctx, U0, t0, target, nullptr, nsteps, ckpt_every, loss, dU0, dD, dparams);
}

etd_status etd_run_vjp(etd_ctx *ctx, const void *U0, double t0, int64_t nsteps, int64_t ckpt_every,
                       const void *Ubar_N, void *dU0, double *dD, double *dparams) {
  if (!Ubar_N) return fail(ctx, ETD_ERR_INVALID_ARG, "Ubar_N is NULL");
  return grad_core(ctx, U0, t0, nullptr, Ubar_N, nsteps, ckpt_every, nullptr, dU0, dD, dparams);
}

}  // extern "C"
