// etd_circ.cuh -- circulant sweeps of periodic axes (sm_103a): the first-axis
// (contiguous) sweep with lanes along the line.
//
// A block holds `lpb` whole lines of m chunks (p = m L); thread j of a line
// owns chunk j.  The chunk is staged in shared memory with cp.async (the
// thread's private slot), so the passes keep only running values in
// registers.  Every solve runs as (see etd_circ.h for the algebra):
//   pass 1: zero-carry chunk summaries F_j, W_j (two FMAs per position, the
//           weights lambda^t are kernel-parameter constants);
//   exchange 1: an inclusive scan of F over the chunks of the line with the
//           constant multiplier Lambda (lane shuffles; lines of several warps
//           add one shared-memory step over the warp totals), closed
//           cyclically by the line total -> carry Yc_j of every chunk;
//   exchange 2: the same suffix scan of G_j = W_j + kappa Yc_j -> carry Zc_j;
//   pass 2: the recurrences y_i = b_i + lambda y_{i-1} and
//           z_i = y_i + lambda z_{i+1} over the chunk from (Yc_j, Zc_j).
// All 5 s solves of the sweep (T, S on U_n; T, S on F(U_n); P on
// U_n + k F(U_n)) share the two rounds; results leave as 32-byte stores.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "etd_circ.h"

namespace etd {

// non-zero after a kernel's bounded wait gave up (1: a tile copy, 2: an
// exchange); one per translation unit that compiles these kernels, read and
// cleared through take_status_here()
static __device__ int g_circ_status;

static inline int take_status_here() {
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

namespace circ {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rdivc(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdivc(double a, double b) { return a / b; }

// F(u) of the autonomous reactions (Section 8's models; periodic problems
// carry no manufactured source).  K: the reaction kind (etd_reaction_kind).
template <typename R, int S, int K>
__device__ __forceinline__ void reaction_kind(const CircArgs<R> &A, const R (&u)[S], R (&f)[S]) {
  if constexpr (K == 1) {
#pragma unroll
    for (int s = 0; s < S; ++s) f[s] = fma(A.rpR[0], u[s], A.rpR[1]);
    return;
  } else if constexpr (K == 2 && S == 2) {  // Brusselator: a + u^2 v - (b+1) u ; b u - u^2 v
    const R uuv = u[0] * u[0] * u[1];
    f[0] = A.rpR[0] + uuv - (A.rpR[1] + R(1)) * u[0];
    f[1] = A.rpR[1] * u[0] - uuv;
    return;
  } else if constexpr (K == 3 && S == 2) {  // Schnakenberg: g (a - u + u^2 v) ; g (b - u^2 v)
    const R uuv = u[0] * u[0] * u[1];
    f[0] = A.rpR[2] * (A.rpR[0] - u[0] + uuv);
    f[1] = A.rpR[2] * (A.rpR[1] - uuv);
    return;
  } else if constexpr (K == 4 && S == 2) {  // Gray-Scott: -u v^2 + F (1-u) ; u v^2 - (F+kappa) v
    const R uvv = u[0] * u[1] * u[1];
    f[0] = A.rpR[0] * (R(1) - u[0]) - uvv;
    f[1] = uvv - (A.rpR[0] + A.rpR[1]) * u[1];
    return;
  } else if constexpr (K == 6 && S == 2) {  // CGL (alpha = 0): u - (1 + i beta) u |u|^2, u = u0 + i u1
    const R beta = A.rpR[0], r = fma(u[0], u[0], u[1] * u[1]);
    f[0] = fma(-r, fma(-beta, u[1], u[0]), u[0]);
    f[1] = fma(-r, fma(beta, u[0], u[1]), u[1]);
    return;
  } else if constexpr (K == 5) {  // enzyme kinetics without a source term
    f[0] = -rdivc(u[0], R(1) + u[0]);
#pragma unroll
    for (int s = 1; s < S; ++s) f[s] = R(0);
    return;
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s) f[s] = R(0);
  }
}
// RK >= 0: the kind fixed at compile time; RK < 0: chosen per call from A.rkind
template <typename R, int S, int RK>
__device__ __forceinline__ void reaction(const CircArgs<R> &A, const R (&u)[S], R (&f)[S]) {
  if constexpr (RK >= 0) {
    reaction_kind<R, S, RK>(A, u, f);
  } else {
    switch (A.rkind) {
      case 1: reaction_kind<R, S, 1>(A, u, f); return;
      case 2: reaction_kind<R, S, 2>(A, u, f); return;
      case 3: reaction_kind<R, S, 3>(A, u, f); return;
      case 4: reaction_kind<R, S, 4>(A, u, f); return;
      case 5: reaction_kind<R, S, 5>(A, u, f); return;
      case 6: reaction_kind<R, S, 6>(A, u, f); return;
      default: reaction_kind<R, S, 0>(A, u, f); return;
    }
  }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// 32-byte global stores (one whole sector per thread and instruction)
__device__ __forceinline__ void st32(float *p, const float *v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st32(double *p, const double *v) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
               : "memory");
}

// ---- TMA (cp.async.bulk.tensor) and mbarrier helpers
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z,
                                            unsigned long long *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
// distributed shared memory: this CTA's shared address `a` in cluster block `rank`
__device__ __forceinline__ unsigned mapa_u32(unsigned a, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// asynchronous stores into another block's shared memory, each completing its
// byte count on that block's mbarrier (no ordering with this block's other
// memory operations: nothing waits for its global stores)
__device__ __forceinline__ void st_async(unsigned ra, float v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f32 [%0], %1, [%2];\n" ::"r"(ra), "f"(v),
               "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async(unsigned ra, double v, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.f64 [%0], %1, [%2];\n" ::"r"(ra), "d"(v),
               "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async2(unsigned ra, float a, float b, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(ra),
               "f"(a), "f"(b), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async2(unsigned ra, double a, double b, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];\n" ::"r"(ra),
               "d"(a), "d"(b), "r"(rbar)
               : "memory");
}
__device__ __forceinline__ void st_async4(unsigned ra, float a, float b, float c, float d, unsigned rbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];\n" ::"r"(
                   ra),
               "f"(a), "f"(b), "f"(c), "f"(d), "r"(rbar)
               : "memory");
}

// Bounded wait for phase `parity` of an mbarrier: gives up after 0.25 s of
// %globaltimer (or 2^22 polls), or at once once an earlier wait of this block
// gave up (*fail, shared, set here), returning false; the caller records the
// failure in g_circ_status and carries on so that every block of a cluster
// still reaches the same barriers and the launch ends.
__device__ __forceinline__ unsigned long long circ_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait_t(unsigned long long *bar, unsigned parity, int *fail) {
  const unsigned a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned ok;
    if constexpr (CLUSTER)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, "
          "1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(ok)
          : "r"(a), "r"(parity)
          : "memory");
    if (ok) return true;
    if ((it & 63) == 0) {
      if (*(volatile int *)fail != 0) return false;
      const unsigned long long t = circ_globaltimer();
      if (it == 0) t0 = t;
      else if (t - t0 > 250000000ull) break;
    }
  }
  *(volatile int *)fail = 1;
  return false;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int *fail) {
  return mbar_wait_t<false>(bar, parity, fail);
}
// acquiring at cluster scope (phases completed by other blocks' st.async)
__device__ __forceinline__ bool mbar_wait_cluster(unsigned long long *bar, unsigned parity, int *fail) {
  return mbar_wait_t<true>(bar, parity, fail);
}

// solve q of species s: 0 T on U, 1 S on U, 2 T on F, 3 S on F, 4 P on U + k F
__host__ __device__ constexpr int qmat(int q) { return q == 4 ? 0 : (q & 1) ? 2 : 1; }

}  // namespace circ

// Thread j of a line: chunk j.  Block: lpb lines x m threads (max(m, 256)
// threads).  Persistent: block b takes the line groups b, b + gridDim.x, ...
// and stages the next group's chunks (cp.async into the other half of its
// double buffer) while it solves the current one.
template <typename R, int S, int L, int NT, int RK = -1>
__global__ void __launch_bounds__(NT, NT == 256 ? 3 : 1) circ_first_kernel(const __grid_constant__ CircArgs<R> A) {
  using namespace circ;
  extern __shared__ __align__(16) unsigned char circ_smem[];
  constexpr int VW = 16 / sizeof(R);   // elements per 16 bytes
  constexpr int CSZ = L;               // chunk slot (unpadded: three blocks fit an SM)
  constexpr int NQ = 5;
  const int m = A.m, tid = threadIdx.x, nthr = blockDim.x;
  const int lb = tid / m, j = tid - lb * m;
  const int lane = tid & 31;
  const int G = m < 32 ? m : 32;       // lanes of one line in a warp
  const int gl = lane & (G - 1);
  const int nw = m > 32 ? m / 32 : 1;  // warps of one line
  const int w = j >> 5;
  R *stage0 = reinterpret_cast<R *>(circ_smem);         // [2 buffers][S][nthr][CSZ]
  R *tot = stage0 + (size_t)2 * S * nthr * CSZ;         // [2][lpb][nw][S][NQ]
  const long long ngrp = (A.nlines + A.lpb - 1) / A.lpb;
  // A slot holds NGR 16-byte granules; granule g sits at position g ^ sw, so
  // the 8 lanes of a quarter warp reading granule g of their slots hit 8
  // different 4-bank groups (unswizzled, slots 64 or 32 bytes apart collide)
  constexpr int NGR = CSZ / VW;
  const int sw = NGR > 1 ? ((tid / (8 / NGR)) & (NGR - 1)) : 0;
  using V16 = std::conditional_t<sizeof(R) == 4, float4, double2>;  // 16 bytes
  // stage U_n of line group gi into buffer bi: thread-private slot per species
  auto stage = [&](long long gi, int bi) {
    const long long ln = gi * A.lpb + lb;
    if (gi < ngrp && ln < A.nlines) {
      const long long b0 = ln * (long long)A.p + (long long)j * L;
      R *dst = stage0 + (size_t)bi * S * nthr * CSZ;
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int v = 0; v < L; v += VW)
          cp_async16(dst + ((size_t)s * nthr + tid) * CSZ + ((v / VW) ^ sw) * VW, A.in[0] + s * A.N + b0 + v);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  stage(blockIdx.x, 0);
  int bi = 0;
#pragma unroll 1
  for (long long gi = blockIdx.x; gi < ngrp; gi += gridDim.x, bi ^= 1) {
  const long long line = gi * A.lpb + lb;
  const bool ok = line < A.nlines;
  stage(gi + gridDim.x, bi ^ 1);                        // prefetch the next group
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");  // this thread's chunk of the current group
  R *stage = stage0 + (size_t)bi * S * nthr * CSZ;
  const long long base = line * (long long)A.p + (long long)j * L;
  // granule g of species s in this thread's slot
  auto gran = [&](int s, int g) -> R * { return stage + ((size_t)s * nthr + tid) * CSZ + (g ^ sw) * VW; };
  // the slot of species s as L values (16-byte loads)
  auto load_slot = [&](int s, R (&v)[L]) {
#pragma unroll
    for (int g = 0; g < NGR; ++g) {
      const V16 q = *reinterpret_cast<const V16 *>(gran(s, g));
      if constexpr (VW == 4) {
        v[4 * g] = q.x; v[4 * g + 1] = q.y; v[4 * g + 2] = q.z; v[4 * g + 3] = q.w;
      } else {
        v[2 * g] = q.x; v[2 * g + 1] = q.y;
      }
    }
  };

  // ---- pass 1: zero-carry summaries of every solve
  R ty[S][NQ], tw[S][NQ];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int q = 0; q < NQ; ++q) ty[s][q] = tw[s][q] = R(0);
  R ub[S][VW];  // the current granule of every species
#pragma unroll
  for (int t = 0; t < L; ++t) {
    R u[S], f[S];
    if (t % VW == 0) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const V16 q = *reinterpret_cast<const V16 *>(gran(s, t / VW));
        if constexpr (VW == 4) {
          ub[s][0] = q.x; ub[s][1] = q.y; ub[s][2] = q.z; ub[s][3] = q.w;
        } else {
          ub[s][0] = q.x; ub[s][1] = q.y;
        }
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = ub[s][t % VW];
    reaction<R, S, RK>(A, u, f);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const R b[NQ] = {u[s], u[s], f[s], f[s], fma(A.kR, f[s], u[s])};
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        ty[s][q] = fma(M.lam, ty[s][q], b[q]);
        tw[s][q] = fma(M.pw[t], ty[s][q], tw[s][q]);
      }
    }
  }

  // ---- exchange 1: forward carries Yc_j (inclusive scan of F, cyclic closure)
  R Yc[S][NQ];
  if (G == 32) {  // whole warps per line: every step of the scan runs (no per-step test)
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = ty[s][q];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const R o = __shfl_up_sync(FULL, v, 1 << k);
          v = gl >= (1 << k) ? fma(M.sc[k], o, v) : v;
        }
        ty[s][q] = v;
      }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = ty[s][q];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int d = 1 << k;
          if (d < G) {
            const R o = __shfl_up_sync(FULL, v, d, G);
            if (gl >= d) v = fma(M.sc[k], o, v);
          }
        }
        ty[s][q] = v;  // inclusive prefix within the warp
      }
  }
  R Cw[S][NQ], Tot[S][NQ];
  if (nw > 1) {
    R *t1 = tot + ((size_t)(lb * nw + w) * S) * NQ;
    if (lane == 31)
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int q = 0; q < NQ; ++q) t1[s * NQ + q] = ty[s][q];
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = lane < nw ? tot[((size_t)(lb * nw + lane) * S + s) * NQ + q] : R(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          if ((1 << k) >= nw) break;
          const R o = __shfl_up_sync(FULL, v, 1 << k);
          if (lane >= (1 << k)) v = fma(M.sw[k], o, v);
        }
        const R prev = __shfl_sync(FULL, v, (w + 31) & 31);
        Cw[s][q] = w > 0 ? prev : R(0);
        Tot[s][q] = __shfl_sync(FULL, v, nw - 1);
      }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        Cw[s][q] = R(0);
        Tot[s][q] = __shfl_sync(FULL, ty[s][q], G - 1, G);
      }
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const CircMat<R> &M = A.mat[s][qmat(q)];
      const R *lp = A.lpow[s][qmat(q)];
      const R sf = (nw > 1) ? fma(lp[gl + 1], Cw[s][q], ty[s][q]) : ty[s][q];  // inclusive over the line
      R ex = __shfl_up_sync(FULL, sf, 1, G);
      if (gl == 0) ex = Cw[s][q];
      const R y0 = Tot[s][q] * M.inv1m;
      Yc[s][q] = fma(lp[j], y0, ex);
    }

  // ---- exchange 2: backward carries Zc_j (suffix scan of G = W + kappa Yc)
  R Zc[S][NQ];
  if (G == 32) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = fma(M.kap, Yc[s][q], tw[s][q]);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const R o = __shfl_down_sync(FULL, v, 1 << k);
          v = gl + (1 << k) < 32 ? fma(M.sc[k], o, v) : v;
        }
        tw[s][q] = v;
      }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = fma(M.kap, Yc[s][q], tw[s][q]);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const int d = 1 << k;
          if (d < G) {
            const R o = __shfl_down_sync(FULL, v, d, G);
            if (gl + d < G) v = fma(M.sc[k], o, v);
          }
        }
        tw[s][q] = v;  // inclusive suffix within the warp
      }
  }
  if (nw > 1) {
    R *t2 = tot + ((size_t)A.lpb * nw * S) * NQ + ((size_t)(lb * nw + w) * S) * NQ;
    if (lane == 0)
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll
        for (int q = 0; q < NQ; ++q) t2[s * NQ + q] = tw[s][q];
    __syncthreads();
    const R *tb = tot + ((size_t)A.lpb * nw * S) * NQ;
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const CircMat<R> &M = A.mat[s][qmat(q)];
        R v = lane < nw ? tb[((size_t)(lb * nw + lane) * S + s) * NQ + q] : R(0);
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          if ((1 << k) >= nw) break;
          const R o = __shfl_down_sync(FULL, v, 1 << k);
          if (lane + (1 << k) < nw) v = fma(M.sw[k], o, v);
        }
        const R nxt = __shfl_sync(FULL, v, (w + 1) & 31);
        Cw[s][q] = (w + 1 < nw) ? nxt : R(0);
        Tot[s][q] = __shfl_sync(FULL, v, 0);
      }
  } else {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        Cw[s][q] = R(0);
        Tot[s][q] = __shfl_sync(FULL, tw[s][q], 0, G);
      }
  }
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const CircMat<R> &M = A.mat[s][qmat(q)];
      const R *lp = A.lpow[s][qmat(q)];
      const R sb = (nw > 1) ? fma(lp[32 - gl], Cw[s][q], tw[s][q]) : tw[s][q];  // suffix over the line
      R nx = __shfl_down_sync(FULL, sb, 1, G);
      if (gl == G - 1) nx = Cw[s][q];
      const R z0 = Tot[s][q] * M.inv1m;
      Zc[s][q] = fma(lp[m - 1 - j], z0, nx);
    }

  // ---- pass 2: recurrences from the carries, combination, 32-byte stores.
  // Order: R on U_n per species; P on U_n + k F(U_n) for all species at once,
  // evaluating F once per position and leaving it in the thread's staging
  // slot in place of U_n (no later pass reads U_n); R on F per species.
  if (ok) {

    // R = 9T - 8S of right-hand side h (0: U_n, 1: F) from the slot, species s
    auto solve_R = [&](int s, int h) {
      const CircMat<R> &MT = A.mat[s][1], &MS = A.mat[s][2];
      R b[L];
      load_slot(s, b);
      R zt[L], ys[L];
      R y = Yc[s][2 * h], y2 = Yc[s][2 * h + 1];
#pragma unroll
      for (int t = 0; t < L; ++t) {
        y = fma(MT.lam, y, b[t]);
        zt[t] = y;
        y2 = fma(MS.lam, y2, b[t]);
        ys[t] = y2;
      }
      R z = Zc[s][2 * h], z2 = Zc[s][2 * h + 1];
#pragma unroll
      for (int t = L - 1; t >= 0; --t) {
        z = fma(MT.lam, z, zt[t]);
        z2 = fma(MS.lam, z2, ys[t]);
        zt[t] = fma(A.cT[s], z, -A.cS[s] * z2);
      }
      R *o = A.out[h] + s * A.N + base;
#pragma unroll
      for (int t = 0; t < L; t += 32 / (int)sizeof(R)) st32(o + t, zt + t);
    };
#pragma unroll
    for (int s = 0; s < S; ++s) solve_R(s, 0);
    {
      R zp[S][L];
      R y[S];
#pragma unroll
      for (int s = 0; s < S; ++s) y[s] = Yc[s][4];
      R ub[S][VW], fb[S][VW];
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], f[S];
        if (t % VW == 0) {
#pragma unroll
          for (int s = 0; s < S; ++s) {
            const V16 q = *reinterpret_cast<const V16 *>(gran(s, t / VW));
            if constexpr (VW == 4) {
              ub[s][0] = q.x; ub[s][1] = q.y; ub[s][2] = q.z; ub[s][3] = q.w;
            } else {
              ub[s][0] = q.x; ub[s][1] = q.y;
            }
          }
        }
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = ub[s][t % VW];
        reaction<R, S, RK>(A, u, f);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          y[s] = fma(A.mat[s][0].lam, y[s], fma(A.kR, f[s], u[s]));
          zp[s][t] = y[s];
          fb[s][t % VW] = f[s];
        }
        if (t % VW == VW - 1) {  // F replaces U_n in the slot, one granule at a time
#pragma unroll
          for (int s = 0; s < S; ++s) {
            V16 q;
            if constexpr (VW == 4) q = make_float4(fb[s][0], fb[s][1], fb[s][2], fb[s][3]);
            else q = make_double2(fb[s][0], fb[s][1]);
            *reinterpret_cast<V16 *>(gran(s, t / VW)) = q;
          }
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const CircMat<R> &MP = A.mat[s][0];
        R z = Zc[s][4];
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
          z = fma(MP.lam, z, zp[s][t]);
          zp[s][t] = A.cP[s] * z;
        }
        R *o = A.out[2] + s * A.N + base;
#pragma unroll
        for (int t = 0; t < L; t += 32 / (int)sizeof(R)) st32(o + t, zp[s] + t);
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) solve_R(s, 1);
  }  // ok
  }  // line groups
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// ===================================================== strided axes
//
// Lines along a strided axis (MIDDLE: axis 1 of a 3D grid, LAST: the last
// axis).  A block covers 32 neighbouring lines (lanes: coalesced 128-byte row
// segments) times WB chunks of L positions (warps); a line longer than WB L
// is split over cs blocks that form one thread-block cluster.  The block's
// input fields are staged in shared memory with cp.async ([row][32 lines],
// conflict-free), so the passes keep only running values in registers.
// Every group of solves (one right-hand side field each) is exchanged once:
//   chunks of the block: each thread composes the zero-carry summaries of
//     the chunks before it (forward prefix) and after it (backward composite
//     W, with the forward coupling K) from shared memory;
//   blocks of the line: the block composites are published in shared memory,
//     one cluster barrier, one warp per solve reads the cs composites through
//     distributed shared memory, closes the line cyclically and hands the
//     block's carries to its threads.
// MIDDLE: R_2 on c_U, R_2 on c_f, P_2 on w (three groups, in place).
// LAST: U* = P_d w; F(U*); f1 = 9 c_U + 2k c_f + k F*, f2 = 8 c_U + 3k/2 c_f
//       + k/2 F* (written over the staged c_U, c_f); U_{n+1} = T_d f1 - S_d f2.

namespace circ {

// Exchange of NG solves of this thread's chunk j of column c (block rank,
// cs blocks; warp w, half h of a warp that holds 32 / NC chunks):
// F[q], W[q] -> carries Yc[q] (y before the chunk), Zc[q] (z after it).
// xF, xW: [NG][max(WB, cs)][NC] (after the chunk compositions they take the
// gathered block composites); blk: [2][NG][NC] published composites;
// car: [2][NG][NC].  Loops over chunks and blocks run unrolled over the
// solves only, so each step keeps NG values in flight.
template <typename R, int WB, int NC, int NG, typename MatIdx>
__device__ __forceinline__ void strided_exchange(const CircArgs<R> &A, MatIdx mi, const R (&F)[NG], const R (&W)[NG],
                                                 R (&Yc)[NG], R (&Zc)[NG], R *xF, R *xW, R *blk, R *car,
                                                 const R *tab, int j, int c, int w, int h, int rank) {
  constexpr int HP = 32 / NC, NW = WB / HP;
  constexpr int TS = 2 * (WB + 1) + 35;  // per matrix: K_{nL}, Lambda^n (n <= WB); K, Lambda at block
                                         // multiples (b <= 16); K_{m L}
  namespace cg = cooperative_groups;
  const int cs = A.cs;
  const int XS = WB > cs ? WB : cs;  // row count of xF / xW
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    xF[(q * XS + j) * NC + c] = F[q];
    xW[(q * XS + j) * NC + c] = W[q];
  }
  __syncthreads();
  R PF[NG], Ws[NG], LM[NG];
  const R *Kq[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    LM[q] = A.mat[mi(q) / 3][mi(q) % 3].lamL;
    Kq[q] = tab + mi(q) * TS;  // K_{nL} in shared memory
    PF[q] = Ws[q] = R(0);
  }
  // chunks of the block: forward prefix before j, backward composite after j
#pragma unroll 4
  for (int i = 0; i < j; ++i)
#pragma unroll
    for (int q = 0; q < NG; ++q) PF[q] = fma(LM[q], PF[q], xF[(q * XS + i) * NC + c]);
#pragma unroll 4
  for (int i = WB - 1; i > j; --i)
#pragma unroll
    for (int q = 0; q < NG; ++q)
      Ws[q] = fma(LM[q], fma(Kq[q][WB - 1 - i], xF[(q * XS + i) * NC + c], Ws[q]), xW[(q * XS + i) * NC + c]);
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    if (j == 0) blk[(NG + q) * NC + c] = fma(LM[q], fma(Kq[q][WB - 1], F[q], Ws[q]), W[q]);
    if (j == WB - 1) blk[q * NC + c] = fma(LM[q], PF[q], F[q]);
  }
  if (cs > 1) {
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();  // composites published (and xF / xW free: every thread has read them)
    for (int b = w * HP + h; b < cs; b += NW * HP) {  // spread over the warps: block b's composites
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        xF[(q * XS + b) * NC + c] = *cl.map_shared_rank(blk + q * NC + c, b);
        xW[(q * XS + b) * NC + c] = *cl.map_shared_rank(blk + (NG + q) * NC + c, b);
      }
    }
  } else {
    __syncthreads();
    if (j == 0) {  // (w = 0, h = 0)
#pragma unroll
      for (int q = 0; q < NG; ++q) {
        xF[(q * XS) * NC + c] = blk[q * NC + c];
        xW[(q * XS) * NC + c] = blk[(NG + q) * NC + c];
      }
    }
  }
  __syncthreads();
  if (w < NG) {
    // warp q: the line's cyclic closure and this block's carries for solve q
    // (with NC = 16 both halves of the warp compute; half 0 writes)
    const int q = w;
    const int sg = mi(q);
    const CircMat<R> &M = A.mat[sg / 3][sg % 3];
    const R *tk = tab + sg * TS, *tl = tk + (WB + 1), *tkb = tl + (WB + 1), *tlb = tkb + 17;
    const R LB = tl[WB];  // Lambda^WB
    const R *gF = xF + (size_t)q * XS * NC + c, *gW = xW + (size_t)q * XS * NC + c;
    // the forward chain over blocks 0 .. cs-1 and the backward chain over
    // cs-1 .. 0 are independent: one loop runs both
    R ftot = R(0), pfb = R(0), fr = R(0), wl = R(0), wsr = R(0);
#pragma unroll 4
    for (int i = 0; i < cs; ++i) {
      const R f = gF[i * NC];
      if (i == rank) {
        pfb = ftot;
        fr = f;
      }
      ftot = fma(LB, ftot, f);
      const int b = cs - 1 - i;
      if (b == rank) wsr = wl;  // composite of the blocks after this one
      wl = fma(LB, fma(tkb[i], gF[b * NC], wl), gW[b * NC]);
    }
    const R y0 = ftot * M.inv1m;
    const R z0 = fma(tlb[17], y0, wl) * M.inv1m;  // K_{mL}
    const R ycb = fma(tlb[rank], y0, pfb);
    const R ycn = fma(LB, ycb, fr);
    const R zcb = fma(tlb[cs - 1 - rank], z0, fma(tkb[cs - 1 - rank], ycn, wsr));
    if (h == 0) {
      car[q * NC + c] = ycb;
      car[(NG + q) * NC + c] = zcb;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    const int sg = mi(q);
    const R *K = Kq[q], *lp = Kq[q] + (WB + 1);
    const R ycb = car[q * NC + c], zcb = car[(NG + q) * NC + c];
    Yc[q] = fma(lp[j], ycb, PF[q]);
    const R yn = fma(LM[q], Yc[q], F[q]);
    Zc[q] = fma(lp[WB - 1 - j], zcb, fma(K[WB - 1 - j], yn, Ws[q]));
  }
}

// Exchange number x of a line split over a cluster (cs > 1), push form.
// The block's two exchange buffers alternate: exchange x receives the cluster's
// block composites in buf[x & 1] ([F, W][cs][NC][NG]) and composes its own
// chunks in buf[(x + 1) & 1] ([F, W][NG][WB][NC]).  The block's composites
// go to every other block's receive buffer by st.async, which completes their
// bytes on that block's mbarrier xbar[x & 1]; the wait is on this block's own
// barrier and on nothing of the sender's other memory traffic (a cluster
// barrier's release would first drain the sender's outstanding global stores).
// Reuse needs no further barrier: a block pushes exchange x + 1 only after it
// received this block's exchange-x push, which this block sends after its
// last read of buf[(x + 1) & 1] for exchange x - 1 and before its composition
// in it; likewise for x + 2 into buf[x & 1].  xbar[x & 1] is re-armed for
// exchange x + 2 (ng_next2 solves) once exchange x has been read.
template <typename R, int WB, int NC, int NG, typename MatIdx>
__device__ __forceinline__ void strided_exchange_push(const CircArgs<R> &A, MatIdx mi, const R (&F)[NG],
                                                      const R (&W)[NG], R (&Yc)[NG], R (&Zc)[NG], R *buf0, R *buf1,
                                                      unsigned long long *xbar, int x, int ng_next2, R *car,
                                                      const R *tab, int j, int c, int w, int h, int rank, int tid,
                                                      int *fail) {
  static_assert(WB > 1, "the first and last chunk of a block are different threads");
  constexpr int TS = 2 * (WB + 1) + 35;
  const int cs = A.cs;
  R *rb = (x & 1) ? buf1 : buf0;
  R *xF = (x & 1) ? buf0 : buf1;
  R *xW = xF + NG * WB * NC;
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    xF[(q * WB + j) * NC + c] = F[q];
    xW[(q * WB + j) * NC + c] = W[q];
  }
  __syncthreads();
  R PF[NG], Ws[NG], LM[NG];
  const R *Kq[NG];
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    LM[q] = A.mat[mi(q) / 3][mi(q) % 3].lamL;
    Kq[q] = tab + mi(q) * TS;
    PF[q] = Ws[q] = R(0);
  }
#pragma unroll 4
  for (int i = 0; i < j; ++i)
#pragma unroll
    for (int q = 0; q < NG; ++q) PF[q] = fma(LM[q], PF[q], xF[(q * WB + i) * NC + c]);
#pragma unroll 4
  for (int i = WB - 1; i > j; --i)
#pragma unroll
    for (int q = 0; q < NG; ++q)
      Ws[q] = fma(LM[q], fma(Kq[q][WB - 1 - i], xF[(q * WB + i) * NC + c], Ws[q]), xW[(q * WB + i) * NC + c]);
  // the block's composites (last chunk: forward, first chunk: backward) to
  // slot `rank` of every block's receive buffer
  const unsigned long long *bar = xbar + (x & 1);
  if (j == WB - 1 || j == 0) {
    const int fw = (j == 0) ? 1 : 0;
    R v[NG];
#pragma unroll
    for (int q = 0; q < NG; ++q)
      v[q] = fw ? fma(LM[q], fma(Kq[q][WB - 1], F[q], Ws[q]), W[q]) : fma(LM[q], PF[q], F[q]);
    R *slot = rb + ((fw * cs + rank) * NC + c) * NG;
#pragma unroll
    for (int q = 0; q < NG; ++q) slot[q] = v[q];
    const unsigned la = smem_u32(slot), lbar = smem_u32(bar);
    for (int d = 1; d < cs; ++d) {
      int dst = rank + d;
      if (dst >= cs) dst -= cs;
      const unsigned ra = mapa_u32(la, (unsigned)dst), rbar = mapa_u32(lbar, (unsigned)dst);
      if constexpr (sizeof(R) == 4 && NG % 4 == 0) {
#pragma unroll
        for (int k = 0; k < NG; k += 4) st_async4(ra + k * 4, v[k], v[k + 1], v[k + 2], v[k + 3], rbar);
      } else if constexpr (NG % 2 == 0) {
#pragma unroll
        for (int k = 0; k < NG; k += 2) st_async2(ra + k * (unsigned)sizeof(R), v[k], v[k + 1], rbar);
      } else {
#pragma unroll
        for (int k = 0; k < NG; ++k) st_async(ra + k * (unsigned)sizeof(R), v[k], rbar);
      }
    }
  }
  __syncthreads();  // own slots written; the composition buffer is read
  if (w < NG) {
    if (!mbar_wait_cluster(xbar + (x & 1), (unsigned)((x >> 1) & 1), fail)) atomicOr(&g_circ_status, 2);
    const int q = w;
    const int sg = mi(q);
    const CircMat<R> &M = A.mat[sg / 3][sg % 3];
    const R *tk = tab + sg * TS, *tl = tk + (WB + 1), *tkb = tl + (WB + 1), *tlb = tkb + 17;
    const R LB = tl[WB];
    const R *gF = rb + (size_t)c * NG + q, *gW = rb + ((size_t)cs * NC + c) * NG + q;
    R ftot = R(0), pfb = R(0), fr = R(0), wl = R(0), wsr = R(0);
#pragma unroll 4
    for (int i = 0; i < cs; ++i) {
      const R f = gF[i * NC * NG];
      if (i == rank) {
        pfb = ftot;
        fr = f;
      }
      ftot = fma(LB, ftot, f);
      const int b = cs - 1 - i;
      if (b == rank) wsr = wl;
      wl = fma(LB, fma(tkb[i], gF[b * NC * NG], wl), gW[b * NC * NG]);
    }
    const R y0 = ftot * M.inv1m;
    const R z0 = fma(tlb[17], y0, wl) * M.inv1m;
    const R ycb = fma(tlb[rank], y0, pfb);
    const R ycn = fma(LB, ycb, fr);
    const R zcb = fma(tlb[cs - 1 - rank], z0, fma(tkb[cs - 1 - rank], ycn, wsr));
    if (h == 0) {
      car[q * NC + c] = ycb;
      car[(NG + q) * NC + c] = zcb;
    }
  }
  __syncthreads();
  if (tid == 0) mbar_expect_tx(xbar + (x & 1), (unsigned)((cs - 1) * 2 * ng_next2 * NC * (int)sizeof(R)));
#pragma unroll
  for (int q = 0; q < NG; ++q) {
    const R *K = Kq[q], *lp = Kq[q] + (WB + 1);
    const R ycb = car[q * NC + c], zcb = car[(NG + q) * NC + c];
    Yc[q] = fma(lp[j], ycb, PF[q]);
    const R yn = fma(LM[q], Yc[q], F[q]);
    Zc[q] = fma(lp[WB - 1 - j], zcb, fma(K[WB - 1 - j], yn, Ws[q]));
  }
}

}  // namespace circ

template <typename R, int S, int L, int KIND, int WB, int NC, int RK = -1>
__global__ void __launch_bounds__(WB * NC) circ_strided_kernel(const __grid_constant__ CircArgs<R> A) {
  using namespace circ;
  namespace cg = cooperative_groups;
  extern __shared__ __align__(128) unsigned char circ_smem[];
  constexpr int ROWS = WB * L;           // rows of the line in this block
  constexpr int VW = 16 / sizeof(R);
  constexpr int HP = 32 / NC;            // chunks per warp (lanes: NC columns x HP chunks)
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const int c = lane % NC, h = lane / NC, j = w * HP + h;  // column, half, chunk
  const int cs = A.cs;
  const int rank = (int)(blockIdx.x % (unsigned)cs);
  // persistent: cluster (or block) cid walks the line groups cid, cid + ncl, ...
  const int ncl = (int)(gridDim.x / (unsigned)cs), cid = (int)(blockIdx.x / (unsigned)cs);
  const long long st = A.st;
  const int ngroups = A.ngroups;
  const unsigned nlob = (unsigned)A.nlo_blocks;
  auto group_base = [&](int g) -> long long {  // row 0, lane 0 of this block's tile of group g
    const unsigned hi = (unsigned)g / nlob, lo = (unsigned)g - hi * nlob;
    return (long long)lo * NC + ((long long)rank * ROWS) * st + (long long)hi * A.lst;
  };
  // tile [3 fields][S][ROWS * NC]: row t of chunk j at ((j / HP) L + t) 32 + (j % HP) NC,
  // so a warp's HP chunks read one 32-wide row (conflict-free)
  R *tile = reinterpret_cast<R *>(circ_smem);
  constexpr int XS = WB > 16 ? WB : 16;         // exchange rows (chunks of a block, or gathered blocks)
  constexpr size_t EX = (size_t)2 * 2 * S * XS * NC;  // one exchange buffer
  // two exchange buffers.  cs > 1: they alternate between receiving the
  // cluster's composites and composing the block's chunks (push exchange).
  // cs = 1: buf0 = [F, W][2S][XS][NC], buf1 = the block composites
  // [3 exchanges][2][2S][NC]
  R *buf0 = tile + (size_t)3 * S * ROWS * NC;
  R *buf1 = buf0 + EX;
  R *car = buf1 + EX;                          // [2][2S][NC]
  constexpr int TS = 2 * (WB + 1) + 35;
  R *tab = car + (size_t)2 * 2 * S * NC;       // [S * 3 matrices][TS]: the exchange's coefficient tables
  // A.tabg: the same tables prepared in global memory (blocks lean enough for
  // two per SM read them through L1 and have no shared copy)
  const R *tabp = A.tabg ? A.tabg : tab;
  for (int e = tid; !A.tabg && e < S * 3 * TS; e += WB * NC) {
    const int mx = e / TS, o = e - mx * TS;
    const R *kch = A.kch[mx / 3][mx % 3], *lpw = A.lpow[mx / 3][mx % 3];
    R v;
    if (o <= WB) v = kch[o];                                                    // K_{oL}
    else if (o <= 2 * WB + 1) v = lpw[o - (WB + 1)];                            // Lambda^n
    else if (o < 2 * WB + 2 + 17) {                                             // K at block multiples
      const int b = o - (2 * WB + 2);
      v = b * WB <= A.m ? kch[b * WB] : R(0);
    } else if (o < 2 * WB + 2 + 34) {                                           // Lambda at block multiples
      const int b = o - (2 * WB + 2 + 17);
      v = b * WB <= A.m ? lpw[b * WB] : R(0);
    } else v = kch[A.m];                                                        // K_{mL}
    tab[e] = v;
  }
  __syncthreads();
  auto Tf = [&](int f, int s) -> R * { return tile + (size_t)(f * S + s) * ROWS * NC; };
  // this thread's column of its chunk in field f, species s (row t at + t * 32)
  auto Tc = [&](int f, int s) -> R * { return Tf(f, s) + (w * L) * 32 + h * NC + c; };
  // NC = 32: every field buffer is one TMA box per species, completed on the
  // field's mbarrier (phase = this block's group count & 1)
  constexpr bool TMA = (NC == 32);
  __shared__ __align__(8) unsigned long long fbar[3];
  // push exchanges: xbar[b] completes when the other blocks' composites are in buf[b]
  __shared__ __align__(8) unsigned long long xbar[2];
  __shared__ int wait_fail;  // a bounded wait of this block gave up: later waits return at once
  if (tid == 0) wait_fail = 0;
  // solves of exchange number x (LAST: P, then T and S; MIDDLE: T and S twice, then P)
  auto ng_of = [&](int x) { return KIND == SWEEP_LAST ? ((x & 1) ? 2 * S : S) : (x % 3 == 2 ? S : 2 * S); };
  if (TMA || cs > 1) {
    if (tid == 0) {
      if constexpr (TMA)
        for (int f = 0; f < 3; ++f) mbar_init(&fbar[f], 1);
      if (cs > 1) {
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
      }
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
      if (cs > 1) {  // armed for exchanges 0 and 1
        mbar_expect_tx(&xbar[0], (unsigned)((cs - 1) * 2 * ng_of(0) * NC * (int)sizeof(R)));
        mbar_expect_tx(&xbar[1], (unsigned)((cs - 1) * 2 * ng_of(1) * NC * (int)sizeof(R)));
      }
    }
    // every block's barriers exist (and are armed) before any block pushes
    if (cs > 1) cg::this_cluster().sync();
    else __syncthreads();
  }
  int xc = 0;  // exchanges so far
  // one exchange of NG solves (blk_slot: composites slot of the one-block path)
  auto exchange = [&](auto mi, const auto &F, const auto &W, auto &Yc, auto &Zc, int blk_slot) {
    constexpr int NG = sizeof(F) / sizeof(R);
    if (cs > 1)
      strided_exchange_push<R, WB, NC, NG>(A, mi, F, W, Yc, Zc, buf0, buf1, xbar, xc, ng_of(xc + 2), car, tabp, j, c,
                                           w, h, rank, tid, &wait_fail);
    else
      strided_exchange<R, WB, NC, NG>(A, mi, F, W, Yc, Zc, buf0, buf0 + EX / 2,
                                      buf1 + (size_t)blk_slot * 2 * 2 * S * NC, car, tabp, j, c, w, h, rank);
    ++xc;
  };
  // stage field fld of group g into its buffer (TMA, or cp.async with 16-byte
  // pieces: always one commit group, empty past the last group, so the wait
  // counts hold)
  auto stage = [&](int fld, int g) {
    if constexpr (TMA) {
      if (tid == 0 && g < ngroups) {
        const unsigned hi = (unsigned)g / nlob, lo = (unsigned)g - hi * nlob;
        mbar_expect_tx(&fbar[fld], (unsigned)(S * ROWS * NC * sizeof(R)));
#pragma unroll
        for (int s = 0; s < S; ++s)
          tma_load_3d(Tf(fld, s), &A.tmap[fld], (int)(lo * NC), (int)(hi * A.p + rank * ROWS), s, &fbar[fld]);
      }
      return;
    }
    if (g < ngroups) {
      constexpr int PER_ROW = NC / VW;  // 16-byte pieces per row segment
      const long long gb = group_base(g);
#pragma unroll
      for (int s = 0; s < S; ++s)
#pragma unroll 1
        for (int k = tid; k < ROWS * PER_ROW; k += WB * NC) {
          const int row = k / PER_ROW, col = (k % PER_ROW) * VW;
          const int cj = row / L, ct = row - cj * L;
          cp_async16(Tf(fld, s) + ((cj / HP) * L + ct) * 32 + (cj % HP) * NC + col,
                     A.in[fld] + s * A.N + gb + (long long)row * st + col);
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  const int r0 = j * L;  // this thread's first row in the tile
  int it = 0;            // groups this block has processed (mbarrier phase)
  // wait until field fld of the current group is in shared memory; with
  // cp.async, `pending` is how many later commit groups may stay in flight
  // (TMA: every thread observes the field's mbarrier phase itself, no block barrier)
  auto wait_field = [&](int fld, int pending) {
    if constexpr (TMA) {
      if (!mbar_wait(&fbar[fld], (unsigned)(it & 1), &wait_fail)) atomicOr(&g_circ_status, 1);
    } else {
      if (pending >= 2) asm volatile("cp.async.wait_group 2;\n" ::: "memory");
      else if (pending == 1) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      __syncthreads();
    }
  };
  // the block is done with field fld of this group: refill its buffer with group gn
  auto refill = [&](int fld, int gn) {
    __syncthreads();
    stage(fld, gn);
  };

  if constexpr (KIND == SWEEP_MIDDLE) {
    // fields in order c_U, c_f, w; each is exchanged on its own, and its
    // buffer refilled with the next group's field right after its last read
    stage(0, cid);
    stage(1, cid);
    stage(2, cid);
#pragma unroll 1
    for (int g = cid; g < ngroups; g += ncl) {
      const long long mybase = group_base(g) + (long long)r0 * st + c;
      // R_2 = 9 T - 8 S on c_U, then on c_f
#pragma unroll 1
      for (int fld = 0; fld < 2; ++fld) {
        wait_field(fld, 2);
        R F[2 * S], W[2 * S], Yc[2 * S], Zc[2 * S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &MT = A.mat[s][1], &MS = A.mat[s][2];
          R y0 = R(0), w0 = R(0), y1 = R(0), w1 = R(0);
          const R *col = Tc(fld, s);
#pragma unroll
          for (int t = 0; t < L; ++t) {
            const R b = col[t * 32];
            y0 = fma(MT.lam, y0, b);
            w0 = fma(MT.pw[t], y0, w0);
            y1 = fma(MS.lam, y1, b);
            w1 = fma(MS.pw[t], y1, w1);
          }
          F[2 * s] = y0; W[2 * s] = w0;
          F[2 * s + 1] = y1; W[2 * s + 1] = w1;
        }
        auto mi = [&](int q) { return (q >> 1) * 3 + ((q & 1) ? 2 : 1); };
        exchange(mi, F, W, Yc, Zc, fld);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &MT = A.mat[s][1], &MS = A.mat[s][2];
          const R *col = Tc(fld, s);
          R *out = A.out[fld] + s * A.N + mybase;
          R zt[L], ys[L];
          R y = Yc[2 * s], y2 = Yc[2 * s + 1];
#pragma unroll
          for (int t = 0; t < L; ++t) {
            const R b = col[t * 32];
            y = fma(MT.lam, y, b);
            zt[t] = y;
            y2 = fma(MS.lam, y2, b);
            ys[t] = y2;
          }
          R z = Zc[2 * s], z2 = Zc[2 * s + 1];
          R *op = out + (long long)(L - 1) * st;  // row t of this chunk, stepped down
#pragma unroll
          for (int t = L - 1; t >= 0; --t) {
            z = fma(MT.lam, z, zt[t]);
            z2 = fma(MS.lam, z2, ys[t]);
            *op = fma(A.cT[s], z, -A.cS[s] * z2);  // R = 9T - 8S
            op -= st;
          }
        }
        refill(fld, g + ncl);  // every thread is done with this field's buffer
      }
      // P_2 on w
      {
        wait_field(2, 2);
        R F[S], W[S], Yc[S], Zc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &M = A.mat[s][0];
          R y = R(0), w = R(0);
          const R *col = Tc(2, s);
#pragma unroll
          for (int t = 0; t < L; ++t) {
            y = fma(M.lam, y, col[t * 32]);
            w = fma(M.pw[t], y, w);
          }
          F[s] = y;
          W[s] = w;
        }
        auto mi = [&](int q) { return q * 3; };
        exchange(mi, F, W, Yc, Zc, 2);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &M = A.mat[s][0];
          const R *col = Tc(2, s);
          R *out = A.out[2] + s * A.N + mybase;
          R ys[L];
          R y = Yc[s];
#pragma unroll
          for (int t = 0; t < L; ++t) {
            y = fma(M.lam, y, col[t * 32]);
            ys[t] = y;
          }
          R z = Zc[s];
          R *op = out + (long long)(L - 1) * st;  // row t of this chunk, stepped down
#pragma unroll
          for (int t = L - 1; t >= 0; --t) {
            z = fma(M.lam, z, ys[t]);
            *op = A.cP[s] * z;
            op -= st;
          }
        }
        refill(2, g + ncl);
      }
      ++it;
    }
  } else {
    // buffers: 2 = w (phase A), 0 = c_U, 1 = c_f (phase C, overwritten by f1, f2)
    stage(2, cid);
    stage(0, cid);
    stage(1, cid);
#pragma unroll 1
    for (int g = cid; g < ngroups; g += ncl) {
      const long long mybase = group_base(g) + (long long)r0 * st + c;
      // ---- phase A: U* = P_d w
      wait_field(2, 2);  // w of g (c_U, c_f may still be in flight)
      R Ustar[S][L];
      {
        R F[S], W[S], Yc[S], Zc[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &M = A.mat[s][0];
          const R *col = Tc(2, s);
          R y = R(0), w = R(0);
#pragma unroll
          for (int t = 0; t < L; ++t) {
            y = fma(M.lam, y, col[t * 32]);
            w = fma(M.pw[t], y, w);
          }
          F[s] = y;
          W[s] = w;
        }
        auto mi = [&](int q) { return q * 3 + 0; };
        exchange(mi, F, W, Yc, Zc, 0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const CircMat<R> &M = A.mat[s][0];
          const R *col = Tc(2, s);
          R y = Yc[s];
#pragma unroll
          for (int t = 0; t < L; ++t) {
            y = fma(M.lam, y, col[t * 32]);
            Ustar[s][t] = y;
          }
          R z = Zc[s];
#pragma unroll
          for (int t = L - 1; t >= 0; --t) {
            z = fma(M.lam, z, Ustar[s][t]);
            Ustar[s][t] = A.cP[s] * z;
          }
        }
      }
      refill(2, g + ncl);  // w of g fully read: refill with the next group's
      // ---- F(U*, t_{n+1}); f1, f2 over the staged c_U, c_f; summaries of T f1, S f2
      wait_field(0, 1);  // c_U, c_f of g
      wait_field(1, 1);
      R F[2 * S], W[2 * S], Yc[2 * S], Zc[2 * S];
#pragma unroll
      for (int q = 0; q < 2 * S; ++q) F[q] = W[q] = R(0);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], fr[S];
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = Ustar[s][t];
        reaction<R, S, RK>(A, u, fr);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          R *cu = Tc(0, s) + t * 32, *cf = Tc(1, s) + t * 32;
          const R a = *cu, b = *cf;
          const R f1 = fma(A.kR, fr[s], fma(R(2) * A.kR, b, R(9) * a));
          const R f2 = fma(A.half_kR, fr[s], fma(R(1.5) * A.kR, b, R(8) * a));
          *cu = f1;
          *cf = f2;
          const CircMat<R> &MT = A.mat[s][1], &MS = A.mat[s][2];
          F[2 * s] = fma(MT.lam, F[2 * s], f1);
          W[2 * s] = fma(MT.pw[t], F[2 * s], W[2 * s]);
          F[2 * s + 1] = fma(MS.lam, F[2 * s + 1], f2);
          W[2 * s + 1] = fma(MS.pw[t], F[2 * s + 1], W[2 * s + 1]);
        }
      }
      auto mi = [&](int q) { return (q >> 1) * 3 + ((q & 1) ? 2 : 1); };
      exchange(mi, F, W, Yc, Zc, 1);
      // ---- U_{n+1} = T_d f1 - S_d f2
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const CircMat<R> &MT = A.mat[s][1], &MS = A.mat[s][2];
        const R *c1 = Tc(0, s), *c2 = Tc(1, s);
        R zt[L], ys[L];
        R y = Yc[2 * s], y2 = Yc[2 * s + 1];
#pragma unroll
        for (int t = 0; t < L; ++t) {
          y = fma(MT.lam, y, c1[t * 32]);
          zt[t] = y;
          y2 = fma(MS.lam, y2, c2[t * 32]);
          ys[t] = y2;
        }
        R z = Zc[2 * s], z2 = Zc[2 * s + 1];
        R *out = A.out[0] + s * A.N + mybase;
        R *op = out + (long long)(L - 1) * st;  // row t of this chunk, stepped down
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
          z = fma(MT.lam, z, zt[t]);
          z2 = fma(MS.lam, z2, ys[t]);
          *op = fma(A.iaT[s], z, -A.iaS[s] * z2);
          op -= st;
        }
      }
      refill(0, g + ncl);  // f1, f2 of g fully read: refill with the next group's c_U, c_f
      stage(1, g + ncl);
      ++it;
    }
  }
  if constexpr (!TMA) asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  // no block of a cluster leaves while another may still read its shared memory
  if (cs > 1) cg::this_cluster().sync();
}

}  // namespace etd
