// etd_circ.cuh -- circulant sweeps of periodic axes (sm_103a): the first-axis
// (contiguous) sweep with lanes along the line.
//
// A block holds `lpb` whole lines of m chunks (p = m L); thread j of a line
// owns chunk j.  The chunk is staged in shared memory with cp.async (the
// thread's private slot, padded so that 16-byte reads of consecutive threads
// fall on distinct bank groups), so the passes keep only running values in
// registers.  Every solve runs as (see etd_circ.h for the algebra):
//   pass 1: zero-carry chunk summaries F_j, W_j (two FMAs per position, the
//           weights lambda^t are kernel-parameter constants);
//   round 1: an inclusive scan of F over the chunks of the line with the
//           constant multiplier Lambda (lane shuffles; lines of several warps
//           add one shared-memory step over the warp totals), closed
//           cyclically by the line total -> carry Yc_j of every chunk;
//   round 2: the same suffix scan of G_j = W_j + kappa Yc_j -> carry Zc_j;
//   pass 2: the recurrences y_i = b_i + lambda y_{i-1} and
//           z_i = y_i + lambda z_{i+1} over the chunk from (Yc_j, Zc_j).
// All 5 s solves of the sweep (T, S on U_n; T, S on F(U_n); P on
// U_n + k F(U_n)) share the two rounds; results leave as 32-byte stores.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "etd_circ.h"

namespace etd {

namespace circ {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ float rdivc(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double rdivc(double a, double b) { return a / b; }

// F(u) of the autonomous reactions (Section 8's models; periodic problems
// carry no manufactured source)
template <typename R, int S>
__device__ __forceinline__ void reaction(const CircArgs<R> &A, const R (&u)[S], R (&f)[S]) {
  switch (A.rkind) {
    case 1:
#pragma unroll
      for (int s = 0; s < S; ++s) f[s] = fma(A.rpR[0], u[s], A.rpR[1]);
      return;
    case 2:
      if constexpr (S == 2) {  // Brusselator: a + u^2 v - (b+1) u ; b u - u^2 v
        const R uuv = u[0] * u[0] * u[1];
        f[0] = A.rpR[0] + uuv - (A.rpR[1] + R(1)) * u[0];
        f[1] = A.rpR[1] * u[0] - uuv;
        return;
      }
      break;
    case 3:
      if constexpr (S == 2) {  // Schnakenberg: g (a - u + u^2 v) ; g (b - u^2 v)
        const R uuv = u[0] * u[0] * u[1];
        f[0] = A.rpR[2] * (A.rpR[0] - u[0] + uuv);
        f[1] = A.rpR[2] * (A.rpR[1] - uuv);
        return;
      }
      break;
    case 4:
      if constexpr (S == 2) {  // Gray-Scott: -u v^2 + F (1-u) ; u v^2 - (F+kappa) v
        const R uvv = u[0] * u[1] * u[1];
        f[0] = A.rpR[0] * (R(1) - u[0]) - uvv;
        f[1] = uvv - (A.rpR[0] + A.rpR[1]) * u[1];
        return;
      }
      break;
    case 5:  // enzyme kinetics without a source term
      f[0] = -rdivc(u[0], R(1) + u[0]);
#pragma unroll
      for (int s = 1; s < S; ++s) f[s] = R(0);
      return;
    default:
      break;
  }
#pragma unroll
  for (int s = 0; s < S; ++s) f[s] = R(0);
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

// solve q of species s: 0 T on U, 1 S on U, 2 T on F, 3 S on F, 4 P on U + k F
__host__ __device__ constexpr int qmat(int q) { return q == 4 ? 0 : (q & 1) ? 2 : 1; }

}  // namespace circ

// Thread j of a line: chunk j.  Block: lpb lines x m threads (max(m, 256) threads).
template <typename R, int S, int L>
__global__ void __launch_bounds__(512) circ_first_kernel(const __grid_constant__ CircArgs<R> A) {
  using namespace circ;
  extern __shared__ __align__(16) unsigned char circ_smem[];
  constexpr int VW = 16 / sizeof(R);   // elements per 16 bytes
  constexpr int CSZ = L + VW;          // padded chunk slot
  constexpr int NQ = 5;
  const int m = A.m, tid = threadIdx.x, nthr = blockDim.x;
  const int lb = tid / m, j = tid - lb * m;
  const long long line = (long long)blockIdx.x * A.lpb + lb;
  const bool ok = line < A.nlines;
  const int lane = tid & 31;
  const int G = m < 32 ? m : 32;       // lanes of one line in a warp
  const int gl = lane & (G - 1);
  const int nw = m > 32 ? m / 32 : 1;  // warps of one line
  const int w = j >> 5;
  R *stage = reinterpret_cast<R *>(circ_smem);
  R *tot = stage + (size_t)S * nthr * CSZ;  // [2][lpb][nw][S][NQ]

  // ---- stage U_n: thread-private padded slot per species ([s][tid][CSZ])
  const long long base = line * (long long)A.p + (long long)j * L;
  if (ok) {
#pragma unroll
    for (int s = 0; s < S; ++s)
#pragma unroll
      for (int v = 0; v < L; v += VW)
        cp_async16(stage + ((size_t)s * nthr + tid) * CSZ + v, A.in[0] + s * A.N + base + v);
  }
  cp_async_wait_all();
  auto su = [&](int s, int t) -> R { return stage[((size_t)s * nthr + tid) * CSZ + t]; };

  // ---- pass 1: zero-carry summaries of every solve
  R ty[S][NQ], tw[S][NQ];
#pragma unroll
  for (int s = 0; s < S; ++s)
#pragma unroll
    for (int q = 0; q < NQ; ++q) ty[s][q] = tw[s][q] = R(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    R u[S], f[S];
#pragma unroll
    for (int s = 0; s < S; ++s) u[s] = su(s, t);
    reaction<R, S>(A, u, f);
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

  // ---- round 1: forward carries Yc_j (inclusive scan of F, cyclic closure)
  R Yc[S][NQ];
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

  // ---- round 2: backward carries Zc_j (suffix scan of G = W + kappa Yc)
  R Zc[S][NQ];
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

  // ---- pass 2: recurrences from the carries, combination, 32-byte stores
  if (!ok) return;
#pragma unroll
  for (int s = 0; s < S; ++s) {
    const CircMat<R> &MP = A.mat[s][0], &MT = A.mat[s][1], &MS = A.mat[s][2];
    R fs[L];
#pragma unroll
    for (int t = 0; t < L; ++t) {
      R u[S], f[S];
#pragma unroll
      for (int r = 0; r < S; ++r) u[r] = su(r, t);
      reaction<R, S>(A, u, f);
      fs[t] = f[s];
    }
    R zt[L], ys[L];
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // h = 0: right-hand side U_n, h = 1: F(U_n)
      R y = Yc[s][2 * h];
#pragma unroll
      for (int t = 0; t < L; ++t) {
        y = fma(MT.lam, y, h ? fs[t] : su(s, t));
        zt[t] = y;
      }
      R z = Zc[s][2 * h];
#pragma unroll
      for (int t = L - 1; t >= 0; --t) {
        z = fma(MT.lam, z, zt[t]);
        zt[t] = z;
      }
      y = Yc[s][2 * h + 1];
#pragma unroll
      for (int t = 0; t < L; ++t) {
        y = fma(MS.lam, y, h ? fs[t] : su(s, t));
        ys[t] = y;
      }
      z = Zc[s][2 * h + 1];
#pragma unroll
      for (int t = L - 1; t >= 0; --t) {
        z = fma(MS.lam, z, ys[t]);
        zt[t] = fma(A.cT[s], zt[t], -A.cS[s] * z);  // R = 9T - 8S
      }
      R *o = A.out[h] + s * A.N + base;
#pragma unroll
      for (int t = 0; t < L; t += 32 / (int)sizeof(R)) st32(o + t, zt + t);
    }
    R y = Yc[s][4];
#pragma unroll
    for (int t = 0; t < L; ++t) {
      y = fma(MP.lam, y, fma(A.kR, fs[t], su(s, t)));
      zt[t] = y;
    }
    R z = Zc[s][4];
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      z = fma(MP.lam, z, zt[t]);
      zt[t] = A.cP[s] * z;
    }
    R *o = A.out[2] + s * A.N + base;
#pragma unroll
    for (int t = 0; t < L; t += 32 / (int)sizeof(R)) st32(o + t, zt + t);
  }
}

}  // namespace etd
