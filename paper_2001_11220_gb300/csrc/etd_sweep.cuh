// etd_sweep.cuh -- fused axis sweeps of one ETD-RDP-IF step (sm_103a).
//
// One block owns `nlb` complete lines of the swept axis; each thread owns one
// chunk of L consecutive positions of one line for every species, in
// registers.  Every line solve x = M^{-1} b (M tridiagonal, Section 7, with
// the LU factors of the Thomas variant precomputed per line matrix) runs in
// two register passes around one shared-memory exchange:
//   pass 1: per chunk, the zero-carry forward value at the chunk end
//           F_j = sum_t v_t b_t and the zero-carry backward value at the chunk
//           start Y_j = sum_t w_t b_t (dot products with precomputed weights);
//   scan:   one thread per (line, solve) chains the chunks: forward carries
//           G_in[j] and backward carries X[j+1] (and, for cyclic lines, the
//           Sherman-Morrison scalar in FP64);
//   pass 2: the exact Thomas recurrences over the chunk from those carries.
// All solves of a sweep share the one exchange, so a sweep reads each input
// field once and writes each output field once (Figs. flow2d / flow3d fused
// into FIRST / MIDDLE / LAST).
//
// Thread mapping: lanes walk neighbouring lines (l = tid % nlb), so table
// reads are warp broadcasts and, on strided axes, every load of position i is
// one coalesced row segment across the warp.  Pair mode (FP32, strided axes
// with an even stride): each thread owns the same chunk of two neighbouring
// lines as one float2 and runs every recurrence in the packed two-lane FP32
// instructions, halving the instructions per point.
#pragma once

#include <climits>

#include "etd_internal.h"

namespace etd {

#ifndef ETD_MAX_THREADS
#define ETD_MAX_THREADS 512
#endif

template <typename R>
__device__ __forceinline__ R ld_nc(const R *p) { return __ldg(p); }
// COH: the data may have been written earlier in the same launch (persistent
// ensemble step): load at the L2 (.cg), never through the read-only path
template <bool COH, typename R>
__device__ __forceinline__ R ld_in(const R *p) {
  if constexpr (COH) return __ldcg(p); else return __ldg(p);
}

// ------------------------------------------------------------ lane values
// V = R (one line per thread) or float2 (a pair of neighbouring lines).  For
// V = R the helpers are exactly the scalar operations (FP64 results do not
// change); for float2 they are the packed two-lane instructions.
template <typename R, int PK> struct LaneT { using T = R; };
template <> struct LaneT<float, 2> { using T = float2; };

__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double vfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float vmul(float a, float b) { return a * b; }
__device__ __forceinline__ double vmul(double a, double b) { return a * b; }
__device__ __forceinline__ float2 vmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float vsub(float a, float b) { return a - b; }
__device__ __forceinline__ double vsub(double a, double b) { return a - b; }
// a - b in one rounding: b * (-1) is exact
__device__ __forceinline__ float2 vsub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ float vneg(float a) { return -a; }
__device__ __forceinline__ double vneg(double a) { return -a; }
__device__ __forceinline__ float2 vneg(float2 a) { return make_float2(-a.x, -a.y); }

template <typename V> struct Splat;
template <> struct Splat<float> { __device__ static float of(float c) { return c; } };
template <> struct Splat<double> { __device__ static double of(double c) { return c; } };
template <> struct Splat<float2> { __device__ static float2 of(float c) { return make_float2(c, c); } };

template <typename V> __device__ __forceinline__ bool v_nonzero(V a) { return a != V(0); }
template <> __device__ __forceinline__ bool v_nonzero<float2>(float2 a) { return a.x != 0.f || a.y != 0.f; }

__device__ __forceinline__ float v_shfl_up(float a, int off) { return __shfl_up_sync(0xffffffffu, a, off); }
__device__ __forceinline__ double v_shfl_up(double a, int off) { return __shfl_up_sync(0xffffffffu, a, off); }
__device__ __forceinline__ float2 v_shfl_up(float2 a, int off) {
  return make_float2(__shfl_up_sync(0xffffffffu, a.x, off), __shfl_up_sync(0xffffffffu, a.y, off));
}
__device__ __forceinline__ float v_shfl_down(float a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
__device__ __forceinline__ double v_shfl_down(double a, int off) { return __shfl_down_sync(0xffffffffu, a, off); }
__device__ __forceinline__ float2 v_shfl_down(float2 a, int off) {
  return make_float2(__shfl_down_sync(0xffffffffu, a.x, off), __shfl_down_sync(0xffffffffu, a.y, off));
}
__device__ __forceinline__ float v_shfl(float a, int src) { return __shfl_sync(0xffffffffu, a, src); }
__device__ __forceinline__ double v_shfl(double a, int src) { return __shfl_sync(0xffffffffu, a, src); }
__device__ __forceinline__ float2 v_shfl(float2 a, int src) {
  return make_float2(__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src));
}

// Sherman-Morrison scalar sigma = (v . y) / (1 + v . z) in FP64 from the
// line's first (y_0) and last (y_{p-1}) values, one per lane of V, stored
// in the precision the sweep uses it in (FP32 sweeps round it once here)
template <typename T>
__device__ __forceinline__ void put_sigma(T *dst, const MatTab<float> &M, float y0, float yl) {
  if (M.sm_inv != 0.0) dst[0] = (T)(((double)y0 + M.sm_c * (double)yl) * M.sm_inv);
  else dst[0] = T(0);
}
__device__ __forceinline__ void put_sigma(double *dst, const MatTab<double> &M, double y0, double yl) {
  if (M.sm_inv != 0.0) dst[0] = (y0 + M.sm_c * yl) * M.sm_inv;
  else dst[0] = 0.0;
}
__device__ __forceinline__ void put_sigma(float *dst, const MatTab<float> &M, float2 y0, float2 yl) {
  put_sigma(dst, M, y0.x, yl.x);
  put_sigma(dst + 1, M, y0.y, yl.y);
}
template <typename R>
__device__ __forceinline__ R get_sigma(const R *src, R) { return src[0]; }
__device__ __forceinline__ float2 get_sigma(const float *src, float2) { return make_float2(src[0], src[1]); }

// a / b in the reactions: IEEE division in FP64; the hardware fast divide
// (a few ulp) in FP32, whose arithmetic error budget is far larger
__device__ __forceinline__ double rdiv(double a, double b) { return a / b; }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdividef(a, b); }

// ---------------------------------------------------------------- reaction

template <typename R, int S>
__device__ __forceinline__ void reaction_point(const SweepArgs<R> &A, const R (&u)[S], R (&f)[S], R src) {
  switch (A.rkind) {
    case 1:
#pragma unroll
      for (int s = 0; s < S; ++s) f[s] = fma(A.rpR[0], u[s], A.rpR[1]);
      return;
    case 2:
      if constexpr (S == 2) {  // Brusselator: a + u^2 v - (b+1) u ; b u - u^2 v
        const R a = A.rpR[0], b = A.rpR[1];
        const R uuv = u[0] * u[0] * u[1];
        f[0] = a + uuv - (b + R(1)) * u[0];
        f[1] = b * u[0] - uuv;
        return;
      }
      break;
    case 3:
      if constexpr (S == 2) {  // Schnakenberg: g (a - u + u^2 v) ; g (b - u^2 v)
        const R a = A.rpR[0], b = A.rpR[1], g = A.rpR[2];
        const R uuv = u[0] * u[0] * u[1];
        f[0] = g * (a - u[0] + uuv);
        f[1] = g * (b - uuv);
        return;
      }
      break;
    case 4:
      if constexpr (S == 2) {  // Gray-Scott: -u v^2 + F (1-u) ; u v^2 - (F+kappa) v
        const R F = A.rpR[0], kap = A.rpR[1];
        const R uvv = u[0] * u[1] * u[1];
        f[0] = F * (R(1) - u[0]) - uvv;
        f[1] = uvv - (F + kap) * u[1];
        return;
      }
      break;
    case 6:
      if constexpr (S == 2) {  // CGL (alpha = 0): u - (1 + i beta) u |u|^2, u = u0 + i u1
        const R beta = A.rpR[0], r = fma(u[0], u[0], u[1] * u[1]);
        f[0] = fma(-r, fma(-beta, u[1], u[0]), u[0]);
        f[1] = fma(-r, fma(beta, u[0], u[1]), u[1]);
        return;
      }
      break;
    case 5:  // enzyme kinetics (Section 8.1) plus the manufactured source
      f[0] = -rdiv(u[0], R(1) + u[0]) + src;
#pragma unroll
      for (int s = 1; s < S; ++s) f[s] = R(0);
      return;
    default:
      break;
  }
#pragma unroll
  for (int s = 0; s < S; ++s) f[s] = R(0);
}

// e^{-t} prod_{b != axis} sin(pi x_b / L_b) for one line: x axis line index
// (y + z ny), strided axes (lo, hi) line coordinates; 0 without a source
template <typename R>
__device__ __forceinline__ R line_source_base(const SweepArgs<R> &A, bool contig, long long line, long long lo,
                                              long long hi, R exp_mt) {
  if (A.phi[0] == nullptr) return R(0);
  R q = exp_mt;
  if (contig) {
    q *= A.phi[1][line % A.ny];
    if (A.phi[2]) q *= A.phi[2][line / A.ny];
  } else if (A.axis == 1) {  // lo = x, hi = z
    q *= A.phi[0][lo];
    if (A.phi[2]) q *= A.phi[2][hi];
  } else {  // axis 2: lo = x + y nx
    q *= A.phi[0][lo % A.nx] * A.phi[1][lo / A.nx];
  }
  return q;
}

// ------------------------------------------------------------ chunk loads

// 32-byte global accesses (sm_100+): one instruction moves a whole sector per
// thread, so a warp's chunk loads and stores on contiguous lines fill every
// sector they touch (16-byte accesses leave each sector half written per
// instruction); the address must be 32-byte aligned
__device__ __forceinline__ void ld32B(const float *p, float *v) {
  asm volatile("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p));
}
__device__ __forceinline__ void ld32B(const double *p, double *v) {
  asm volatile("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];\n"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(p));
}
__device__ __forceinline__ void ld32B_cg(const float *p, float *v) {
  asm volatile("ld.global.cg.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
               : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void ld32B_cg(const double *p, double *v) {
  asm volatile("ld.global.cg.v4.f64 {%0, %1, %2, %3}, [%4];\n"
               : "=d"(v[0]), "=d"(v[1]), "=d"(v[2]), "=d"(v[3])
               : "l"(p)
               : "memory");
}
__device__ __forceinline__ void st32B(float *p, const float *v) {
  asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};\n" ::"l"(p), "f"(v[0]), "f"(v[1]),
               "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
               : "memory");
}
__device__ __forceinline__ void st32B(double *p, const double *v) {
  asm volatile("st.global.v4.f64 [%0], {%1, %2, %3, %4};\n" ::"l"(p), "d"(v[0]), "d"(v[1]), "d"(v[2]), "d"(v[3])
               : "memory");
}

template <typename R, int L, bool CONTIG, bool COH = false>
__device__ __forceinline__ void load_chunk(R (&v)[L], const R *__restrict__ p, long long off, long long st,
                                           int cnt) {
  if constexpr (CONTIG && L % (32 / sizeof(R)) == 0) {
    if (cnt == L && ((reinterpret_cast<uintptr_t>(p + off) & 31) == 0)) {
#pragma unroll
      for (int t = 0; t < L; t += 32 / sizeof(R)) {
        if constexpr (COH) ld32B_cg(p + off + t, v + t); else ld32B(p + off + t, v + t);
      }
      return;
    }
  }
  if constexpr (CONTIG) {
    constexpr int VW = 16 / sizeof(R);
    if (L % VW == 0 && cnt == L && ((reinterpret_cast<uintptr_t>(p + off) & 15) == 0)) {
      using V4 = typename V4T<R>::T;
      (void)sizeof(V4);
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int t = 0; t < L; t += 4) {
          float4 q = ld_in<COH>(reinterpret_cast<const float4 *>(p + off + t));
          v[t] = q.x; v[t + 1] = q.y; v[t + 2] = q.z; v[t + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < L; t += 2) {
          double2 q = ld_in<COH>(reinterpret_cast<const double2 *>(p + off + t));
          v[t] = q.x; v[t + 1] = q.y;
        }
      }
      return;
    }
  }
  const R *q = p + off;
  if (st <= INT_MAX / L) {  // 32-bit offsets within the chunk; full chunks without per-element tests
    const int s32 = (int)st;
    if (cnt == L) {
#pragma unroll
      for (int t = 0; t < L; ++t) v[t] = ld_in<COH>(q + t * s32);
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) v[t] = (t < cnt) ? ld_in<COH>(q + t * s32) : R(0);
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < L; ++t) v[t] = (t < cnt) ? ld_in<COH>(q + (long long)t * st) : R(0);
}

template <typename R, int L, bool CONTIG>
__device__ __forceinline__ void store_chunk(const R (&v)[L], R *__restrict__ p, long long off, long long st,
                                            int cnt) {
  if constexpr (CONTIG && L % (32 / sizeof(R)) == 0) {
    if (cnt == L && ((reinterpret_cast<uintptr_t>(p + off) & 31) == 0)) {
#pragma unroll
      for (int t = 0; t < L; t += 32 / sizeof(R)) st32B(p + off + t, v + t);
      return;
    }
  }
  if constexpr (CONTIG) {
    constexpr int VW = 16 / sizeof(R);
    if (L % VW == 0 && cnt == L && ((reinterpret_cast<uintptr_t>(p + off) & 15) == 0)) {
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int t = 0; t < L; t += 4)
          *reinterpret_cast<float4 *>(p + off + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
      } else {
#pragma unroll
        for (int t = 0; t < L; t += 2)
          *reinterpret_cast<double2 *>(p + off + t) = make_double2(v[t], v[t + 1]);
      }
      return;
    }
  }
  R *q = p + off;
  if (st <= INT_MAX / L) {
    const int s32 = (int)st;
    if (cnt == L) {
#pragma unroll
      for (int t = 0; t < L; ++t) q[t * s32] = v[t];
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t)
        if (t < cnt) q[t * s32] = v[t];
    }
    return;
  }
#pragma unroll
  for (int t = 0; t < L; ++t)
    if (t < cnt) q[(long long)t * st] = v[t];
}


// ------------------------------------------- interior chunks, FP32 fast path
// In chunks 0 < j < m-1 every row has l = u = -r, so the forward multiplier
// is the constant r and alpha = -r e: only e (and v, w, z) vary per position,
// read four positions per load.  Edge chunks (Neumann rows, padding) and FP64
// use the exact per-position tables.
template <typename R>
__device__ __forceinline__ bool interior_chunk(const MatTab<R> &M, int j, int m) {
  if constexpr (sizeof(R) == 4) return j > 0 && j < m - 1 && M.e1 != nullptr;
  else return false;
}

template <int L>
__device__ __forceinline__ void load_row4(const float *__restrict__ p, float (&a)[L]) {
#pragma unroll
  for (int t = 0; t < L; t += 4) {
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p + t));
    a[t] = v.x;
    a[t + 1] = v.y;
    a[t + 2] = v.z;
    a[t + 3] = v.w;
  }
}

// ------------------------------------------------------ pass 1 / pass 2

// chunk summaries of one RHS against one matrix
template <typename R, int L>
__device__ __forceinline__ void pass1(const MatTab<R> &M, int m, int j, const R (&b)[L], R &F, R &Y) {
  R f = R(0), y = R(0);
  if constexpr (sizeof(R) == 4 && L % 4 == 0) {
    if (interior_chunk(M, j, m)) {
      float v[L], w[L];
      load_row4<L>(M.v1 + j * L, v);
      load_row4<L>(M.w1 + j * L, w);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        f = fmaf(v[t], b[t], f);
        y = fmaf(w[t], b[t], y);
      }
      F = f;
      Y = y;
      return;
    }
  }
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const typename V2T<R>::T vw = M.sum[j * L + t];
    f = fma(vw.x, b[t], f);
    y = fma(vw.y, b[t], y);
  }
  F = f;
  Y = y;
}

// two RHS against one matrix (one table read)
template <typename R, int L>
__device__ __forceinline__ void pass1x2(const MatTab<R> &M, int m, int j, const R (&b0)[L], const R (&b1)[L],
                                        R &F0, R &Y0, R &F1, R &Y1) {
  R f0 = R(0), y0 = R(0), f1 = R(0), y1 = R(0);
  if constexpr (sizeof(R) == 4 && L % 4 == 0) {
    if (interior_chunk(M, j, m)) {
      float v[L], w[L];
      load_row4<L>(M.v1 + j * L, v);
      load_row4<L>(M.w1 + j * L, w);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        f0 = fmaf(v[t], b0[t], f0);
        y0 = fmaf(w[t], b0[t], y0);
        f1 = fmaf(v[t], b1[t], f1);
        y1 = fmaf(w[t], b1[t], y1);
      }
      F0 = f0; Y0 = y0; F1 = f1; Y1 = y1;
      return;
    }
  }
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const typename V2T<R>::T vw = M.sum[j * L + t];
    f0 = fma(vw.x, b0[t], f0);
    y0 = fma(vw.y, b0[t], y0);
    f1 = fma(vw.x, b1[t], f1);
    y1 = fma(vw.y, b1[t], y1);
  }
  F0 = f0; Y0 = y0; F1 = f1; Y1 = y1;
}

// exact Thomas recurrences over the chunk given the forward carry Gin (g at
// the position before the chunk), the backward carry Xr (x at the position
// after the chunk) and the Sherman-Morrison scalar sig (0 for open lines)
template <typename R, int L>
__device__ __forceinline__ void pass2(const MatTab<R> &M, int m, int j, const R (&b)[L], R Gin, R Xr, R sig,
                                      R (&x)[L]) {
  if constexpr (sizeof(R) == 4 && L % 4 == 0) {
    if (interior_chunk(M, j, m)) {
      float e[L];
      load_row4<L>(M.e1 + j * L, e);
      const float r = (float)M.r;
      float g = Gin;
#pragma unroll
      for (int t = 0; t < L; ++t) {
        g = fmaf(r, g, b[t]) * e[t];
        x[t] = g;
      }
      float xn = Xr;
      if (sig != 0.f) {
        float z[L];
        load_row4<L>(M.z1 + j * L, z);
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
          xn = fmaf(r * e[t], xn, x[t]);
          x[t] = fmaf(-sig, z[t], xn);
        }
      } else {
#pragma unroll
        for (int t = L - 1; t >= 0; --t) {
          xn = fmaf(r * e[t], xn, x[t]);
          x[t] = xn;
        }
      }
      return;
    }
  }
  R g = Gin;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const typename V4T<R>::T q = M.pos[j * L + t];
    g = fma(q.x, g, b[t]) * q.y;
    x[t] = g;
  }
  R xn = Xr;
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    const typename V4T<R>::T q = M.pos[j * L + t];
    xn = fma(-q.z, xn, x[t]);
    x[t] = fma(-sig, q.w, xn);
  }
}

// ------------------------------------------------- pass 1 / pass 2, FP32
// FP32 sweeps read per-position coefficient rows (MatTab::rows1, and
// MatTab::rows2 with each value in both lanes of a float2 for line pairs):
// row k at k m L (k: 0 ne = nl e, 1 e, 2 -alpha, 3 z, 4 v, 5 w), entry (t, j)
// at j L + t for every position (edge chunks and padding included), 16 bytes
// per load.  The forward recurrence runs as g_i = ne_i g_{i-1} + e_i b_i: one
// FMA on the dependency chain per position (e_i b_i is off the chain).  FP64
// keeps the operation order of Section 7 (pass1 / pass2 above).
__device__ __forceinline__ const float *rows_of(const MatTab<float> &M, float) { return M.rows1; }
__device__ __forceinline__ const float2 *rows_of(const MatTab<float> &M, float2) { return M.rows2; }

template <int L>
__device__ __forceinline__ void load_rows(const float *__restrict__ p, float (&a)[L]) {
  static_assert(L % 4 == 0, "FP32 rows are read four positions at a time");
#pragma unroll
  for (int t = 0; t < L; t += 4) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p + t));
    a[t] = q.x;
    a[t + 1] = q.y;
    a[t + 2] = q.z;
    a[t + 3] = q.w;
  }
}
template <int L>
__device__ __forceinline__ void load_rows(const float2 *__restrict__ p, float2 (&a)[L]) {
#pragma unroll
  for (int t = 0; t < L; t += 2) {
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p + t));
    a[t] = make_float2(q.x, q.y);
    a[t + 1] = make_float2(q.z, q.w);
  }
}

// chunk summaries F = sum v b, Y = sum w b of one or two right-hand sides
template <typename V, int L>
__device__ __forceinline__ void pass1v(const MatTab<float> &M, int m, int j, const V (&b)[L], V &F, V &Y) {
  const int ml = m * L;
  const V *row = rows_of(M, V()) + j * L;
  V v[L], w[L];
  load_rows<L>(row + 4 * ml, v);
  load_rows<L>(row + 5 * ml, w);
  V f = Splat<V>::of(0.f), y = f;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    f = vfma(v[t], b[t], f);
    y = vfma(w[t], b[t], y);
  }
  F = f;
  Y = y;
}

template <typename V, int L>
__device__ __forceinline__ void pass1x2v(const MatTab<float> &M, int m, int j, const V (&b0)[L], const V (&b1)[L],
                                         V &F0, V &Y0, V &F1, V &Y1) {
  const int ml = m * L;
  const V *row = rows_of(M, V()) + j * L;
  V v[L], w[L];
  load_rows<L>(row + 4 * ml, v);
  load_rows<L>(row + 5 * ml, w);
  V f0 = Splat<V>::of(0.f), y0 = f0, f1 = f0, y1 = f0;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    f0 = vfma(v[t], b0[t], f0);
    y0 = vfma(w[t], b0[t], y0);
    f1 = vfma(v[t], b1[t], f1);
    y1 = vfma(w[t], b1[t], y1);
  }
  F0 = f0; Y0 = y0; F1 = f1; Y1 = y1;
}

// Carries and Sherman-Morrison scalar of one solve: G (forward value before
// the chunk), X (solution after the chunk), ns = -sigma (0 on open lines).
template <typename V> struct Carry { V G, X, ns; };

// Two independent solves (matrices M0, M1; SAME: one matrix, rows read once)
// run interleaved: forward values into g0 / g1 (which may alias b0 / b1),
// then the backward recurrence hands each solution value to epi(t, k, x),
// k = 0, 1, from the last position down.
template <typename V, int L, bool SAME, typename Epi>
__device__ __forceinline__ void pass2x2v(const MatTab<float> &M0, const MatTab<float> &M1, int m, int j,
                                         const V (&b0)[L], const V (&b1)[L], Carry<V> c0, Carry<V> c1, V (&g0)[L],
                                         V (&g1)[L], Epi epi) {
  const int ml = m * L;
  const V *r0 = rows_of(M0, V()) + j * L;
  const V *r1 = SAME ? r0 : rows_of(M1, V()) + j * L;
  {
    V ne0[L], e0[L];
    load_rows<L>(r0, ne0);
    load_rows<L>(r0 + ml, e0);
    if constexpr (SAME) {
#pragma unroll
      for (int t = 0; t < L; ++t) {
        c0.G = vfma(ne0[t], c0.G, vmul(e0[t], b0[t]));
        c1.G = vfma(ne0[t], c1.G, vmul(e0[t], b1[t]));
        g0[t] = c0.G;
        g1[t] = c1.G;
      }
    } else {
      V ne1[L], e1[L];
      load_rows<L>(r1, ne1);
      load_rows<L>(r1 + ml, e1);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        c0.G = vfma(ne0[t], c0.G, vmul(e0[t], b0[t]));
        c1.G = vfma(ne1[t], c1.G, vmul(e1[t], b1[t]));
        g0[t] = c0.G;
        g1[t] = c1.G;
      }
    }
  }
  V na0[L], na1[L];
  load_rows<L>(r0 + 2 * ml, na0);
  if constexpr (SAME) {
#pragma unroll
    for (int t = 0; t < L; ++t) na1[t] = na0[t];
  } else {
    load_rows<L>(r1 + 2 * ml, na1);
  }
  if (v_nonzero(c0.ns) || v_nonzero(c1.ns)) {
    V z0[L], z1[L];
    load_rows<L>(r0 + 3 * ml, z0);
    if constexpr (SAME) {
#pragma unroll
      for (int t = 0; t < L; ++t) z1[t] = z0[t];
    } else {
      load_rows<L>(r1 + 3 * ml, z1);
    }
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      c0.X = vfma(na0[t], c0.X, g0[t]);
      c1.X = vfma(na1[t], c1.X, g1[t]);
      epi(t, 0, vfma(c0.ns, z0[t], c0.X));
      epi(t, 1, vfma(c1.ns, z1[t], c1.X));
    }
  } else {
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      c0.X = vfma(na0[t], c0.X, g0[t]);
      c1.X = vfma(na1[t], c1.X, g1[t]);
      epi(t, 0, c0.X);
      epi(t, 1, c1.X);
    }
  }
}

// one solve: forward values into g (may alias b), solutions to epi(t, x)
template <typename V, int L, typename Epi>
__device__ __forceinline__ void pass2v(const MatTab<float> &M, int m, int j, const V (&b)[L], Carry<V> c, V (&g)[L],
                                       Epi epi) {
  const int ml = m * L;
  const V *row = rows_of(M, V()) + j * L;
  {
    V ne[L], e[L];
    load_rows<L>(row, ne);
    load_rows<L>(row + ml, e);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      c.G = vfma(ne[t], c.G, vmul(e[t], b[t]));
      g[t] = c.G;
    }
  }
  V na[L];
  load_rows<L>(row + 2 * ml, na);
  if (v_nonzero(c.ns)) {
    V z[L];
    load_rows<L>(row + 3 * ml, z);
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      c.X = vfma(na[t], c.X, g[t]);
      epi(t, vfma(c.ns, z[t], c.X));
    }
  } else {
#pragma unroll
    for (int t = L - 1; t >= 0; --t) {
      c.X = vfma(na[t], c.X, g[t]);
      epi(t, c.X);
    }
  }
}

// --------------------------------------------------------------- scan

// chunk-table entry j through the read-only path: the compiler may then
// hoist these loads past the scan's shared-memory stores
__device__ __forceinline__ float4 ld_chunk(const MatTab<float> &M, int j) { return __ldg(M.chunk + j); }
__device__ __forceinline__ double4 ld_chunk(const MatTab<double> &M, int j) {
  const double2 *p = reinterpret_cast<const double2 *>(M.chunk + j);
  const double2 a = __ldg(p), b = __ldg(p + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

// Chunk-table cache in shared memory (entries of the block's chunks, filled
// at the start of the sweep; see chunk_sweep)
__device__ __forceinline__ float4 ld_cc(const float4 *p, int j) { return p[j]; }
__device__ __forceinline__ double4 ld_cc(const double4 *p, int j) {
  const double2 *q = reinterpret_cast<const double2 *>(p + j);
  const double2 a = q[0], b = q[1];
  return make_double4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_cc(float4 *p, int j, float4 v) { p[j] = v; }
__device__ __forceinline__ void st_cc(double4 *p, int j, double4 v) {
  double2 *q = reinterpret_cast<double2 *>(p + j);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}

// chunk entry jb + j of M: from the block's cache cc (entry j) when there is one
template <typename R>
__device__ __forceinline__ typename V4T<R>::T chunk_at(const MatTab<R> &M, int jb,
                                                      const typename V4T<R>::T *cc, int j) {
  return cc ? ld_cc(cc, j) : ld_chunk(M, jb + j);
}

// Sequential carry chain of one (line, solve) over m chunks (chunk-table
// entries jb .. jb+m-1): F[j] (chunk summary) becomes the forward carry
// G_in[j], Y[j] the backward carry X[j+1], starting from the forward carry G0
// into the first chunk and the solution value X0 after the last (0 and 0 for
// a whole line); G and X return the forward value after the last chunk and
// the solution value at the first position.  The chain runs in batches of 8
// chunks whose loads are all issued before the batch's dependent FMAs (rows
// and chunk tables are padded to a multiple of 8; padding entries may hold
// anything: the forward value is taken at chunk m-1 and the backward carry is
// held at X0 past the end).
template <typename R, typename V>
__device__ __forceinline__ void chain_line(const MatTab<R> &M, V *F, V *Y, int m, int jb, V G0, V X0, V &Gout,
                                           V &Xout) {
  constexpr int SB = 8;
  const int nb = (m + SB - 1) / SB;
  V G = G0, Gl = G0;
  for (int b = 0; b < nb; ++b) {
    const int j0 = b * SB;
    V f[SB];
    R a[SB];
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      f[k] = F[j0 + k];
      a[k] = ld_chunk(M, jb + j0 + k).x;
    }
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      F[j0 + k] = G;
      G = vfma(Splat<V>::of(a[k]), G, f[k]);
      Gl = (j0 + k == m - 1) ? G : Gl;
    }
  }
  V X = X0;
  for (int b = nb - 1; b >= 0; --b) {
    const int j0 = b * SB;
    V gi[SB], yv[SB];
    R cy[SB], cz[SB];
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      const typename V4T<R>::T c = ld_chunk(M, jb + j0 + k);
      gi[k] = F[j0 + k];
      yv[k] = Y[j0 + k];
      cy[k] = c.y;
      cz[k] = c.z;
    }
#pragma unroll
    for (int k = SB - 1; k >= 0; --k) {
      const V y = vfma(Splat<V>::of(cy[k]), gi[k], yv[k]);
      Y[j0 + k] = X;
      X = (j0 + k < m) ? vfma(Splat<V>::of(cz[k]), X, y) : X;
    }
  }
  Gout = Gl;
  Xout = X;
}

__device__ __forceinline__ float4 ld_segc(const MatTab<float> &M, int k) { return __ldg(M.segc + k); }
__device__ __forceinline__ double4 ld_segc(const MatTab<double> &M, int k) {
  const double2 *p = reinterpret_cast<const double2 *>(M.segc + k);
  const double2 a = __ldg(p), b = __ldg(p + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

// lane k of a lane value (one line or a pair)
__device__ __forceinline__ float v_get(float a, int) { return a; }
__device__ __forceinline__ double v_get(double a, int) { return a; }
__device__ __forceinline__ float v_get(float2 a, int k) { return k ? a.y : a.x; }
__device__ __forceinline__ void v_set(float &a, int, float x) { a = x; }
__device__ __forceinline__ void v_set(double &a, int, double x) { a = x; }
__device__ __forceinline__ void v_set(float2 &a, int k, float x) {
  if (k) a.y = x;
  else a.x = x;
}

// solve q of a sweep -> (species, matrix index)
template <typename R, int S, int KIND>
__device__ __forceinline__ void solve_matrix(int q, int &s, int &g) {
  if constexpr (KIND == SWEEP_LAST) {
    if (q < S) { s = q; g = 0; } else { s = (q - S) >> 1; g = 1 + ((q - S) & 1); }
  } else {
    s = q / 5;
    const int r = q - 5 * s;
    g = (r == 4) ? 0 : 1 + (r & 1);
  }
}


// chain_line reading the chunk entries from the block's cache cc (entry j = chunk jb + j)
template <typename R, typename V>
__device__ __forceinline__ void chain_line_cc(const MatTab<R> &M, V *F, V *Y, int m, int jb, V G0, V X0, V &Gout,
                                           V &Xout, const typename V4T<R>::T *cc) {
  constexpr int SB = 8;
  const int nb = (m + SB - 1) / SB;
  V G = G0, Gl = G0;
  for (int b = 0; b < nb; ++b) {
    const int j0 = b * SB;
    V f[SB];
    R a[SB];
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      f[k] = F[j0 + k];
      a[k] = chunk_at(M, jb, cc, j0 + k).x;
    }
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      F[j0 + k] = G;
      G = vfma(Splat<V>::of(a[k]), G, f[k]);
      Gl = (j0 + k == m - 1) ? G : Gl;
    }
  }
  V X = X0;
  for (int b = nb - 1; b >= 0; --b) {
    const int j0 = b * SB;
    V gi[SB], yv[SB];
    R cy[SB], cz[SB];
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      const typename V4T<R>::T c = chunk_at(M, jb, cc, j0 + k);
      gi[k] = F[j0 + k];
      yv[k] = Y[j0 + k];
      cy[k] = c.y;
      cz[k] = c.z;
    }
#pragma unroll
    for (int k = SB - 1; k >= 0; --k) {
      const V y = vfma(Splat<V>::of(cy[k]), gi[k], yv[k]);
      Y[j0 + k] = X;
      X = (j0 + k < m) ? vfma(Splat<V>::of(cz[k]), X, y) : X;
    }
  }
  Gout = Gl;
  Xout = X;
}

// Long lines (m > 32 chunks): one warp per (line, solve).  Each lane composes
// the affine chunk maps of a contiguous block of chunks, a shuffle scan over
// the lanes gives every block its carries, and the lane re-walks its block to
// emit G_in[j] and X[j+1] (forward map G -> Aend G + F, backward map
// X -> Bst X + Y + kappa G_in).  V is the lane value (one line or a pair);
// sSig holds PK Sherman-Morrison scalars per (solve, line unit).
template <typename R, typename V, int PK, typename SigT, typename GetMat>
__device__ __forceinline__ void scan_lines_warp(const SweepArgs<R> &A, V *sF, V *sY, SigT *sSig, int q0, int nq,
                                                GetMat mat) {
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  // full warps only: a trailing partial warp (blockDim not a multiple of 32) stays out of the shuffles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp >= nw) return;
  const int per = (m + 31) >> 5;
  const int j0 = min(lane * per, m), j1 = min(j0 + per, m);
  const V one = Splat<V>::of(R(1)), zero = Splat<V>::of(R(0));
  for (int u = warp; u < nlb * nq; u += nw) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    const MatTab<R> &M = mat(q);
    V *F = sF + (q * nlb + l) * pitch;  // shared-memory offsets in 32-bit arithmetic
    V *Y = sY + (q * nlb + l) * pitch;
    // forward: block map G_out = a G_in + b
    V a = one, b = zero;
    for (int jj = j0; jj < j1; ++jj) {
      const V Aj = Splat<V>::of(ld_chunk(M, jj).x);
      b = vfma(Aj, b, F[jj]);
      a = vmul(a, Aj);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const V ap = v_shfl_up(a, off), bp = v_shfl_up(b, off);
      if (lane >= off) {
        b = vfma(a, bp, b);
        a = vmul(a, ap);
      }
    }
    V G = v_shfl_up(b, 1);
    if (lane == 0) G = zero;
    const V Gtot = v_shfl(b, 31);  // forward value at the last position
    for (int jj = j0; jj < j1; ++jj) {
      const typename V4T<R>::T c = ld_chunk(M, jj);
      const V f = F[jj];
      F[jj] = G;
      Y[jj] = vfma(Splat<V>::of(c.y), G, Y[jj]);
      G = vfma(Splat<V>::of(c.x), G, f);
    }
    // backward: block map X_out = a X_in + b, composed from the right
    a = one;
    b = zero;
    for (int jj = j1 - 1; jj >= j0; --jj) {
      const V Bj = Splat<V>::of(ld_chunk(M, jj).z);
      b = vfma(Bj, b, Y[jj]);
      a = vmul(a, Bj);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const V an = v_shfl_down(a, off), bn = v_shfl_down(b, off);
      if (lane + off < 32) {
        b = vfma(a, bn, b);
        a = vmul(a, an);
      }
    }
    V X = v_shfl_down(b, 1);
    if (lane == 31) X = zero;
    for (int jj = j1 - 1; jj >= j0; --jj) {
      const V yv = Y[jj];
      Y[jj] = X;
      X = vfma(Splat<V>::of(ld_chunk(M, jj).z), X, yv);
    }
    const V X0 = v_shfl(X, 0);  // first position of the line
    if (lane == 0) put_sigma(sSig + (q * nlb + l) * PK, M, X0, Gtot);
  }
}

// Where a block's chunks sit in their lines, for the carry chains.
struct SegCtx {
  int phase;       // SEG_WHOLE: whole lines; SEG_SUMMARY: zero-carry chains, segment summaries
                   // to global memory; SEG_SOLVE: chains start from the segment carries
  int seg;         // segment of this block
  int jb;          // first chunk of the segment (chunk-table offset)
  int mv;          // chunks of the segment inside the line
  long long gl0;   // global index of the block's line (unit) 0
  int nvalid;      // lines (units) of the block inside the grid
};

__device__ __forceinline__ SegCtx whole_lines(int m) { return SegCtx{SEG_WHOLE, 0, 0, m, 0, 0}; }

// Chunk-table cache of a cluster-segmented block (see chunk_sweep): matrix
// (s, g) holds the chunk entries jb .. jb + cpitch - 1 at (3 s + g) * cpitch,
// followed by every matrix's nseg segment entries at 3 S cpitch + (3 s + g) nseg.
template <typename R, int S, int KIND>
__device__ __forceinline__ const typename V4T<R>::T *chunk_cache(const void *cache, int cpitch, int q) {
  int ms, mg;
  solve_matrix<R, S, KIND>(q, ms, mg);
  return reinterpret_cast<const typename V4T<R>::T *>(cache) + (3 * ms + mg) * cpitch;
}
template <typename R, int S, int KIND>
__device__ __forceinline__ const typename V4T<R>::T *segment_cache(const void *cache, int cpitch, int nseg, int q) {
  int ms, mg;
  solve_matrix<R, S, KIND>(q, ms, mg);
  return reinterpret_cast<const typename V4T<R>::T *>(cache) + 3 * S * cpitch + (3 * ms + mg) * nseg;
}

// ---- thread-block clusters (cluster-segmented sweeps)
// Split cluster barrier: arrive publishes this thread's shared-memory writes
// (release), wait returns once every thread of the cluster has arrived
// (acquire).  Hardware barriers: no spinning in software.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release;\n" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire;\n" ::: "memory"); }
__device__ __forceinline__ unsigned cluster_nranks() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;\n" : "=r"(r));
  return r;
}
// address of the same shared-memory object in block `rank` of the cluster
__device__ __forceinline__ unsigned dsmem_map(unsigned cta_addr, unsigned rank) {
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(cta_addr), "r"(rank));
  return r;
}
// a segment summary (G, X) from distributed shared memory
__device__ __forceinline__ void ld_dsmem_pair(unsigned a, float &g, float &x) {
  asm volatile("ld.shared::cluster.v2.f32 {%0, %1}, [%2];\n" : "=f"(g), "=f"(x) : "r"(a));
}
__device__ __forceinline__ void ld_dsmem_pair(unsigned a, double &g, double &x) {
  asm volatile("ld.shared::cluster.v2.f64 {%0, %1}, [%2];\n" : "=d"(g), "=d"(x) : "r"(a));
}
__device__ __forceinline__ void ld_dsmem_pair(unsigned a, float2 &g, float2 &x) {
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];\n"
               : "=f"(g.x), "=f"(g.y), "=f"(x.x), "=f"(x.y)
               : "r"(a));
}

// Zero-carry summary of one segment of one (line, solve) without touching
// F/Y: the forward value after the segment, G = sum_j (prod_{i>j} A_i) F_j,
// and the solution value at its first position with zero carries,
// X = sum_j (prod_{i<j} B_i) (Y_j + kappa_j G_in[j]) (chunk maps of the
// segment: forward G -> A G + F, backward X -> B X + Y + kappa G_in).  The
// loads of each batch of SB chunks are issued before its dependent FMAs
// (chunk tables and the exchange rows are padded to a multiple of 8).
template <typename R, typename V>
__device__ __forceinline__ void segment_summary(const MatTab<R> &M, const V *F, const V *Y, int m, int jb, V &Gout,
                                                V &Xout, const typename V4T<R>::T *cc = nullptr) {
  constexpr int SB = 4;
  V G = Splat<V>::of(R(0)), X = G;
  R pb = R(1);
  for (int j0 = 0; j0 < m; j0 += SB) {
    typename V4T<R>::T c[SB];
    V f[SB], y[SB];
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      c[k] = chunk_at(M, jb, cc, j0 + k);
      f[k] = F[j0 + k];
      y[k] = Y[j0 + k];
    }
#pragma unroll
    for (int k = 0; k < SB; ++k) {
      if (j0 + k < m) {
        const V yy = vfma(Splat<V>::of(c[k].y), G, y[k]);
        X = vfma(Splat<V>::of(pb), yy, X);
        pb *= c[k].z;
        G = vfma(Splat<V>::of(c[k].x), G, f[k]);
      }
    }
  }
  Gout = G;
  Xout = X;
}

// Cluster-segmented chaining of solves q0..q0+nq-1 (block = segment sc.seg
// of nlb lines; the cluster's blocks hold the line's other segments, block
// rank = segment).  Every (line, solve) unit publishes its zero-carry segment
// summary in shared memory; after a cluster barrier it reads the summaries of
// all segments, chains them with the segment coefficients (A_seg, K_seg,
// B_seg) into its forward carry G0, the solution value X0 after its segment
// and the line's first value and last forward value (Sherman-Morrison
// scalar), then runs its own chunk chain from (G0, X0).  Chunk and segment
// entries come from the block's table cache (see chunk_sweep).  The summary
// slots follow the Sherman-Morrison scalars; distinct solves use distinct slots,
// so the two exchanges of a LAST sweep never overwrite a slot still being
// read.  Barrier protocol per thread: [wait (closes the previous exchange's
// trailing arrive)] publish, arrive, wait, read + chain, arrive; the block's
// last wait (after its stores) keeps its shared memory alive until every
// block has finished reading it.
template <typename R, typename V, int PK, int S, int KIND>
__device__ __forceinline__ void scan_lines_cluster(const SweepArgs<R> &A, V *sF, V *sY, R *sSig, int q0, int nq,
                                                   const SegCtx &sc, const void *cache) {
  const int cpitch = A.pitch - 1;
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  constexpr int SB = 8;  // segment summaries requested per batch
  const int nlb = A.nlb, pitch = A.pitch;
  V *sSum = reinterpret_cast<V *>(reinterpret_cast<unsigned char *>(sSig) +
                                  ((NQ * nlb * PK * (int)sizeof(double) + 15) & ~15));
  // a launch whose cluster does not span the line's segments must not map
  // ranks it does not have: it reads no remote summary (and gives wrong
  // results, which the host never asks for)
  const int ns = ((int)cluster_nranks() == A.nseg) ? A.nseg : 1;
  if (q0 > 0) cluster_wait();
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    int ms, mg;
    solve_matrix<R, S, KIND>(q, ms, mg);
    V G, X;
    segment_summary<R, V>(A.mat[ms][mg], sF + (q * nlb + l) * pitch, sY + (q * nlb + l) * pitch, sc.mv, sc.jb, G,
                          X, chunk_cache<R, S, KIND>(cache, cpitch, q));
    sSum[2 * (q * nlb + l)] = G;
    sSum[2 * (q * nlb + l) + 1] = X;
  }
  cluster_arrive();
  cluster_wait();
  const V zero = Splat<V>::of(R(0));
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    int ms, mg;
    solve_matrix<R, S, KIND>(q, ms, mg);
    const MatTab<R> &M = A.mat[ms][mg];
    const typename V4T<R>::T *sgc = segment_cache<R, S, KIND>(cache, cpitch, A.nseg, q);
    const unsigned slot = (unsigned)__cvta_generic_to_shared(sSum + 2 * (q * nlb + l));
    V G = zero, G0 = zero, Xf = zero, Xa = zero;
    R pbf = R(1), pba = R(1);
    for (int k0 = 0; k0 < ns; k0 += SB) {
      V sg[SB], sx[SB];
#pragma unroll
      for (int k = 0; k < SB; ++k) {
        sg[k] = zero;
        sx[k] = zero;
        if (k0 + k < ns) ld_dsmem_pair(dsmem_map(slot, (unsigned)(k0 + k)), sg[k], sx[k]);
      }
#pragma unroll
      for (int k = 0; k < SB; ++k) {
        const int kk = k0 + k;
        if (kk < ns) {
          const typename V4T<R>::T c = ld_cc(sgc, kk);
          if (kk == sc.seg) G0 = G;
          const V y = vfma(Splat<V>::of(c.y), G, sx[k]);  // segment kk's first value minus B_seg X_after
          Xf = vfma(Splat<V>::of(pbf), y, Xf);
          pbf *= c.z;
          if (kk > sc.seg) {
            Xa = vfma(Splat<V>::of(pba), y, Xa);
            pba *= c.z;
          }
          G = vfma(Splat<V>::of(c.x), G, sg[k]);
        }
      }
    }
    put_sigma(sSig + (q * nlb + l) * PK, M, Xf, G);  // cyclic line: y_0 = Xf, y_{p-1} = G
    V Gd, Xd;
    chain_line_cc<R, V>(M, sF + (q * nlb + l) * pitch, sY + (q * nlb + l) * pitch, sc.mv, sc.jb, G0, Xa, Gd, Xd,
                        chunk_cache<R, S, KIND>(cache, cpitch, q));
  }
  cluster_arrive();
}

// Chain the chunk summaries of solves q0..q0+nq-1 for every line (or line
// pair) of the block.  sF/sY hold F_j / Y_j on entry and the carries G_in[j]
// / X[j+1] on return; sSig the Sherman-Morrison scalars.  Segmented sweeps:
// see SegCtx (segment summaries and carries are stored per line, pairs as two
// lines).
template <typename R, typename V, int PK, int S, int KIND, bool CL = false>
__device__ __forceinline__ void scan_lines(const SweepArgs<R> &A, V *sF, V *sY, R *sSig, int q0, int nq,
                                           const SegCtx &sc, const void *cache = nullptr) {
  const int nlb = A.nlb, pitch = A.pitch;
  if constexpr (CL) {  // cluster-segmented kernels (compiled separately)
    scan_lines_cluster<R, V, PK, S, KIND>(A, sF, sY, sSig, q0, nq, sc, cache);
    return;
  }
  if (sc.phase == SEG_WHOLE && A.mx > 32) {
    scan_lines_warp<R, V, PK>(A, sF, sY, sSig, q0, nq, [&](int q) -> const MatTab<R> & {
      int ms, mg;
      solve_matrix<R, S, KIND>(q, ms, mg);
      return A.mat[ms][mg];
    });
    return;
  }
  const V zero = Splat<V>::of(R(0));
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    int ms, mg;
    solve_matrix<R, S, KIND>(q, ms, mg);
    const MatTab<R> &M = A.mat[ms][mg];
    V *F = sF + (q * nlb + l) * pitch;  // shared-memory offsets in 32-bit arithmetic
    V *Y = sY + (q * nlb + l) * pitch;
    V G, X;
    if (sc.phase == SEG_WHOLE) {
      chain_line<R, V>(M, F, Y, sc.mv, 0, zero, zero, G, X);
      put_sigma(sSig + (q * nlb + l) * PK, M, X, G);  // cyclic line: y_0 = X, y_{p-1} = G
      continue;
    }
    const bool ok = l < sc.nvalid;
    const long long nl = A.nlines;
    V G0 = zero, X0 = zero;
    if (sc.phase == SEG_SOLVE && ok) {
#pragma unroll
      for (int k = 0; k < PK; ++k) {
        const long long gi = ((q * nl + sc.gl0 + (long long)l * PK + k) * A.nseg + sc.seg) * 2;
        v_set(G0, k, A.seg_car[gi]);
        v_set(X0, k, A.seg_car[gi + 1]);
        sSig[(q * nlb + l) * PK + k] = A.seg_sig[q * nl + sc.gl0 + (long long)l * PK + k];
      }
    }
    chain_line<R, V>(M, F, Y, sc.mv, sc.jb, G0, X0, G, X);
    if (sc.phase == SEG_SUMMARY && ok) {
#pragma unroll
      for (int k = 0; k < PK; ++k) {
        const long long gi = ((q * nl + sc.gl0 + (long long)l * PK + k) * A.nseg + sc.seg) * 2;
        A.seg_sum[gi] = v_get(G, k);
        A.seg_sum[gi + 1] = v_get(X, k);
      }
    }
  }
}

// Chains the segments of every line for solves q0 .. q0+nq-1: from the
// zero-carry summaries (F_seg, Y_seg) and the segment coefficients, the
// forward carry into each segment and the solution value after it, and the
// line's Sherman-Morrison scalar (FP64) from its first and last values.
template <typename R, int S, int KIND>
__global__ void seg_carry_kernel(const __grid_constant__ SweepArgs<R> A, int q0, int nq) {
  const long long nl = A.nlines;
  const int ns = A.nseg;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < nq * nl;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = q0 + (int)(idx / nl);
    const long long gl = idx - (long long)(q - q0) * nl;
    int ms, mg;
    solve_matrix<R, S, KIND>(q, ms, mg);
    const MatTab<R> &M = A.mat[ms][mg];
    const long long base = (q * nl + gl) * ns * 2;
    const R *sum = A.seg_sum + base;
    R *car = A.seg_car + base;
    R G = R(0);
    for (int k = 0; k < ns; ++k) {
      car[2 * k] = G;
      G = fma(ld_segc(M, k).x, G, sum[2 * k]);
    }
    R X = R(0);
    for (int k = ns - 1; k >= 0; --k) {
      const typename V4T<R>::T c = ld_segc(M, k);
      car[2 * k + 1] = X;
      X = fma(c.z, X, fma(c.y, car[2 * k], sum[2 * k + 1]));
    }
    put_sigma(A.seg_sig + q * nl + gl, M, X, G);
  }
}

// -------------------------------------------------------------- the sweep

// What one thread knows about its chunk of one line (or line pair).
template <typename R, int PK = 1>
struct ChunkPos {
  using V = typename LaneT<R, PK>::T;
  int l, j;      // line (pair) within the block/tile, chunk index within the block
  int jt;        // chunk index within the line (line tables; = j unless segmented)
  int i0, cnt;   // first position of the chunk, positions inside the line
  bool thr_ok;   // the thread owns a chunk (false for padding threads)
  V qbase;       // manufactured-source factor of the line(s) (0: none)
  SegCtx sc;     // where the block's chunks sit in their lines
};

// per-lane manufactured source p0 ((p1 lf - 1) q + q/(1+q)) at q = qbase phi_axis[i]
template <typename R>
__device__ __forceinline__ R source_of(const SweepArgs<R> &A, R q) {
  return A.rpR[0] * ((A.rpR[1] * A.src_lfR - R(1)) * q + rdiv(q, R(1) + q));
}

// Manufactured source at the L positions i0 .. i0+L-1 of a chunk of one line
// (PK = 1) or line pair (PK = 2): zero without a source and past the end of
// the line (cnt positions inside).  Full FP32 chunks read phi four at a time
// (chunk starts are multiples of 4, the phi tables 16-byte aligned).
template <typename R, int L, int PK>
__device__ __forceinline__ void chunk_sources(const SweepArgs<R> &A, typename LaneT<R, PK>::T qbase, int i0, int cnt,
                                              typename LaneT<R, PK>::T (&src)[L]) {
  using V = typename LaneT<R, PK>::T;
  const V zero = Splat<V>::of(R(0));
  if (!v_nonzero(qbase)) {
#pragma unroll
    for (int t = 0; t < L; ++t) src[t] = zero;
    return;
  }
  const R *phia = A.phi[A.axis] + i0;
  R ph[L];
  bool full = false;
  if constexpr (sizeof(R) == 4 && L % 4 == 0) {
    if (cnt == L) {
#pragma unroll
      for (int t = 0; t < L; t += 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(phia + t));
        ph[t] = q.x;
        ph[t + 1] = q.y;
        ph[t + 2] = q.z;
        ph[t + 3] = q.w;
      }
      full = true;
    }
  }
  if (!full) {
#pragma unroll
    for (int t = 0; t < L; ++t) ph[t] = (t < cnt) ? __ldg(phia + t) : R(0);
  }
#pragma unroll
  for (int t = 0; t < L; ++t) {
    if constexpr (PK == 1) src[t] = source_of(A, qbase * ph[t]);
    else src[t] = make_float2(source_of(A, qbase.x * ph[t]), source_of(A, qbase.y * ph[t]));
  }
  if (cnt < L) {
#pragma unroll
    for (int t = 0; t < L; ++t)
      if (t >= cnt) src[t] = zero;
  }
}

// One fused sweep of one block on register-resident chunks.  load(f, s, v)
// fills v with input field f (FIRST: 0 = U_n; MIDDLE/LAST: 0 = c_U, 1 = c_f,
// 2 = w) of species s, zero past the end of the line; store(f, s, v) writes
// output field f (FIRST/MIDDLE: c_U, c_f, w; LAST: 0 = U_{n+1}).  exch is the
// block's exchange space (chunk summaries, carries, Sherman-Morrison scalars).
// PK = 2: every value is a float2 holding a pair of neighbouring lines.
template <typename R, int S, int L, int KIND, int PK, bool CL = false, typename LoadF, typename StoreF>
__device__ __forceinline__ void chunk_sweep(const SweepArgs<R> &A, const ChunkPos<R, PK> &c, unsigned char *exch,
                                            LoadF load, StoreF store) {
  using V = typename LaneT<R, PK>::T;
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  const int l = c.l, j = c.j, jt = c.jt, cnt = c.cnt, i0 = c.i0;
  const bool thr_ok = c.thr_ok;
  const V zero = Splat<V>::of(R(0));
  auto react = [&](const V (&u)[S], V (&f)[S], V src) {
    if constexpr (PK == 1) {
      reaction_point<R, S>(A, u, f, src);
    } else {
      R ux[S], uy[S], fx[S], fy[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        ux[s] = u[s].x;
        uy[s] = u[s].y;
      }
      reaction_point<R, S>(A, ux, fx, src.x);
      reaction_point<R, S>(A, uy, fy, src.y);
#pragma unroll
      for (int s = 0; s < S; ++s) f[s] = make_float2(fx[s], fy[s]);
    }
  };
  auto p1 = [&](const MatTab<R> &M, const V (&b)[L], V &F, V &Y) {
    if constexpr (sizeof(R) == 8) pass1<R, L>(M, m, jt, b, F, Y);
    else pass1v<V, L>(M, m, jt, b, F, Y);
  };
  auto p1x2 = [&](const MatTab<R> &M, const V (&b0)[L], const V (&b1)[L], V &F0, V &Y0, V &F1, V &Y1) {
    if constexpr (sizeof(R) == 8) pass1x2<R, L>(M, m, jt, b0, b1, F0, Y0, F1, Y1);
    else pass1x2v<V, L>(M, m, jt, b0, b1, F0, Y0, F1, Y1);
  };
  V *sF = reinterpret_cast<V *>(exch);
  V *sY = sF + NQ * nlb * pitch;
  R *sSig = reinterpret_cast<R *>(exch + ((2 * NQ * nlb * pitch * (int)sizeof(V) + 15) & ~15));
  // Chunk-table cache (cluster-segmented sweeps): the chunk entries of this
  // block's chunks (jb .. jb + pitch - 2) of the 3 matrices of every species
  // and every matrix's segment entries, copied once at the start so that the
  // serial chains of the segment exchange read shared memory instead of
  // waiting on the global tables (blocks of other segments ran on the SM
  // before, so those entries are rarely in L1).  It follows the
  // Sherman-Morrison scalars and the cluster summaries, as sized by
  // sweep_smem_bytes.  Whole-line sweeps keep reading the global tables (their
  // chains are short and the copy cost more than it saved).
  using C4 = typename V4T<R>::T;
  auto cache_base = [&]() {  // recomputed where needed (keeps no pointer live across the sweep)
    return reinterpret_cast<C4 *>(reinterpret_cast<unsigned char *>(sSig) +
                                  ((NQ * nlb * PK * (int)sizeof(double) + 15) & ~15) +
                                  (CL ? ((2 * NQ * nlb * (int)sizeof(V) + 15) & ~15) : 0));
  };
  if constexpr (CL) {
    C4 *cch = cache_base();
    const int cpitch = pitch - 1;
    for (int idx = threadIdx.x; idx < 3 * S * cpitch; idx += blockDim.x) {
      const int mi = idx / cpitch;
      st_cc(cch, idx, ld_chunk(A.mat[mi / 3][mi % 3], c.sc.jb + (idx - mi * cpitch)));
    }
    C4 *csg = cch + 3 * S * cpitch;
    for (int idx = threadIdx.x; idx < 3 * S * A.nseg; idx += blockDim.x) {
      const int mi = idx / A.nseg;
      st_cc(csg, idx, ld_segc(A.mat[mi / 3][mi % 3], idx - mi * A.nseg));
    }
  }
  const int myidx = l * pitch + j;
  const int qstride = nlb * pitch;
  auto put = [&](int q, V F, V Y) {
    if (thr_ok) {
      sF[q * qstride + myidx] = F;
      sY[q * qstride + myidx] = Y;
    }
  };
  auto carries = [&](int q, V &Gin, V &Xr, V &sig) {
    Gin = sF[q * qstride + myidx];
    Xr = sY[q * qstride + myidx];
    sig = get_sigma(sSig + (q * nlb + l) * PK, zero);
  };
  auto carry = [&](int q) {  // FP32 form: ns = -sigma
    Carry<V> cq;
    V sg;
    carries(q, cq.G, cq.X, sg);
    cq.ns = vneg(sg);
    return cq;
  };
  const V k9 = Splat<V>::of(R(9)), km8 = Splat<V>::of(R(-8));
  auto scx = [&](int ph) {
    SegCtx x = c.sc;
    x.phase = ph;
    return x;
  };
  // solve q -> (species, matrix): FIRST/MIDDLE: q = 5s + {0: T.cU, 1: S.cU, 2: T.cf, 3: S.cf, 4: P.w}
  //                               LAST: q = s (P.w), S + 2s (T.f1), S + 2s + 1 (S.f2)
  if constexpr (KIND == SWEEP_FIRST || KIND == SWEEP_MIDDLE) {
    // FIRST keeps U_n and F(U_n) and forms w = U_n + k F(U_n) where a solve
    // reads it (one FMA per value instead of S*L live registers)
    constexpr bool WREG = (KIND == SWEEP_MIDDLE);
    V cu[S][L], cf[S][L], w[WREG ? S : 1][L];
    const V kk = Splat<V>::of(A.kR);
    auto wfirst = [&](int s, V (&o)[L]) {
#pragma unroll
      for (int t = 0; t < L; ++t) o[t] = vfma(kk, cf[s][t], cu[s][t]);
    };
    if constexpr (KIND == SWEEP_FIRST) {
      // U_n, F(U_n, t_n)
#pragma unroll
      for (int s = 0; s < S; ++s) load(0, s, cu[s]);
      V src[L];
      chunk_sources<R, L, PK>(A, c.qbase, i0, cnt, src);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        V u[S], f[S];
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = cu[s][t];
        react(u, f, src[t]);
#pragma unroll
        for (int s = 0; s < S; ++s) cf[s][t] = f[s];
      }
      if (cnt < L) {  // F = 0 past the end of the line
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
          for (int t = 0; t < L; ++t)
            if (t >= cnt) cf[s][t] = zero;
      }
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        load(0, s, cu[s]);
        load(1, s, cf[s]);
        load(2, s, w[s]);
      }
    }
    // pass 1: five solves per species share one exchange
#pragma unroll
    for (int s = 0; s < S; ++s) {
      V F0, Y0, F1, Y1;
      p1x2(A.mat[s][1], cu[s], cf[s], F0, Y0, F1, Y1);
      put(5 * s + 0, F0, Y0);
      put(5 * s + 2, F1, Y1);
      p1x2(A.mat[s][2], cu[s], cf[s], F0, Y0, F1, Y1);
      put(5 * s + 1, F0, Y0);
      put(5 * s + 3, F1, Y1);
      if constexpr (WREG) {
        p1(A.mat[s][0], w[s], F0, Y0);
      } else {
        V wt[L];
        wfirst(s, wt);
        p1(A.mat[s][0], wt, F0, Y0);
      }
      put(5 * s + 4, F0, Y0);
    }
    __syncthreads();
    scan_lines<R, V, PK, S, KIND, CL>(A, sF, sY, sSig, 0, NQ,
                                  scx(A.segphase == SEG_WHOLE || A.segphase == SEG_CLUSTER ? A.segphase
                                      : A.segphase == SEG_SUMMARY                           ? SEG_SUMMARY
                                                                                            : SEG_SOLVE),
                                  CL ? (const void *)cache_base() : nullptr);
    if (A.segphase == SEG_SUMMARY) return;  // segment summaries written
    __syncthreads();
    // pass 2: w <- P w (first: FIRST forms w from c_U, c_f before they are
    // overwritten), c_U <- 9 T c_U - 8 S c_U, c_f likewise
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if constexpr (sizeof(R) == 4) {
        if constexpr (WREG) {
          pass2v<V, L>(A.mat[s][0], m, jt, w[s], carry(5 * s + 4), w[s], [&](int t, V x) { w[s][t] = x; });
          store(2, s, w[s]);
        } else {
          V wt[L];
          wfirst(s, wt);
          pass2v<V, L>(A.mat[s][0], m, jt, wt, carry(5 * s + 4), wt, [&](int t, V x) { wt[t] = x; });
          store(2, s, wt);
        }
        // T on (c_U, c_f) into (xa, xc); S on (c_U, c_f) in place, folded into 9 T - 8 S
        V xa[L], xc[L];
        pass2x2v<V, L, true>(A.mat[s][1], A.mat[s][1], m, jt, cu[s], cf[s], carry(5 * s + 0), carry(5 * s + 2), xa,
                             xc, [&](int t, int k, V x) {
                               if (k == 0) xa[t] = x;
                               else xc[t] = x;
                             });
        pass2x2v<V, L, true>(A.mat[s][2], A.mat[s][2], m, jt, cu[s], cf[s], carry(5 * s + 1), carry(5 * s + 3),
                             cu[s], cf[s], [&](int t, int k, V x) {
                               if (k == 0) xa[t] = vfma(k9, xa[t], vmul(km8, x));
                               else xc[t] = vfma(k9, xc[t], vmul(km8, x));
                             });
        store(0, s, xa);
        store(1, s, xc);
      } else {
        V xa[L], xb[L], G, X, sg;
        carries(5 * s + 4, G, X, sg);
        if constexpr (WREG) {
          pass2<R, L>(A.mat[s][0], m, jt, w[s], G, X, sg, xa);
        } else {
          wfirst(s, xb);
          pass2<R, L>(A.mat[s][0], m, jt, xb, G, X, sg, xa);
        }
        store(2, s, xa);
        carries(5 * s + 0, G, X, sg);
        pass2<R, L>(A.mat[s][1], m, jt, cu[s], G, X, sg, xa);
        carries(5 * s + 1, G, X, sg);
        pass2<R, L>(A.mat[s][2], m, jt, cu[s], G, X, sg, xb);
#pragma unroll
        for (int t = 0; t < L; ++t) xa[t] = vfma(k9, xa[t], vmul(km8, xb[t]));
        store(0, s, xa);
        carries(5 * s + 2, G, X, sg);
        pass2<R, L>(A.mat[s][1], m, jt, cf[s], G, X, sg, xa);
        carries(5 * s + 3, G, X, sg);
        pass2<R, L>(A.mat[s][2], m, jt, cf[s], G, X, sg, xb);
#pragma unroll
        for (int t = 0; t < L; ++t) xa[t] = vfma(k9, xa[t], vmul(km8, xb[t]));
        store(1, s, xa);
      }
    }
  } else {
    // LAST: phase A  U* = P_d w ; phase B  U_{n+1} = T_d f1 - S_d f2
    // c_U and c_f are read once U* is known (fewer live registers in phase A)
    V cu[S][L], cf[S][L], w[S][L];
#pragma unroll
    for (int s = 0; s < S; ++s) load(2, s, w[s]);
#pragma unroll
    for (int s = 0; s < S; ++s) {
      V F0, Y0;
      p1(A.mat[s][0], w[s], F0, Y0);
      put(s, F0, Y0);
    }
    __syncthreads();
    scan_lines<R, V, PK, S, KIND, CL>(A, sF, sY, sSig, 0, S,
                                  scx(A.segphase == SEG_WHOLE || A.segphase == SEG_CLUSTER ? A.segphase
                                      : A.segphase == SEG_SUMMARY                           ? SEG_SUMMARY
                                                                                            : SEG_SOLVE),
                                  CL ? (const void *)cache_base() : nullptr);
    if (A.segphase == SEG_SUMMARY) return;  // P summaries written
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if constexpr (sizeof(R) == 4) {
        pass2v<V, L>(A.mat[s][0], m, jt, w[s], carry(s), w[s], [&](int t, V x) { w[s][t] = x; });  // w <- U*
      } else {
        V x[L], G, X, sg;
        carries(s, G, X, sg);
        pass2<R, L>(A.mat[s][0], m, jt, w[s], G, X, sg, x);
#pragma unroll
        for (int t = 0; t < L; ++t) w[s][t] = x[t];  // w now holds U*
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      load(0, s, cu[s]);
      load(1, s, cf[s]);
    }
    // F(U*, t_{n+1}); f1, f2 overwrite c_U, c_f
    const R k = A.kR;
    const V k2 = Splat<V>::of(R(2) * k), kk = Splat<V>::of(k), k15 = Splat<V>::of(R(1.5) * k),
            k05 = Splat<V>::of(R(0.5) * k), k8 = Splat<V>::of(R(8));
    V src[L];
    chunk_sources<R, L, PK>(A, c.qbase, i0, cnt, src);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      V u[S], f[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = w[s][t];
      react(u, f, src[t]);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const V fs = (cnt == L || t < cnt) ? f[s] : zero;
        const V a = cu[s][t], b = cf[s][t];
        cu[s][t] = vfma(k9, a, vfma(k2, b, vmul(kk, fs)));
        cf[s][t] = vfma(k8, a, vfma(k15, b, vmul(k05, fs)));
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      V F0, Y0, F1, Y1;
      p1(A.mat[s][1], cu[s], F0, Y0);
      p1(A.mat[s][2], cf[s], F1, Y1);
      put(S + 2 * s, F0, Y0);
      put(S + 2 * s + 1, F1, Y1);
    }
    __syncthreads();
    scan_lines<R, V, PK, S, KIND, CL>(A, sF, sY, sSig, S, 2 * S,
                                  scx(A.segphase == SEG_WHOLE || A.segphase == SEG_CLUSTER ? A.segphase
                                      : A.segphase == SEG_SOLVE                             ? SEG_SUMMARY
                                                                                            : SEG_SOLVE),
                                  CL ? (const void *)cache_base() : nullptr);
    if (A.segphase == SEG_SOLVE) return;  // T and S summaries written
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if constexpr (sizeof(R) == 4) {
        // T f1 and S f2 interleaved in place; c_U <- T f1 - S f2
        pass2x2v<V, L, false>(A.mat[s][1], A.mat[s][2], m, jt, cu[s], cf[s], carry(S + 2 * s), carry(S + 2 * s + 1),
                              cu[s], cf[s], [&](int t, int k, V x) {
                                if (k == 0) cu[s][t] = x;
                                else cu[s][t] = vsub(cu[s][t], x);
                              });
        store(0, s, cu[s]);
      } else {
        V xa[L], xb[L], G, X, sg;
        carries(S + 2 * s, G, X, sg);
        pass2<R, L>(A.mat[s][1], m, jt, cu[s], G, X, sg, xa);
        carries(S + 2 * s + 1, G, X, sg);
        pass2<R, L>(A.mat[s][2], m, jt, cf[s], G, X, sg, xb);
#pragma unroll
        for (int t = 0; t < L; ++t) xa[t] = vsub(xa[t], xb[t]);
        store(0, s, xa);
      }
    }
  }
}

// ---- circulant line solves of periodic axes (symmetric M: M^T = M), the
// factorisation of the forward circulant sweeps: pass 1 gives the chunk's
// zero-carry summaries F (forward value at its end) and W = sum_t lambda^t ytilde_t;
// one thread per (line, solve) chains the m chunks of its line (cyclic
// closures by 1/(1 - lambda^p)) and leaves the carries Yc_j (y before chunk j)
// and Zc_j (z after it) in place of F_j, W_j; pass 2 runs both recurrences.
template <typename R, int L>
__device__ __forceinline__ void cpass1(const typename SweepArgs<R>::CircLine &M, const R (&b)[L], R &F, R &Wv) {
  R y = R(0), w = R(0);
#pragma unroll
  for (int t = 0; t < L; ++t) {
    y = fma(M.lam, y, b[t]);
    w = fma(M.pw[t], y, w);
  }
  F = y;
  Wv = w;
}
template <typename R, int L>
__device__ __forceinline__ void cpass2(const typename SweepArgs<R>::CircLine &M, const R (&b)[L], R Yc, R Zc,
                                       R (&x)[L]) {
  R y = Yc;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    y = fma(M.lam, y, b[t]);
    x[t] = y;
  }
  R z = Zc;
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    z = fma(M.lam, z, x[t]);
    x[t] = z * M.ialpha;
  }
}
template <typename R, typename CIdx>
__device__ __forceinline__ void circ_chains(const SweepArgs<R> &A, R *sF, R *sY, int q0, int nq, CIdx cidx) {
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    const int ci = cidx(q);
    const typename SweepArgs<R>::CircLine &M = A.cl[ci / 3][ci % 3];
    R *F = sF + (q * nlb + l) * pitch;
    R *Y = sY + (q * nlb + l) * pitch;
    R t = R(0);
    for (int j = 0; j < m; ++j) t = fma(M.lamL, t, F[j]);
    R y = t * M.inv1m;  // y entering chunk 0 (cyclic)
    for (int j = 0; j < m; ++j) {
      const R f = F[j];
      F[j] = y;
      y = fma(M.lamL, y, f);
    }
    R g = R(0);
    for (int j = m - 1; j >= 0; --j) {
      const R gj = fma(M.kap, F[j], Y[j]);  // backward value at the chunk start with its forward carry
      Y[j] = gj;
      g = fma(M.lamL, g, gj);
    }
    R z = g * M.inv1m;  // z after the last chunk (cyclic)
    for (int j = m - 1; j >= 0; --j) {
      const R gj = Y[j];
      Y[j] = z;
      z = fma(M.lamL, z, gj);
    }
  }
}

// Whole-line sweep of a periodic axis on the circulant factorisation (the
// ensemble's periodic instances; lines of whole chunks): the same solves and
// combinations as chunk_sweep, with constant-coefficient passes and the line
// chains of circ_chains instead of the line tables.
template <typename R, int S, int L, int KIND, typename LoadF, typename StoreF>
__device__ __forceinline__ void circ_chunk_sweep(const SweepArgs<R> &A, const ChunkPos<R, 1> &c, unsigned char *exch,
                                                 LoadF load, StoreF store) {
  using CL_ = typename SweepArgs<R>::CircLine;
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  const int nlb = A.nlb, pitch = A.pitch;
  const int myidx = c.l * pitch + c.j, qstride = nlb * pitch;
  R *sF = reinterpret_cast<R *>(exch);
  R *sY = sF + NQ * nlb * pitch;
  auto p1 = [&](int q, const CL_ &M, const R (&b)[L]) {
    R F, W;
    cpass1<R, L>(M, b, F, W);
    if (c.thr_ok) {
      sF[q * qstride + myidx] = F;
      sY[q * qstride + myidx] = W;
    }
  };
  auto p2 = [&](int q, const CL_ &M, const R (&b)[L], R (&x)[L]) {
    cpass2<R, L>(M, b, sF[q * qstride + myidx], sY[q * qstride + myidx], x);
  };
  auto react = [&](const R (&u)[S], R (&f)[S], R src) { reaction_point<R, S>(A, u, f, src); };
  R src[L];
  chunk_sources<R, L, 1>(A, c.qbase, c.i0, c.cnt, src);
  if constexpr (KIND == SWEEP_FIRST || KIND == SWEEP_MIDDLE) {
    // q = 5s + {0: T c_U, 1: S c_U, 2: T c_f, 3: S c_f, 4: P w}
    auto cid = [](int q) { const int r = q % 5; return (q / 5) * 3 + (r == 4 ? 0 : 1 + (r & 1)); };
    R cu[S][L], cf[S][L], w[KIND == SWEEP_MIDDLE ? S : 1][L];
    const R k = A.kR;
    if constexpr (KIND == SWEEP_FIRST) {
#pragma unroll
      for (int s = 0; s < S; ++s) load(0, s, cu[s]);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], f[S];
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = cu[s][t];
        react(u, f, src[t]);
#pragma unroll
        for (int s = 0; s < S; ++s) cf[s][t] = f[s];
      }
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        load(0, s, cu[s]);
        load(1, s, cf[s]);
        load(2, s, w[s]);
      }
    }
    auto wof = [&](int s, R (&o)[L]) {  // the P right-hand side
#pragma unroll
      for (int t = 0; t < L; ++t) {
        if constexpr (KIND == SWEEP_MIDDLE) o[t] = w[s][t];
        else o[t] = fma(k, cf[s][t], cu[s][t]);
      }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) {
      p1(5 * s + 0, A.cl[s][1], cu[s]);
      p1(5 * s + 1, A.cl[s][2], cu[s]);
      p1(5 * s + 2, A.cl[s][1], cf[s]);
      p1(5 * s + 3, A.cl[s][2], cf[s]);
      R wt[L];
      wof(s, wt);
      p1(5 * s + 4, A.cl[s][0], wt);
    }
    __syncthreads();
    circ_chains<R>(A, sF, sY, 0, NQ, cid);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R wt[L], xa[L], xb[L];
      wof(s, wt);
      p2(5 * s + 4, A.cl[s][0], wt, xa);
      store(2, s, xa);
      p2(5 * s + 0, A.cl[s][1], cu[s], xa);
      p2(5 * s + 1, A.cl[s][2], cu[s], xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] = fma(R(9), xa[t], R(-8) * xb[t]);
      store(0, s, xa);
      p2(5 * s + 2, A.cl[s][1], cf[s], xa);
      p2(5 * s + 3, A.cl[s][2], cf[s], xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] = fma(R(9), xa[t], R(-8) * xb[t]);
      store(1, s, xa);
    }
  } else {
    // q = s (P w), S + 2s (T f1), S + 2s + 1 (S f2)
    auto cid = [](int q) {
      if (q < S) return q * 3;
      const int r = q - S;
      return (r / 2) * 3 + 1 + (r & 1);
    };
    R w[S][L];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      load(2, s, w[s]);
      p1(s, A.cl[s][0], w[s]);
    }
    __syncthreads();
    circ_chains<R>(A, sF, sY, 0, S, cid);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) p2(s, A.cl[s][0], w[s], w[s]);  // U*
    R cu[S][L], cf[S][L];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      load(0, s, cu[s]);
      load(1, s, cf[s]);
    }
    const R k = A.kR;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      R u[S], f[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = w[s][t];
      react(u, f, src[t]);
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const R a = cu[s][t], b = cf[s][t];
        cu[s][t] = fma(R(9), a, fma(R(2) * k, b, k * f[s]));
        cf[s][t] = fma(R(8), a, fma(R(1.5) * k, b, R(0.5) * k * f[s]));
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      p1(S + 2 * s, A.cl[s][1], cu[s]);
      p1(S + 2 * s + 1, A.cl[s][2], cf[s]);
    }
    __syncthreads();
    circ_chains<R>(A, sF, sY, S, 2 * S, cid);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R xa[L], xb[L];
      p2(S + 2 * s, A.cl[s][1], cu[s], xa);
      p2(S + 2 * s + 1, A.cl[s][2], cf[s], xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] = xa[t] - xb[t];
      store(0, s, xa);
    }
  }
}

// line pairs: L positions of two neighbouring lines, 8-byte loads (st2 = stride in pairs)
template <int L>
__device__ __forceinline__ void load_pairs(float2 (&v)[L], const float2 *__restrict__ p, int st2, int cnt) {
  if (cnt == L) {
#pragma unroll
    for (int t = 0; t < L; ++t) v[t] = __ldg(p + t * st2);
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t) v[t] = (t < cnt) ? __ldg(p + t * st2) : make_float2(0.f, 0.f);
  }
}

template <int L>
__device__ __forceinline__ void store_pairs(const float2 (&v)[L], float2 *__restrict__ p, int st2, int cnt) {
  if (cnt == L) {
#pragma unroll
    for (int t = 0; t < L; ++t) p[t * st2] = v[t];
  } else {
#pragma unroll
    for (int t = 0; t < L; ++t)
      if (t < cnt) p[t * st2] = v[t];
  }
}

// Register kernel: one block per group of nlb lines (nlb line pairs for
// PK = 2) and, for segmented sweeps, per segment of mx chunks of those lines;
// inputs loaded straight from global memory (vector loads on x, coalesced row
// segments on strided axes).
// COH: inputs may have been written earlier in the same launch (coherent loads)
// CIRCF: periodic whole-chunk lines on the circulant factorisation (circ_chunk_sweep)
template <typename R, int S, int L, bool CONTIG, int KIND, int PK = 1, bool CL = false, bool COH = false,
          bool CIRCF = false>
__device__ __forceinline__ void sweep_block(const SweepArgs<R> &A, int bid, unsigned char *smem, double t_eval,
                                            R exp_mt) {
  (void)t_eval;
  const int m = A.m, mx = A.mx, nlb = A.nlb, nseg = A.nseg;
  const int seg = bid % nseg;
  const int lb = bid / nseg;  // line block
  const int tid = threadIdx.x;
  // threads past nlb*mx (batched launches size blocks for the largest
  // instance) own no chunk but still take part in every barrier and scan
  const bool thr_ok = tid < nlb * mx;
  int l = tid % nlb, j = tid / nlb;
  if (!thr_ok) { l = 0; j = 0; }
  const int jg = seg * mx + j;  // chunk within the line
  const bool chunk_in = jg < m;
  SegCtx sc;
  sc.phase = SEG_WHOLE;
  sc.seg = seg;
  sc.jb = seg * mx;
  sc.mv = min(mx, m - seg * mx);
  const long long N = A.N;
  if constexpr (PK == 2) {
    // strided axis, even stride: pair l covers lines lo, lo + 1 of one row
    static_assert(!CONTIG && sizeof(R) == 4, "line pairs: FP32 strided sweeps");
    static_assert(!COH, "line pairs: read-only inputs");
    const long long lo0 = (long long)(lb % A.nlo_blocks) * nlb * 2;
    const long long lo = lo0 + 2 * l;
    const long long hi = lb / A.nlo_blocks;
    const bool line_ok = thr_ok && lo < A.st;
    sc.gl0 = hi * A.st + lo0;
    sc.nvalid = (int)min((long long)nlb, (A.st - lo0) / 2);
    ChunkPos<R, 2> c;
    c.qbase = line_ok ? make_float2(line_source_base(A, false, 0, lo, hi, exp_mt),
                                    line_source_base(A, false, 0, lo + 1, hi, exp_mt))
                      : make_float2(0.f, 0.f);
    c.l = l;
    c.j = j;
    c.jt = chunk_in ? jg : m - 1;
    c.i0 = jg * L;
    c.cnt = (line_ok && chunk_in) ? max(0, min(L, A.n - c.i0)) : 0;
    c.thr_ok = thr_ok;
    c.sc = sc;
    const long long off0 = (lo + hi * A.st * A.n + (long long)c.i0 * A.st) >> 1;  // in pairs
    const int st2 = (int)(A.st >> 1);
    const int cnt = c.cnt;
    auto load = [&](int f, int s, float2 (&v)[L]) {
      load_pairs<L>(v, reinterpret_cast<const float2 *>(A.in[f] + s * N) + off0, st2, cnt);
    };
    auto store = [&](int f, int s, const float2 (&v)[L]) {
      store_pairs<L>(v, reinterpret_cast<float2 *>(A.out[f] + s * N) + off0, st2, cnt);
    };
    chunk_sweep<R, S, L, KIND, 2, CL>(A, c, smem, load, store);
  } else {
    long long base;
    bool line_ok;
    ChunkPos<R> c;
    if constexpr (CONTIG) {
      const long long line0 = (long long)lb * nlb;
      const long long line = line0 + l;
      line_ok = thr_ok && line < A.nlines;
      base = line * A.n;
      c.qbase = line_ok ? line_source_base(A, true, line, 0, 0, exp_mt) : R(0);
      sc.gl0 = line0;
      sc.nvalid = (int)min((long long)nlb, A.nlines - line0);
    } else {
      const long long lo0 = (long long)(lb % A.nlo_blocks) * nlb;
      const long long lo = lo0 + l;
      const long long hi = lb / A.nlo_blocks;
      line_ok = thr_ok && lo < A.st;
      base = lo + hi * A.st * A.n;
      c.qbase = line_ok ? line_source_base(A, false, 0, lo, hi, exp_mt) : R(0);
      sc.gl0 = hi * A.st + lo0;
      sc.nvalid = (int)min((long long)nlb, A.st - lo0);
    }
    const long long st = CONTIG ? 1 : A.st;
    c.l = l;
    c.j = j;
    c.jt = chunk_in ? jg : m - 1;
    c.i0 = jg * L;
    c.cnt = (line_ok && chunk_in) ? max(0, min(L, A.n - c.i0)) : 0;
    c.thr_ok = thr_ok;
    c.sc = sc;
    const long long off0 = base + (long long)c.i0 * st;
    const int cnt = c.cnt;
    auto load = [&](int f, int s, R (&v)[L]) { load_chunk<R, L, CONTIG, COH>(v, A.in[f] + s * N, off0, st, cnt); };
    auto store = [&](int f, int s, const R (&v)[L]) {
      store_chunk<R, L, CONTIG>(v, A.out[f] + s * N, off0, st, cnt);
    };
    if constexpr (CIRCF) circ_chunk_sweep<R, S, L, KIND>(A, c, smem, load, store);
    else chunk_sweep<R, S, L, KIND, 1, CL>(A, c, smem, load, store);
  }
}

// CL: cluster-segmented (launched with nseg-block clusters, A.segphase = SEG_CLUSTER)
template <typename R, int S, int L, bool CONTIG, int KIND, int PK = 1, bool CL = false>
__global__ void __launch_bounds__(ETD_MAX_THREADS) sweep_kernel(const __grid_constant__ SweepArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  sweep_block<R, S, L, CONTIG, KIND, PK, CL>(A, blockIdx.x, smem, A.t_eval, A.exp_mtR);
  // the other blocks of the cluster may still read this block's summaries
  if constexpr (CL) cluster_wait();
}

// Batched ensemble: one launch covers every instance; block b belongs to the
// instance i with block_start[i] <= b < block_start[i+1].
template <typename R, int S, int L, bool CONTIG, int KIND>
__global__ void __launch_bounds__(ETD_MAX_THREADS) sweep_kernel_batched(const SweepArgs<R> *__restrict__ args,
                                                              const int *__restrict__ block_start, int ninst,
                                                              double t_eval, R exp_mt) {
  extern __shared__ __align__(16) unsigned char smem[];
  int lo = 0, hi = ninst - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (block_start[mid] <= b) lo = mid; else hi = mid - 1;
  }
  sweep_block<R, S, L, CONTIG, KIND>(args[lo], b - block_start[lo], smem, t_eval, exp_mt);
}

}  // namespace etd
