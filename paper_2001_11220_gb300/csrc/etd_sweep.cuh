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
// Thread mapping: contiguous axis (x): lanes walk the chunks of a line
// (j = tid % m) and load L consecutive elements with vector loads; strided
// axes: lanes walk neighbouring lines (l = tid % nlb) so every load of
// position i is one coalesced row segment across the warp.
#pragma once

#include "etd_internal.h"

namespace etd {

#ifndef ETD_MAX_THREADS
#define ETD_MAX_THREADS 512
#endif

template <typename R>
__device__ __forceinline__ R ld_nc(const R *p) { return __ldg(p); }

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
      for (int s = 0; s < S; ++s) f[s] = fma((R)A.rp[0], u[s], (R)A.rp[1]);
      return;
    case 2:
      if constexpr (S == 2) {  // Brusselator: a + u^2 v - (b+1) u ; b u - u^2 v
        const R a = (R)A.rp[0], b = (R)A.rp[1];
        const R uuv = u[0] * u[0] * u[1];
        f[0] = a + uuv - (b + R(1)) * u[0];
        f[1] = b * u[0] - uuv;
        return;
      }
      break;
    case 3:
      if constexpr (S == 2) {  // Schnakenberg: g (a - u + u^2 v) ; g (b - u^2 v)
        const R a = (R)A.rp[0], b = (R)A.rp[1], g = (R)A.rp[2];
        const R uuv = u[0] * u[0] * u[1];
        f[0] = g * (a - u[0] + uuv);
        f[1] = g * (b - uuv);
        return;
      }
      break;
    case 4:
      if constexpr (S == 2) {  // Gray-Scott: -u v^2 + F (1-u) ; u v^2 - (F+kappa) v
        const R F = (R)A.rp[0], kap = (R)A.rp[1];
        const R uvv = u[0] * u[1] * u[1];
        f[0] = F * (R(1) - u[0]) - uvv;
        f[1] = uvv - (F + kap) * u[1];
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

// manufactured source p0 ((p1 lf - 1) q + q/(1+q)), q = e^{-t} prod sin(pi x_a/L_a)
template <typename R>
__device__ __forceinline__ R mms_source(const SweepArgs<R> &A, long long pidx, double exp_mt) {
  const long long x = pidx % A.nx;
  const long long r = pidx / A.nx;
  const long long y = r % A.ny;
  const long long z = r / A.ny;
  R q = (R)exp_mt * A.phi[0][x] * A.phi[1][y];
  if (A.phi[2]) q *= A.phi[2][z];
  return (R)A.rp[0] * (((R)A.rp[1] * (R)A.src_lf - R(1)) * q + rdiv(q, R(1) + q));
}

// e^{-t} prod_{b != axis} sin(pi x_b / L_b) for one line: x axis line index
// (y + z ny), strided axes (lo, hi) line coordinates; 0 without a source
template <typename R>
__device__ __forceinline__ R line_source_base(const SweepArgs<R> &A, bool contig, long long line, long long lo,
                                              long long hi, double exp_mt) {
  if (A.phi[0] == nullptr) return R(0);
  R q = (R)exp_mt;
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

template <typename R, int L, bool CONTIG>
__device__ __forceinline__ void load_chunk(R (&v)[L], const R *__restrict__ p, long long off, long long st,
                                           int cnt) {
  if constexpr (CONTIG) {
    constexpr int VW = 16 / sizeof(R);
    if (L % VW == 0 && cnt == L && ((reinterpret_cast<uintptr_t>(p + off) & 15) == 0)) {
      using V4 = typename V4T<R>::T;
      (void)sizeof(V4);
      if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int t = 0; t < L; t += 4) {
          float4 q = __ldg(reinterpret_cast<const float4 *>(p + off + t));
          v[t] = q.x; v[t + 1] = q.y; v[t + 2] = q.z; v[t + 3] = q.w;
        }
      } else {
#pragma unroll
        for (int t = 0; t < L; t += 2) {
          double2 q = __ldg(reinterpret_cast<const double2 *>(p + off + t));
          v[t] = q.x; v[t + 1] = q.y;
        }
      }
      return;
    }
  }
#pragma unroll
  for (int t = 0; t < L; ++t) v[t] = (t < cnt) ? ld_nc(p + off + (long long)t * st) : R(0);
}

template <typename R, int L, bool CONTIG>
__device__ __forceinline__ void store_chunk(const R (&v)[L], R *__restrict__ p, long long off, long long st,
                                            int cnt) {
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
#pragma unroll
  for (int t = 0; t < L; ++t)
    if (t < cnt) p[off + (long long)t * st] = v[t];
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

// --------------------------------------------------------------- scan

// Chain the chunk summaries of solves q0..q0+nq-1 for every line of the
// block.  sF/sY hold F_j / Y_j on entry and the carries G_in[j] / X[j+1] on
// return; sSig the FP64 Sherman-Morrison scalar per (solve, line).
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


// Long lines (m > 32 chunks): one warp per (line, solve).  Each lane composes
// the affine chunk maps of a contiguous block of chunks, a shuffle scan over
// the lanes gives every block its carries, and the lane re-walks its block to
// emit G_in[j] and X[j+1] (forward map G -> Aend G + F, backward map
// X -> Bst X + Y + kappa G_in).
template <typename R, typename GetMat>
__device__ __forceinline__ void scan_lines_warp(const SweepArgs<R> &A, R *sF, R *sY, double *sSig, int q0, int nq,
                                                GetMat mat) {
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  // full warps only: a trailing partial warp (blockDim not a multiple of 32) stays out of the shuffles
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (warp >= nw) return;
  const int per = (m + 31) >> 5;
  const int j0 = min(lane * per, m), j1 = min(j0 + per, m);
  for (int u = warp; u < nlb * nq; u += nw) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    const MatTab<R> &M = mat(q);
    R *F = sF + (size_t)q * nlb * pitch + (size_t)l * pitch;
    R *Y = sY + (size_t)q * nlb * pitch + (size_t)l * pitch;
    // forward: block map G_out = a G_in + b
    R a = R(1), b = R(0);
    for (int jj = j0; jj < j1; ++jj) {
      const R Aj = M.chunk[jj].x;
      b = fma(Aj, b, F[jj]);
      a *= Aj;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const R ap = __shfl_up_sync(0xffffffffu, a, off), bp = __shfl_up_sync(0xffffffffu, b, off);
      if (lane >= off) {
        b = fma(a, bp, b);
        a *= ap;
      }
    }
    R G = __shfl_up_sync(0xffffffffu, b, 1);
    if (lane == 0) G = R(0);
    const R Gtot = __shfl_sync(0xffffffffu, b, 31);  // forward value at the last position
    for (int jj = j0; jj < j1; ++jj) {
      const typename V4T<R>::T c = M.chunk[jj];
      const R f = F[jj];
      F[jj] = G;
      Y[jj] = fma(c.y, G, Y[jj]);
      G = fma(c.x, G, f);
    }
    // backward: block map X_out = a X_in + b, composed from the right
    a = R(1);
    b = R(0);
    for (int jj = j1 - 1; jj >= j0; --jj) {
      const R Bj = M.chunk[jj].z;
      b = fma(Bj, b, Y[jj]);
      a *= Bj;
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
      const R an = __shfl_down_sync(0xffffffffu, a, off), bn = __shfl_down_sync(0xffffffffu, b, off);
      if (lane + off < 32) {
        b = fma(a, bn, b);
        a *= an;
      }
    }
    R X = __shfl_down_sync(0xffffffffu, b, 1);
    if (lane == 31) X = R(0);
    for (int jj = j1 - 1; jj >= j0; --jj) {
      const R yv = Y[jj];
      Y[jj] = X;
      X = fma(M.chunk[jj].z, X, yv);
    }
    const R X0 = __shfl_sync(0xffffffffu, X, 0);  // first position of the line
    if (lane == 0)
      sSig[(size_t)q * nlb + l] = (M.sm_inv != 0.0) ? ((double)X0 + M.sm_c * (double)Gtot) * M.sm_inv : 0.0;
  }
}

template <typename R, int S, int KIND>
__device__ __forceinline__ void scan_lines(const SweepArgs<R> &A, R *sF, R *sY, double *sSig, int q0, int nq,
                                           bool periodic) {
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  if (m > 32) {
    scan_lines_warp<R>(A, sF, sY, sSig, q0, nq, [&](int q) -> const MatTab<R> & {
      int ms, mg;
      solve_matrix<R, S, KIND>(q, ms, mg);
      return A.mat[ms][mg];
    });
    return;
  }
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    int ms, mg;
    solve_matrix<R, S, KIND>(q, ms, mg);
    const MatTab<R> &M = A.mat[ms][mg];
    R *F = sF + (size_t)q * nlb * pitch + (size_t)l * pitch;
    R *Y = sY + (size_t)q * nlb * pitch + (size_t)l * pitch;
    R G = R(0);
#pragma unroll 8
    for (int j = 0; j < m; ++j) {
      const R f = F[j];
      F[j] = G;
      G = fma(M.chunk[j].x, G, f);
    }
    R X = R(0);
#pragma unroll 8
    for (int j = m - 1; j >= 0; --j) {
      const typename V4T<R>::T c = M.chunk[j];
      const R y = fma(c.y, F[j], Y[j]);
      Y[j] = X;
      X = fma(c.z, X, y);
    }
    // cyclic line: y_0 = X, y_{p-1} = G; sigma = (v . y) / (1 + v . z) in FP64
    sSig[(size_t)q * nlb + l] = periodic ? ((double)X + M.sm_c * (double)G) * M.sm_inv : 0.0;
  }
}

// -------------------------------------------------------------- the sweep

// What one thread knows about its chunk of one line.
template <typename R>
struct ChunkPos {
  int l, j;      // line within the block/tile, chunk index
  int i0, cnt;   // first position of the chunk, positions inside the line
  bool thr_ok;   // the thread owns a chunk (false for padding threads)
  R qbase;       // manufactured-source factor of the line (0: none)
};

// One fused sweep of one block on register-resident chunks.  load(f, s, v)
// fills v with input field f (FIRST: 0 = U_n; MIDDLE/LAST: 0 = c_U, 1 = c_f,
// 2 = w) of species s, zero past the end of the line; store(f, s, v) writes
// output field f (FIRST/MIDDLE: c_U, c_f, w; LAST: 0 = U_{n+1}).  exch is the
// block's exchange space (chunk summaries, carries, Sherman-Morrison scalars).
template <typename R, int S, int L, int KIND, typename LoadF, typename StoreF>
__device__ __forceinline__ void chunk_sweep(const SweepArgs<R> &A, const ChunkPos<R> &c, unsigned char *exch,
                                            LoadF load, StoreF store) {
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  const int l = c.l, j = c.j, cnt = c.cnt, i0 = c.i0;
  const bool thr_ok = c.thr_ok;
  const bool periodic = A.mat[0][0].sm_inv != 0.0;
  const R qbase = c.qbase;
  const R *phia = A.phi[A.axis];
  auto src_at = [&](int t) -> R {  // manufactured source at position t of the chunk
    if (qbase == R(0) || t >= cnt) return R(0);
    const R q = qbase * phia[i0 + t];
    return (R)A.rp[0] * (((R)A.rp[1] * (R)A.src_lf - R(1)) * q + rdiv(q, R(1) + q));
  };
  R *sF = reinterpret_cast<R *>(exch);
  R *sY = sF + (size_t)NQ * nlb * pitch;
  double *sSig = reinterpret_cast<double *>(exch + ((2 * (size_t)NQ * nlb * pitch * sizeof(R) + 15) & ~(size_t)15));
  const size_t myidx = (size_t)l * pitch + j;
  auto put = [&](int q, R F, R Y) {
    if (thr_ok) {
      sF[(size_t)q * nlb * pitch + myidx] = F;
      sY[(size_t)q * nlb * pitch + myidx] = Y;
    }
  };
  auto carries = [&](int q, R &Gin, R &Xr, R &sig) {
    Gin = sF[(size_t)q * nlb * pitch + myidx];
    Xr = sY[(size_t)q * nlb * pitch + myidx];
    sig = (R)sSig[(size_t)q * nlb + l];
  };
  // solve q -> (species, matrix): FIRST/MIDDLE: q = 5s + {0: T.cU, 1: S.cU, 2: T.cf, 3: S.cf, 4: P.w}
  //                               LAST: q = s (P.w), S + 2s (T.f1), S + 2s + 1 (S.f2)
  if constexpr (KIND == SWEEP_FIRST || KIND == SWEEP_MIDDLE) {
    R cu[S][L], cf[S][L], w[S][L];
    if constexpr (KIND == SWEEP_FIRST) {
      // U_n, F(U_n, t_n), w* = U_n + k F(U_n)
#pragma unroll
      for (int s = 0; s < S; ++s) load(0, s, cu[s]);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], f[S];
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = cu[s][t];
        reaction_point<R, S>(A, u, f, src_at(t));
#pragma unroll
        for (int s = 0; s < S; ++s) {
          cf[s][t] = (t < cnt) ? f[s] : R(0);
          w[s][t] = fma((R)A.k, cf[s][t], cu[s][t]);
        }
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
      R F0, Y0, F1, Y1;
      pass1x2<R, L>(A.mat[s][1], m, j, cu[s], cf[s], F0, Y0, F1, Y1);
      put(5 * s + 0, F0, Y0);
      put(5 * s + 2, F1, Y1);
      pass1x2<R, L>(A.mat[s][2], m, j, cu[s], cf[s], F0, Y0, F1, Y1);
      put(5 * s + 1, F0, Y0);
      put(5 * s + 3, F1, Y1);
      pass1<R, L>(A.mat[s][0], m, j, w[s], F0, Y0);
      put(5 * s + 4, F0, Y0);
    }
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, 0, NQ, periodic);
    __syncthreads();
    // pass 2: c_U <- 9 T c_U - 8 S c_U, c_f likewise, w <- P w
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R xa[L], xb[L], G, X, sg;
      carries(5 * s + 0, G, X, sg);
      pass2<R, L>(A.mat[s][1], m, j, cu[s], G, X, sg, xa);
      carries(5 * s + 1, G, X, sg);
      pass2<R, L>(A.mat[s][2], m, j, cu[s], G, X, sg, xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] = fma(R(9), xa[t], R(-8) * xb[t]);
      store(0, s, xa);
      carries(5 * s + 2, G, X, sg);
      pass2<R, L>(A.mat[s][1], m, j, cf[s], G, X, sg, xa);
      carries(5 * s + 3, G, X, sg);
      pass2<R, L>(A.mat[s][2], m, j, cf[s], G, X, sg, xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] = fma(R(9), xa[t], R(-8) * xb[t]);
      store(1, s, xa);
      carries(5 * s + 4, G, X, sg);
      pass2<R, L>(A.mat[s][0], m, j, w[s], G, X, sg, xa);
      store(2, s, xa);
    }
  } else {
    // LAST: phase A  U* = P_d w ; phase B  U_{n+1} = T_d f1 - S_d f2
    R cu[S][L], cf[S][L], w[S][L];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      load(0, s, cu[s]);
      load(1, s, cf[s]);
      load(2, s, w[s]);
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R F0, Y0;
      pass1<R, L>(A.mat[s][0], m, j, w[s], F0, Y0);
      put(s, F0, Y0);
    }
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, 0, S, periodic);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R x[L], G, X, sg;
      carries(s, G, X, sg);
      pass2<R, L>(A.mat[s][0], m, j, w[s], G, X, sg, x);
#pragma unroll
      for (int t = 0; t < L; ++t) w[s][t] = x[t];  // w now holds U*
    }
    // F(U*, t_{n+1}); f1, f2 overwrite c_U, c_f
    const R k = (R)A.k;
#pragma unroll
    for (int t = 0; t < L; ++t) {
      R u[S], f[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = w[s][t];
      reaction_point<R, S>(A, u, f, src_at(t));
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const R fs = (t < cnt) ? f[s] : R(0);
        const R a = cu[s][t], b = cf[s][t];
        cu[s][t] = fma(R(9), a, fma(R(2) * k, b, k * fs));
        cf[s][t] = fma(R(8), a, fma(R(1.5) * k, b, R(0.5) * k * fs));
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R F0, Y0, F1, Y1;
      pass1<R, L>(A.mat[s][1], m, j, cu[s], F0, Y0);
      pass1<R, L>(A.mat[s][2], m, j, cf[s], F1, Y1);
      put(S + 2 * s, F0, Y0);
      put(S + 2 * s + 1, F1, Y1);
    }
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, S, 2 * S, periodic);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R xa[L], xb[L], G, X, sg;
      carries(S + 2 * s, G, X, sg);
      pass2<R, L>(A.mat[s][1], m, j, cu[s], G, X, sg, xa);
      carries(S + 2 * s + 1, G, X, sg);
      pass2<R, L>(A.mat[s][2], m, j, cf[s], G, X, sg, xb);
#pragma unroll
      for (int t = 0; t < L; ++t) xa[t] -= xb[t];
      store(0, s, xa);
    }
  }
}

// Register kernel: one block per group of nlb lines, inputs loaded straight
// from global memory (vector loads on x, coalesced row segments on strided axes).
template <typename R, int S, int L, bool CONTIG, int KIND>
__device__ __forceinline__ void sweep_block(const SweepArgs<R> &A, int bid, unsigned char *smem, double t_eval,
                                            double exp_mt) {
  (void)t_eval;
  const int m = A.m, nlb = A.nlb;
  const int tid = threadIdx.x;
  // threads past nlb*m (batched launches size blocks for the largest
  // instance) own no chunk but still take part in every barrier and scan
  const bool thr_ok = tid < nlb * m;
  // lanes walk neighbouring lines on every axis: table reads are warp broadcasts
  int l = tid % nlb, j = tid / nlb;
  if (!thr_ok) { l = 0; j = 0; }
  long long base;
  bool line_ok;
  ChunkPos<R> c;
  if constexpr (CONTIG) {
    const long long line = (long long)bid * nlb + l;
    line_ok = thr_ok && line < A.nlines;
    base = line * A.n;
    c.qbase = line_ok ? line_source_base(A, true, line, 0, 0, exp_mt) : R(0);
  } else {
    const long long lo = (long long)(bid % A.nlo_blocks) * nlb + l;
    const long long hi = bid / A.nlo_blocks;
    line_ok = thr_ok && lo < A.st;
    base = lo + hi * A.st * A.n;
    c.qbase = line_ok ? line_source_base(A, false, 0, lo, hi, exp_mt) : R(0);
  }
  const long long st = CONTIG ? 1 : A.st;
  c.l = l;
  c.j = j;
  c.i0 = j * L;
  c.cnt = line_ok ? max(0, min(L, A.n - c.i0)) : 0;
  c.thr_ok = thr_ok;
  const long long off0 = base + (long long)c.i0 * st;
  const long long N = A.N;
  const int cnt = c.cnt;
  auto load = [&](int f, int s, R (&v)[L]) { load_chunk<R, L, CONTIG>(v, A.in[f] + s * N, off0, st, cnt); };
  auto store = [&](int f, int s, const R (&v)[L]) { store_chunk<R, L, CONTIG>(v, A.out[f] + s * N, off0, st, cnt); };
  chunk_sweep<R, S, L, KIND>(A, c, smem, load, store);
}

template <typename R, int S, int L, bool CONTIG, int KIND>
__global__ void __launch_bounds__(ETD_MAX_THREADS) sweep_kernel(const __grid_constant__ SweepArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  sweep_block<R, S, L, CONTIG, KIND>(A, blockIdx.x, smem, A.t_eval, A.exp_mt);
}

// Batched ensemble: one launch covers every instance; block b belongs to the
// instance i with block_start[i] <= b < block_start[i+1].
template <typename R, int S, int L, bool CONTIG, int KIND>
__global__ void __launch_bounds__(ETD_MAX_THREADS) sweep_kernel_batched(const SweepArgs<R> *__restrict__ args,
                                                              const int *__restrict__ block_start, int ninst,
                                                              double t_eval, double exp_mt) {
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
