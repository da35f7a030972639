// etd_sweep_smem.cuh -- persistent, shared-memory-staged fused sweeps.
//
// Each block loops over tiles of `nlb` complete lines.  The input fields of
// the next tile are copied into shared memory with cp.async while the current
// tile is solved (double buffering), so HBM traffic overlaps the solves.
// Compute mapping for every axis: l = tid % nlb (lanes walk neighbouring
// lines), j = tid / nlb (chunk of L positions) -- all lanes of a warp read the
// same table entry (broadcast).  Staged layouts:
//   strided axes: tile[i * nlb + l]       (a row segment of nlb lines is one
//                 contiguous global segment: 16-byte async copies)
//   x axis:       tile[l * (m L + 1) + i] (odd pitch: lanes = lines read
//                 without bank conflicts); results are staged the same way
//                 and written back as contiguous row segments.
// The line-solve arithmetic (two passes around one exchange) is the one of
// etd_sweep.cuh.
#pragma once

#include "etd_sweep.cuh"

namespace etd {

__device__ __forceinline__ unsigned smem_addr(const void *p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// async global -> shared copy of BYTES (4, 8 or 16); src_bytes < BYTES zero-fills the rest
template <int BYTES>
__device__ __forceinline__ void cp_async(void *dst, const void *src, int src_bytes) {
  if constexpr (BYTES == 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_addr(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
  } else {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(smem_addr(dst)), "l"(src), "n"(BYTES),
                 "r"(src_bytes)
                 : "memory");
  }
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct TileCoord {
  long long gbase;  // element offset of (line 0, position 0) within a field
  long long line0;  // x axis: first line
  long long lo0;    // strided axes: first low line index
  long long hi;     // strided axes: high line index
  int nvalid;       // lines of the tile inside the grid
};

template <typename R, bool CONTIG>
__device__ __forceinline__ TileCoord tile_coord(const SweepArgs<R> &A, int tile) {
  TileCoord c;
  if constexpr (CONTIG) {
    c.line0 = (long long)tile * A.nlb;
    c.lo0 = 0;
    c.hi = 0;
    c.gbase = c.line0 * A.n;
    c.nvalid = (int)min((long long)A.nlb, A.nlines - c.line0);
  } else {
    c.line0 = 0;
    c.lo0 = (long long)(tile % A.nlo_blocks) * A.nlb;
    c.hi = tile / A.nlo_blocks;
    c.gbase = c.lo0 + c.hi * A.st * A.n;
    c.nvalid = (int)min((long long)A.nlb, A.st - c.lo0);
  }
  return c;
}

// pointer to staged input field f (species-major within each carried field)
template <typename R, int S, int KIND>
__device__ __forceinline__ const R *staged_src(const SweepArgs<R> &A, int f) {
  if constexpr (KIND == SWEEP_FIRST) return A.in[0] + (long long)f * A.N;
  else return A.in[f / S] + (long long)(f % S) * A.N;
}

// issue the async copies of one tile's input fields into buf
template <typename R, int S, int L, bool CONTIG, int KIND>
__device__ __forceinline__ void issue_tile(const SweepArgs<R> &A, const TileCoord &c, R *buf, int lp, int cc) {
  constexpr int NIN = (KIND == SWEEP_FIRST) ? S : 3 * S;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int n = A.n, nlb = A.nlb, te = A.sp.tile_elems;
#pragma unroll
  for (int f = 0; f < NIN; ++f) {
    const R *src = staged_src<R, S, KIND>(A, f) + c.gbase;
    R *dst = buf + (size_t)f * te;
    if constexpr (CONTIG) {
      // thread (lp, cc): elements cc + k m of line lp (consecutive threads,
      // consecutive global addresses)
      if (lp < nlb) {
        const bool valid = lp < c.nvalid;
#pragma unroll
        for (int k = 0; k < L; ++k) {
          const int i = cc + k * A.m;
          if (i < n)
            cp_async<sizeof(R)>(dst + lp * (A.m * L + 1) + i, valid ? src + (long long)lp * n + i : src,
                                valid ? (int)sizeof(R) : 0);
        }
      }
    } else if (A.sp.vec) {
      constexpr int VW = 16 / sizeof(R);
      const int G = nlb / VW;  // 16-byte groups per row segment (power of two)
      const int sh = __ffs(G) - 1;
      const int total = n * G;
      for (int q = tid; q < total; q += nth) {
        const int i = q >> sh, g = q & (G - 1);
        const int l0 = g * VW;
        const int nv = min(VW, c.nvalid - l0);
        cp_async<16>(dst + i * nlb + l0, nv > 0 ? src + l0 + (long long)i * A.st : src,
                     nv > 0 ? nv * (int)sizeof(R) : 0);
      }
    } else {
      const int sh = __ffs(nlb) - 1;  // nlb is a power of two
      const int total = n * nlb;
      for (int q = tid; q < total; q += nth) {
        const int i = q >> sh, l = q & (nlb - 1);
        const bool valid = l < c.nvalid;
        cp_async<sizeof(R)>(dst + i * nlb + l, valid ? src + l + (long long)i * A.st : src,
                            valid ? (int)sizeof(R) : 0);
      }
    }
  }
}

// e^{-t} prod_{b != axis} sin(pi x_b / L_b) for line l of the tile (0 outside the grid)
template <typename R, bool CONTIG>
__device__ __forceinline__ R source_base(const SweepArgs<R> &A, const TileCoord &c, int l) {
  if (A.phi[0] == nullptr || l >= c.nvalid) return R(0);
  R q = (R)A.exp_mt;
  if constexpr (CONTIG) {  // line index = y + z ny
    const long long line = c.line0 + l;
    const long long y = line % A.ny, z = line / A.ny;
    q *= A.phi[1][y];
    if (A.phi[2]) q *= A.phi[2][z];
  } else if (A.axis == 1) {  // lo = x, hi = z
    q *= A.phi[0][c.lo0 + l];
    if (A.phi[2]) q *= A.phi[2][c.hi];
  } else {  // axis 2: lo = x + y nx
    const long long lo = c.lo0 + l;
    q *= A.phi[0][lo % A.nx] * A.phi[1][lo / A.nx];
  }
  return q;
}

template <typename R>
__device__ __forceinline__ R source_at(const SweepArgs<R> &A, R q) {
  return (R)A.rp[0] * (((R)A.rp[1] * (R)A.src_lf - R(1)) * q + q / (R(1) + q));
}

// two solves over the chunk: y1 = M1^{-1} b1, y2 = M2^{-1} b2.  q1/q2 point
// at the chunk's L table entries, b1(t)/b2(t) return the right-hand side at
// position t of the chunk (zero past the end of the line).
template <typename R, int L, bool PER, typename B1, typename B2>
__device__ __forceinline__ void solve2(const typename V4T<R>::T *__restrict__ q1, const typename V4T<R>::T *__restrict__ q2,
                                       B1 b1, B2 b2, R G1, R X1, R s1, R G2, R X2, R s2, R (&y1)[L], R (&y2)[L]) {
  R g1 = G1, g2 = G2;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const typename V4T<R>::T a1 = q1[t], a2 = q2[t];
    g1 = fma(a1.x, g1, b1(t)) * a1.y;
    g2 = fma(a2.x, g2, b2(t)) * a2.y;
    y1[t] = g1;
    y2[t] = g2;
  }
  R x1 = X1, x2 = X2;
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    const typename V4T<R>::T a1 = q1[t], a2 = q2[t];
    x1 = fma(-a1.z, x1, y1[t]);
    x2 = fma(-a2.z, x2, y2[t]);
    if constexpr (PER) {
      y1[t] = fma(-s1, a1.w, x1);
      y2[t] = fma(-s2, a2.w, x2);
    } else {
      y1[t] = x1;
      y2[t] = x2;
    }
  }
}

template <typename R, int L, bool PER, typename B1>
__device__ __forceinline__ void solve1(const typename V4T<R>::T *__restrict__ q, B1 b1, R G, R X, R s, R (&y)[L]) {
  R g = G;
#pragma unroll
  for (int t = 0; t < L; ++t) {
    const typename V4T<R>::T a = q[t];
    g = fma(a.x, g, b1(t)) * a.y;
    y[t] = g;
  }
  R x = X;
#pragma unroll
  for (int t = L - 1; t >= 0; --t) {
    const typename V4T<R>::T a = q[t];
    x = fma(-a.z, x, y[t]);
    if constexpr (PER) y[t] = fma(-s, a.w, x);
    else y[t] = x;
  }
}

#define ETD_SOLVE2(PERV, ...) (PERV ? solve2<R, L, true>(__VA_ARGS__) : solve2<R, L, false>(__VA_ARGS__))
#define ETD_SOLVE1(PERV, ...) (PERV ? solve1<R, L, true>(__VA_ARGS__) : solve1<R, L, false>(__VA_ARGS__))

// Tile layouts (positions past the end of a line are zero and stay zero):
//   strided: element (line l, position i) at i * nlb + l, rows 0 .. m L - 1
//   x axis:  element (line l, position i) at l * cp + i, cp = m L + 1 (odd)
template <typename R, int S, int L, bool CONTIG, int KIND>
__device__ __forceinline__ void compute_tile(const SweepArgs<R> &A, const TileCoord &c, const R *buf,
                                             unsigned char *smem, int lp, int cc) {
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  using V4 = typename V4T<R>::T;
  using V2 = typename V2T<R>::T;
  const int m = A.m, nlb = A.nlb, n = A.n, te = A.sp.tile_elems, pitch = A.pitch;
  const int cp = m * L + 1;
  const int tid = threadIdx.x;
  const bool thr_ok = tid < nlb * m;
  const int l = thr_ok ? tid % nlb : 0;
  const int j = thr_ok ? tid / nlb : 0;
  const int cnt = max(0, min(L, n - j * L));  // real positions of this chunk
  const bool periodic = A.mat[0][0].sm_inv != 0.0;
  R *sF = reinterpret_cast<R *>(smem + A.sp.off_sum);
  R *sY = sF + (size_t)NQ * nlb * pitch;
  double *sSig = reinterpret_cast<double *>(smem + A.sp.off_sig);
  const size_t myidx = (size_t)l * pitch + j;
  auto put = [&](int q, R F, R Y) {
    if (thr_ok) {
      sF[(size_t)q * nlb * pitch + myidx] = F;
      sY[(size_t)q * nlb * pitch + myidx] = Y;
    }
  };
  auto carries = [&](int q, R &G, R &X, R &sg) {
    G = sF[(size_t)q * nlb * pitch + myidx];
    X = sY[(size_t)q * nlb * pitch + myidx];
    sg = (R)sSig[(size_t)q * nlb + l];
  };
  // offset of position t of this thread's chunk in a field tile, and the stride between positions
  const int off0 = CONTIG ? l * cp + j * L : (j * L) * nlb + l;
  const int pstep = CONTIG ? 1 : nlb;
  auto at = [&](const R *f, int t) -> R { return f[off0 + t * pstep]; };
  const bool lvalid = thr_ok && l < c.nvalid;
  const R k = (R)A.k;
  const R qbase = source_base<R, CONTIG>(A, c, l);
  const R *phia = A.phi[A.axis];
  auto src_at = [&](int t) -> R {
    return (qbase != R(0)) ? source_at(A, qbase * phia[min(j * L + t, n - 1)]) : R(0);
  };
  // strided outputs: coalesced row segments straight to global memory
  auto gstore = [&](int fld, int s, const R (&y)[L]) {
    if (lvalid) {
      R *po = A.out[fld] + (long long)s * A.N + c.gbase + l + (long long)(j * L) * A.st;
#pragma unroll
      for (int t = 0; t < L; ++t)
        if (t < cnt) po[(long long)t * A.st] = y[t];
    }
  };

  if constexpr (KIND == SWEEP_FIRST || KIND == SWEEP_MIDDLE) {
    R *f0s = reinterpret_cast<R *>(smem + A.sp.off_f0);    // FIRST: F(U_n) per species
    R *outs = reinterpret_cast<R *>(smem + A.sp.off_out);  // x axis: staged results
    const R *fu[S];
    const R *ff[S];
    const R *fw[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      fu[s] = buf + (size_t)s * te;
      ff[s] = (KIND == SWEEP_FIRST) ? f0s + (size_t)s * te : buf + (size_t)(S + s) * te;
      fw[s] = buf + (size_t)(2 * S + s) * te;
    }
    // pass 1 (FIRST also evaluates F(U_n, t_n) and keeps it in shared memory)
    R aF[NQ], aY[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) aF[q] = aY[q] = R(0);
    const V2 *vT[S], *vS[S], *vP[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      vT[s] = A.mat[s][1].sum + j * L;
      vS[s] = A.mat[s][2].sum + j * L;
      vP[s] = A.mat[s][0].sum + j * L;
    }
#pragma unroll
    for (int t = 0; t < L; ++t) {
      R u[S], f[S], w[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = at(fu[s], t);
      if constexpr (KIND == SWEEP_FIRST) {
        reaction_point<R, S>(A, u, f, src_at(t));
#pragma unroll
        for (int s = 0; s < S; ++s) {
          if (thr_ok && t < cnt) f0s[(size_t)s * te + off0 + t * pstep] = f[s];
          w[s] = fma(k, f[s], u[s]);
        }
      } else {
#pragma unroll
        for (int s = 0; s < S; ++s) {
          f[s] = at(ff[s], t);
          w[s] = at(fw[s], t);
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const V2 a = vT[s][t], b = vS[s][t], p = vP[s][t];
        aF[5 * s + 0] = fma(a.x, u[s], aF[5 * s + 0]);
        aY[5 * s + 0] = fma(a.y, u[s], aY[5 * s + 0]);
        aF[5 * s + 1] = fma(b.x, u[s], aF[5 * s + 1]);
        aY[5 * s + 1] = fma(b.y, u[s], aY[5 * s + 1]);
        aF[5 * s + 2] = fma(a.x, f[s], aF[5 * s + 2]);
        aY[5 * s + 2] = fma(a.y, f[s], aY[5 * s + 2]);
        aF[5 * s + 3] = fma(b.x, f[s], aF[5 * s + 3]);
        aY[5 * s + 3] = fma(b.y, f[s], aY[5 * s + 3]);
        aF[5 * s + 4] = fma(p.x, w[s], aF[5 * s + 4]);
        aY[5 * s + 4] = fma(p.y, w[s], aY[5 * s + 4]);
      }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) put(q, aF[q], aY[q]);
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, 0, NQ, periodic);
    __syncthreads();
    // pass 2: c_U <- 9 T c_U - 8 S c_U ; c_f likewise ; w <- P w
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const V4 *qT = A.mat[s][1].pos + j * L;
      const V4 *qS = A.mat[s][2].pos + j * L;
      const V4 *qP = A.mat[s][0].pos + j * L;
#pragma unroll 1
      for (int fld = 0; fld < 3; ++fld) {
        R ya[L], yb[L], G1, X1, s1, G2, X2, s2;
        if (fld < 2) {
          const R *pb = fld == 0 ? fu[s] : ff[s];
          carries(5 * s + 2 * fld, G1, X1, s1);
          carries(5 * s + 2 * fld + 1, G2, X2, s2);
          auto bget = [&](int t) { return at(pb, t); };
          ETD_SOLVE2(periodic, qT, qS, bget, bget, G1, X1, s1, G2, X2, s2, ya, yb);
#pragma unroll
          for (int t = 0; t < L; ++t) ya[t] = fma(R(9), ya[t], R(-8) * yb[t]);
        } else {
          carries(5 * s + 4, G1, X1, s1);
          if constexpr (KIND == SWEEP_FIRST) {
            auto bget = [&](int t) { return fma(k, at(ff[s], t), at(fu[s], t)); };
            ETD_SOLVE1(periodic, qP, bget, G1, X1, s1, ya);
          } else {
            auto bget = [&](int t) { return at(fw[s], t); };
            ETD_SOLVE1(periodic, qP, bget, G1, X1, s1, ya);
          }
        }
        if constexpr (CONTIG) {
          R *o = outs + (size_t)(fld * S + s) * te + off0;
#pragma unroll
          for (int t = 0; t < L; ++t) o[t] = ya[t];  // padding positions are never written back
        } else {
          gstore(fld, s, ya);
        }
      }
    }
    if constexpr (CONTIG) {
      // coalesced write-back: thread (lp, cc) writes elements cc + k m of line lp
      __syncthreads();
      if (lp < nlb && lp < c.nvalid) {
#pragma unroll
        for (int f = 0; f < 3 * S; ++f) {
          const R *o = outs + (size_t)f * te + lp * cp;
          R *dst = A.out[f / S] + (long long)(f % S) * A.N + c.gbase + (long long)lp * n;
#pragma unroll
          for (int kk = 0; kk < L; ++kk) {
            const int i = cc + kk * m;
            if (i < n) dst[i] = o[i];
          }
        }
      }
    }
  } else {
    // LAST (strided): phase A  U* = P_d w ; F(U*, t_{n+1}) ; f1, f2 ; phase B  U_{n+1} = T_d f1 - S_d f2
    R *bu = const_cast<R *>(buf);  // the tile is ours: U*, f1, f2 overwrite w, c_U, c_f in place
    R *pu[S], *pf[S], *pw[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      pu[s] = bu + (size_t)s * te;
      pf[s] = bu + (size_t)(S + s) * te;
      pw[s] = bu + (size_t)(2 * S + s) * te;
    }
    R aF[S], aY[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const V2 *vP = A.mat[s][0].sum + j * L;
      R f = R(0), y = R(0);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        const R w = at(pw[s], t);
        f = fma(vP[t].x, w, f);
        y = fma(vP[t].y, w, y);
      }
      aF[s] = f;
      aY[s] = y;
    }
#pragma unroll
    for (int s = 0; s < S; ++s) put(s, aF[s], aY[s]);
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, 0, S, periodic);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R y[L], G, X, sg;
      carries(s, G, X, sg);
      auto bget = [&](int t) { return at(pw[s], t); };
      ETD_SOLVE1(periodic, A.mat[s][0].pos + j * L, bget, G, X, sg, y);
      if (thr_ok) {
#pragma unroll
        for (int t = 0; t < L; ++t)
          if (t < cnt) pw[s][off0 + t * pstep] = y[t];  // own chunk only: no barrier needed
      }
    }
    R bF[2 * S], bY[2 * S];
#pragma unroll
    for (int q = 0; q < 2 * S; ++q) bF[q] = bY[q] = R(0);
#pragma unroll
    for (int t = 0; t < L; ++t) {
      R u[S], f[S];
#pragma unroll
      for (int s = 0; s < S; ++s) u[s] = at(pw[s], t);
      reaction_point<R, S>(A, u, f, src_at(t));
#pragma unroll
      for (int s = 0; s < S; ++s) {
        const R a = at(pu[s], t), b = at(pf[s], t);
        const R f1 = fma(R(9), a, fma(R(2) * k, b, k * f[s]));
        const R f2 = fma(R(8), a, fma(R(1.5) * k, b, R(0.5) * k * f[s]));
        if (thr_ok && t < cnt) {
          pu[s][off0 + t * pstep] = f1;
          pf[s][off0 + t * pstep] = f2;
        }
        const V2 va = A.mat[s][1].sum[j * L + t], vb = A.mat[s][2].sum[j * L + t];
        bF[2 * s] = fma(va.x, f1, bF[2 * s]);
        bY[2 * s] = fma(va.y, f1, bY[2 * s]);
        bF[2 * s + 1] = fma(vb.x, f2, bF[2 * s + 1]);
        bY[2 * s + 1] = fma(vb.y, f2, bY[2 * s + 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < 2 * S; ++q) put(S + q, bF[q], bY[q]);
    __syncthreads();
    scan_lines<R, S, KIND>(A, sF, sY, sSig, S, 2 * S, periodic);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R ya[L], yb[L], G1, X1, s1, G2, X2, s2;
      carries(S + 2 * s, G1, X1, s1);
      carries(S + 2 * s + 1, G2, X2, s2);
      auto b1 = [&](int t) { return at(pu[s], t); };
      auto b2 = [&](int t) { return at(pf[s], t); };
      ETD_SOLVE2(periodic, A.mat[s][1].pos + j * L, A.mat[s][2].pos + j * L, b1, b2, G1, X1, s1, G2, X2, s2, ya, yb);
#pragma unroll
      for (int t = 0; t < L; ++t) ya[t] -= yb[t];
      gstore(0, s, ya);
    }
  }
}

template <typename R, int S, int L, bool CONTIG, int KIND>
__device__ __forceinline__ void staged_loop(const SweepArgs<R> &A, unsigned char *smem) {
  constexpr int NIN = (KIND == SWEEP_FIRST) ? S : 3 * S;
  const int ntiles = A.sp.ntiles;
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  R *bufs = reinterpret_cast<R *>(smem + A.sp.off_buf);
  const size_t slot_elems = (size_t)NIN * A.sp.tile_elems;
  const int lp = threadIdx.x / A.m, cc = threadIdx.x - (threadIdx.x / A.m) * A.m;
  int slot = 0;
  {
    // positions past the end of a line stay zero for the whole kernel
    float4 *z = reinterpret_cast<float4 *>(smem);
    const int nz = (int)(A.sp.off_sum / 16);
    for (int q = threadIdx.x; q < nz; q += blockDim.x) z[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
  }
  issue_tile<R, S, L, CONTIG, KIND>(A, tile_coord<R, CONTIG>(A, tile), bufs, lp, cc);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    if (A.sp.nbuf == 2) {
      if (next < ntiles)
        issue_tile<R, S, L, CONTIG, KIND>(A, tile_coord<R, CONTIG>(A, next), bufs + (slot ^ 1) * slot_elems, lp, cc);
      cp_async_commit();
      cp_async_wait<1>();  // the current tile's copies have landed
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    compute_tile<R, S, L, CONTIG, KIND>(A, tile_coord<R, CONTIG>(A, tile), bufs + slot * slot_elems, smem, lp, cc);
    __syncthreads();  // tile buffer, staged results and exchange space free for reuse
    if (A.sp.nbuf == 2) {
      slot ^= 1;
    } else if (next < ntiles) {
      issue_tile<R, S, L, CONTIG, KIND>(A, tile_coord<R, CONTIG>(A, next), bufs, lp, cc);
      cp_async_commit();
    }
  }
  cp_async_wait<0>();
}

template <typename R, int S, int L, bool CONTIG, int KIND>
__global__ void __launch_bounds__(ETD_MAX_THREADS, 1) sweep_staged_kernel(const __grid_constant__ SweepArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  staged_loop<R, S, L, CONTIG, KIND>(A, smem);
}

}  // namespace etd
