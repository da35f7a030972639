// etd_tile.cuh -- FP32 fused sweeps on shared-memory tiles with compile-time
// geometry ("tile kernels").
//
// One block owns NLB complete lines.  Every input field of those lines is
// copied into shared memory with 16-byte async copies, the two line-solve
// passes read each thread's chunk from the tile when they need it (nothing
// stays in registers across the chunk exchange, so a thread needs few
// registers and several blocks share an SM, overlapping one block's copies
// with another's solves), results overwrite the tile in place and leave as
// 16-byte row stores.  With NLB and the chunk length L fixed at compile time
// every tile access is one shared-memory instruction at an immediate offset.
//
// Tile layouts (float elements; positions past the end of a line are zero):
//   strided axes: element (position i, line l) at (i / L) CS + (i % L) NLB + l,
//                 CS = L NLB + PADJ: a row segment of NLB lines is contiguous
//                 (one group of 16-byte copies), lanes walk lines, and PADJ
//                 shifts consecutive chunks to other banks when a warp spans
//                 several chunks;
//   x axis:       element (line l, position i) at l PITCH + i, PITCH = 4
//                 (mod 32): four consecutive positions per 16-byte load, the
//                 eight lanes of a quarter-warp on eight different bank groups.
// The arithmetic is the FP32 path of etd_sweep.cuh (pass1v / pass2x2v /
// pass2v around the shared exchange and chunk-carry scan).
#pragma once

#include "etd_sweep_smem.cuh"

namespace etd {

template <int NLB, int PK>
struct TileShape {
  static constexpr int W = NLB / PK;  // line units (lines or pairs) per block
  static constexpr int PADJ = (W < 32) ? NLB : 0;
};

template <int L, int NLB, int PK>
__host__ __device__ constexpr int tile_chunk_stride() {
  return L * NLB + TileShape<NLB, PK>::PADJ;
}

// 16-byte async copies of one strided input field (n rows of NLB floats)
template <int L, int NLB, int PK>
__device__ __forceinline__ void tile_load_strided(float *dst, const float *src, long long st, int n, int nvalid) {
  constexpr int CPR = NLB / 4;  // 16-byte copies per row segment
  constexpr int CS = tile_chunk_stride<L, NLB, PK>();
  for (int q = threadIdx.x; q < n * CPR; q += blockDim.x) {
    const int i = q / CPR, c = q - i * CPR;
    const bool ok = c * 4 < nvalid;
    cp_async<16>(dst + (i / L) * CS + (i % L) * NLB + c * 4, ok ? src + (long long)i * st + c * 4 : src, ok ? 16 : 0);
  }
}

// 16-byte row stores of one strided field from the tile
template <int L, int NLB, int PK>
__device__ __forceinline__ void tile_store_strided(float *dst, const float *tile, long long st, int n, int nvalid) {
  constexpr int CPR = NLB / 4;
  constexpr int CS = tile_chunk_stride<L, NLB, PK>();
  for (int q = threadIdx.x; q < n * CPR; q += blockDim.x) {
    const int i = q / CPR, c = q - i * CPR;
    if (c * 4 < nvalid)
      *reinterpret_cast<float4 *>(dst + (long long)i * st + c * 4) =
          *reinterpret_cast<const float4 *>(tile + (i / L) * CS + (i % L) * NLB + c * 4);
  }
}

// x axis: line l of the tile is row l (n floats, 16-byte aligned rows);
// warps walk lines, lanes walk 16-byte pieces of a row
template <int NLB>
__device__ __forceinline__ void tile_load_rows(float *dst, const float *src, int n, int pitch, int nvalid) {
  const int cpr = n >> 2, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = threadIdx.x >> 5; l < NLB; l += nw) {
    const bool ok = l < nvalid;
    for (int c = lane; c < cpr; c += 32)
      cp_async<16>(dst + l * pitch + c * 4, ok ? src + (long long)l * n + c * 4 : src, ok ? 16 : 0);
  }
}

template <int NLB>
__device__ __forceinline__ void tile_store_rows(float *dst, const float *tile, int n, int pitch, int nvalid) {
  const int cpr = n >> 2, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int l = threadIdx.x >> 5; l < nvalid; l += nw)
    for (int c = lane; c < cpr; c += 32)
      *reinterpret_cast<float4 *>(dst + (long long)l * n + c * 4) =
          *reinterpret_cast<const float4 *>(tile + l * pitch + c * 4);
}

// One thread's view of its chunk in a field tile: position t at p + t * STEP
template <typename V, int L, int STEP>
struct ChunkRef {
  float *p;
  __device__ __forceinline__ void get(V (&v)[L]) const {
    if constexpr (STEP == 1) {  // x tiles: four positions per load
#pragma unroll
      for (int t = 0; t < L; t += 4) {
        const float4 q = *reinterpret_cast<const float4 *>(p + t);
        v[t] = q.x;
        v[t + 1] = q.y;
        v[t + 2] = q.z;
        v[t + 3] = q.w;
      }
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) v[t] = *reinterpret_cast<const V *>(p + t * STEP);
    }
  }
  __device__ __forceinline__ void put(const V (&v)[L]) const {
    if constexpr (STEP == 1) {
#pragma unroll
      for (int t = 0; t < L; t += 4)
        *reinterpret_cast<float4 *>(p + t) = make_float4(v[t], v[t + 1], v[t + 2], v[t + 3]);
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) *reinterpret_cast<V *>(p + t * STEP) = v[t];
    }
  }
};

template <int S, int L, int NLB, int KIND, int PK>
__device__ __forceinline__ void tile_sweep(const SweepArgs<float> &A, unsigned char *smem) {
  using V = typename LaneT<float, PK>::T;
  constexpr bool CONTIG = (KIND == SWEEP_FIRST);
  static_assert(!CONTIG || PK == 1, "x tiles run one line per thread");
  static_assert(L % 4 == 0 && NLB % 4 == 0, "16-byte tile rows and chunk loads");
  constexpr int W = TileShape<NLB, PK>::W;
  constexpr int CS = tile_chunk_stride<L, NLB, PK>();
  constexpr int STEP = CONTIG ? 1 : NLB;
  constexpr int NQ = (KIND == SWEEP_LAST) ? 3 * S : 5 * S;
  const int m = A.m, n = A.n;
  const int xp = A.sp.tile_pitch;   // x tiles: row pitch
  const int ft = A.sp.tile_elems;  // floats per field tile
  float *tiles = reinterpret_cast<float *>(smem);
  const int tid = threadIdx.x;
  const int u = tid % W, j = tid / W;  // line unit (lane-fastest), chunk
  const bool thr_ok = j < m;

  // ---- tile coordinates and async copies of the inputs
  long long gbase;  // element offset of (line 0, position 0) within a field
  int nvalid;       // lines of the tile inside the grid
  long long lo0 = 0, hi = 0, line0 = 0;
  if constexpr (CONTIG) {
    line0 = (long long)blockIdx.x * NLB;
    gbase = line0 * n;
    nvalid = (int)min((long long)NLB, A.nlines - line0);
  } else {
    lo0 = (long long)(blockIdx.x % A.nlo_blocks) * NLB;
    hi = blockIdx.x / A.nlo_blocks;
    gbase = lo0 + hi * A.st * n;
    nvalid = (int)min((long long)NLB, A.st - lo0);
  }
  constexpr int NIN = CONTIG ? S : 3 * S;  // staged input fields (FIRST: U; else c_U, c_f, w)
  auto tile_of = [&](int field, int s) { return tiles + (field * S + s) * ft; };  // 32-bit offsets
#pragma unroll
  for (int f = 0; f < NIN; ++f) {
    const int field = CONTIG ? 0 : f / S, s = CONTIG ? f : f % S;
    const float *src = A.in[field] + (long long)s * A.N + gbase;
    if constexpr (CONTIG) tile_load_rows<NLB>(tile_of(0, s), src, n, xp, nvalid);
    else tile_load_strided<L, NLB, PK>(tile_of(field, s), src, A.st, n, nvalid);
  }
  cp_async_commit();
  // zero the padding positions i in [n, m L) of every field tile (never copied)
  {
    const int npad = m * L - n;
    if (npad > 0) {
      constexpr int NF = 3 * S;
      for (int q = tid; q < NF * NLB * npad; q += blockDim.x) {
        const int f = q / (NLB * npad), r = q - f * (NLB * npad);
        const int l = r / npad, i = n + (r - l * npad);
        float *t = tiles + f * ft;
        if constexpr (CONTIG) t[l * xp + i] = 0.f;
        else t[(i / L) * CS + (i % L) * NLB + l] = 0.f;
      }
    }
  }
  cp_async_wait<0>();
  __syncthreads();

  // ---- this thread's chunk
  const int i0 = j * L;
  const int lane_line = u * PK;  // first line of the unit within the tile
  const bool line_ok = thr_ok && lane_line < nvalid;
  const int cnt = line_ok ? max(0, min(L, n - i0)) : 0;
  const int off = CONTIG ? (lane_line * xp + i0) : (j * CS + lane_line);
  auto ref = [&](int field, int s) { return ChunkRef<V, L, STEP>{tile_of(field, s) + off}; };
  const V zero = Splat<V>::of(0.f);
  // manufactured source: per-line factor times phi_axis at the position
  V qbase = zero;
  if (line_ok) {
    if constexpr (CONTIG) {
      qbase = line_source_base(A, true, line0 + lane_line, 0, 0, A.exp_mtR);
    } else if constexpr (PK == 1) {
      qbase = line_source_base(A, false, 0, lo0 + lane_line, hi, A.exp_mtR);
    } else {
      qbase = make_float2(line_source_base(A, false, 0, lo0 + lane_line, hi, A.exp_mtR),
                          line_source_base(A, false, 0, lo0 + lane_line + 1, hi, A.exp_mtR));
    }
  }
  auto react = [&](const V (&uu)[S], V (&ff)[S], V src) {
    if constexpr (PK == 1) {
      reaction_point<float, S>(A, uu, ff, src);
    } else {
      float ux[S], uy[S], fx[S], fy[S];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        ux[s] = uu[s].x;
        uy[s] = uu[s].y;
      }
      reaction_point<float, S>(A, ux, fx, src.x);
      reaction_point<float, S>(A, uy, fy, src.y);
#pragma unroll
      for (int s = 0; s < S; ++s) ff[s] = make_float2(fx[s], fy[s]);
    }
  };

  // ---- exchange space (after the field tiles)
  V *sF = reinterpret_cast<V *>(smem + A.sp.off_sum);
  V *sY = sF + NQ * W * A.pitch;
  float *sSig = reinterpret_cast<float *>(smem + A.sp.off_sig);
  const int myidx = u * A.pitch + j;
  const int qstride = W * A.pitch;
  auto put = [&](int q, V F, V Y) {
    if (thr_ok) {
      sF[q * qstride + myidx] = F;
      sY[q * qstride + myidx] = Y;
    }
  };
  auto carry = [&](int q) {
    Carry<V> c;
    c.G = sF[q * qstride + myidx];
    c.X = sY[q * qstride + myidx];
    c.ns = vneg(get_sigma(sSig + (q * W + u) * PK, zero));
    return c;
  };
  const V k9 = Splat<V>::of(9.f), km8 = Splat<V>::of(-8.f);

  if constexpr (KIND == SWEEP_FIRST || KIND == SWEEP_MIDDLE) {
    // pass 1: five solves per species share one exchange.  FIRST computes
    // F(U_n, t_n) and w* = U_n + k F in registers, runs pass 1 on them and
    // keeps F and w* in the c_f and w tiles for pass 2.
    if constexpr (CONTIG) {
      V uu[S][L], ff[S][L];
      if (thr_ok) {
#pragma unroll
        for (int s = 0; s < S; ++s) ref(0, s).get(uu[s]);
        V src[L];
        chunk_sources<float, L, PK>(A, qbase, i0, cnt, src);
#pragma unroll
        for (int t = 0; t < L; ++t) {
          V us[S], fs[S];
#pragma unroll
          for (int s = 0; s < S; ++s) us[s] = uu[s][t];
          react(us, fs, src[t]);
#pragma unroll
          for (int s = 0; s < S; ++s) ff[s][t] = fs[s];
        }
        if (cnt < L) {
#pragma unroll
          for (int s = 0; s < S; ++s)
#pragma unroll
            for (int t = 0; t < L; ++t)
              if (t >= cnt) ff[s][t] = zero;
        }
      } else {
#pragma unroll
        for (int s = 0; s < S; ++s)
#pragma unroll
          for (int t = 0; t < L; ++t) uu[s][t] = ff[s][t] = zero;
      }
      const V kk = Splat<V>::of(A.kR);
      const int jj = thr_ok ? j : 0;
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V ww[L];
#pragma unroll
        for (int t = 0; t < L; ++t) ww[t] = vfma(kk, ff[s][t], uu[s][t]);
        if (thr_ok) {
          ref(1, s).put(ff[s]);
          ref(2, s).put(ww);
        }
        V F0, Y0, F1, Y1;
        pass1x2v<V, L>(A.mat[s][1], m, jj, uu[s], ff[s], F0, Y0, F1, Y1);
        put(5 * s + 0, F0, Y0);
        put(5 * s + 2, F1, Y1);
        pass1x2v<V, L>(A.mat[s][2], m, jj, uu[s], ff[s], F0, Y0, F1, Y1);
        put(5 * s + 1, F0, Y0);
        put(5 * s + 3, F1, Y1);
        pass1v<V, L>(A.mat[s][0], m, jj, ww, F0, Y0);
        put(5 * s + 4, F0, Y0);
      }
    } else {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V b0[L], b1[L], b2[L];
        if (thr_ok) {
          ref(0, s).get(b0);
          ref(1, s).get(b1);
          ref(2, s).get(b2);
        } else {
#pragma unroll
          for (int t = 0; t < L; ++t) b0[t] = b1[t] = b2[t] = zero;
        }
        const int jj = thr_ok ? j : 0;
        V F0, Y0, F1, Y1;
        pass1x2v<V, L>(A.mat[s][1], m, jj, b0, b1, F0, Y0, F1, Y1);
        put(5 * s + 0, F0, Y0);
        put(5 * s + 2, F1, Y1);
        pass1x2v<V, L>(A.mat[s][2], m, jj, b0, b1, F0, Y0, F1, Y1);
        put(5 * s + 1, F0, Y0);
        put(5 * s + 3, F1, Y1);
        pass1v<V, L>(A.mat[s][0], m, jj, b2, F0, Y0);
        put(5 * s + 4, F0, Y0);
      }
    }
    __syncthreads();
    scan_lines<float, V, PK, S, KIND>(A, sF, sY, sSig, 0, NQ, whole_lines(m));
    __syncthreads();
    if (thr_ok) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V b0[L], b1[L], xa[L], xc[L];
        ref(0, s).get(b0);
        ref(1, s).get(b1);
        pass2x2v<V, L, true>(A.mat[s][1], A.mat[s][1], m, j, b0, b1, carry(5 * s + 0), carry(5 * s + 2), xa, xc,
                             [&](int t, int k, V x) {
                               if (k == 0) xa[t] = x;
                               else xc[t] = x;
                             });
        pass2x2v<V, L, true>(A.mat[s][2], A.mat[s][2], m, j, b0, b1, carry(5 * s + 1), carry(5 * s + 3), b0, b1,
                             [&](int t, int k, V x) {
                               if (k == 0) xa[t] = vfma(k9, xa[t], vmul(km8, x));
                               else xc[t] = vfma(k9, xc[t], vmul(km8, x));
                             });
        ref(0, s).put(xa);
        ref(1, s).put(xc);
        V w[L];
        ref(2, s).get(w);
        pass2v<V, L>(A.mat[s][0], m, j, w, carry(5 * s + 4), w, [&](int t, V x) { w[t] = x; });
        ref(2, s).put(w);
      }
    }
    __syncthreads();
    // results: c_U, c_f, w tiles -> out[0..2]
#pragma unroll
    for (int f = 0; f < 3 * S; ++f) {
      const int field = f / S, s = f % S;
      float *dst = A.out[field] + (long long)s * A.N + gbase;
      if constexpr (CONTIG) tile_store_rows<NLB>(dst, tile_of(field, s), n, xp, nvalid);
      else tile_store_strided<L, NLB, PK>(dst, tile_of(field, s), A.st, n, nvalid);
    }
  } else {
    // LAST phase A: U* = P_d w
#pragma unroll
    for (int s = 0; s < S; ++s) {
      V b[L];
      if (thr_ok) ref(2, s).get(b);
      else
#pragma unroll
        for (int t = 0; t < L; ++t) b[t] = zero;
      V F0, Y0;
      pass1v<V, L>(A.mat[s][0], m, thr_ok ? j : 0, b, F0, Y0);
      put(s, F0, Y0);
    }
    __syncthreads();
    scan_lines<float, V, PK, S, KIND>(A, sF, sY, sSig, 0, S, whole_lines(m));
    __syncthreads();
    // U*, F(U*, t_{n+1}); f1 = 9 c_U + 2k c_f + k F*, f2 = 8 c_U + 3k/2 c_f + k/2 F* into the c_U, c_f tiles
    if (thr_ok) {
      V us[S][L];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V w[L];
        ref(2, s).get(w);
        pass2v<V, L>(A.mat[s][0], m, j, w, carry(s), w, [&](int t, V x) { us[s][t] = x; });
      }
      const float k = A.kR;
      const V k2 = Splat<V>::of(2.f * k), kk = Splat<V>::of(k), k15 = Splat<V>::of(1.5f * k),
              k05 = Splat<V>::of(0.5f * k), k8 = Splat<V>::of(8.f);
      V f1[S][L], f2[S][L];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        ref(0, s).get(f1[s]);
        ref(1, s).get(f2[s]);
      }
      V src[L];
      chunk_sources<float, L, PK>(A, qbase, i0, cnt, src);
#pragma unroll
      for (int t = 0; t < L; ++t) {
        V uu[S], ff[S];
#pragma unroll
        for (int s = 0; s < S; ++s) uu[s] = us[s][t];
        react(uu, ff, src[t]);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          const V fs = (cnt == L || t < cnt) ? ff[s] : zero;
          const V a = f1[s][t], b = f2[s][t];
          f1[s][t] = vfma(k9, a, vfma(k2, b, vmul(kk, fs)));
          f2[s][t] = vfma(k8, a, vfma(k15, b, vmul(k05, fs)));
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V F0, Y0, F1, Y1;
        pass1v<V, L>(A.mat[s][1], m, j, f1[s], F0, Y0);
        pass1v<V, L>(A.mat[s][2], m, j, f2[s], F1, Y1);
        put(S + 2 * s, F0, Y0);
        put(S + 2 * s + 1, F1, Y1);
        ref(0, s).put(f1[s]);
        ref(1, s).put(f2[s]);
      }
    }
    __syncthreads();
    scan_lines<float, V, PK, S, KIND>(A, sF, sY, sSig, S, 2 * S, whole_lines(m));
    __syncthreads();
    if (thr_ok) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        V b0[L], b1[L];
        ref(0, s).get(b0);
        ref(1, s).get(b1);
        pass2x2v<V, L, false>(A.mat[s][1], A.mat[s][2], m, j, b0, b1, carry(S + 2 * s), carry(S + 2 * s + 1), b0,
                              b1, [&](int t, int k, V x) {
                                if (k == 0) b0[t] = x;
                                else b0[t] = vsub(b0[t], x);
                              });
        ref(0, s).put(b0);
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      float *dst = A.out[0] + (long long)s * A.N + gbase;
      tile_store_strided<L, NLB, PK>(dst, tile_of(0, s), A.st, n, nvalid);
    }
  }
}

template <int S, int L, int NLB, int KIND, int PK>
__global__ void __launch_bounds__(512) sweep_tile_kernel(const __grid_constant__ SweepArgs<float> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  tile_sweep<S, L, NLB, KIND, PK>(A, smem);
}

}  // namespace etd
