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
  R q = A.exp_mtR;
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
  return A.rpR[0] * ((A.rpR[1] * A.src_lfR - R(1)) * q + rdiv(q, R(1) + q));
}

// Tile layouts (positions past the end of a line are zero and stay zero):
//   strided: element (line l, position i) at i * nlb + l, rows 0 .. m L - 1
//   x axis:  element (line l, position i) at l * cp + i, cp = m L + 1 (odd)
// The tile's chunks are copied to registers and solved by chunk_sweep (the
// same code as the register kernel); x-axis results are staged in shared
// memory and written back as contiguous rows, strided results go straight
// to global memory as coalesced row segments.
template <typename R, int S, int L, bool CONTIG, int KIND>
__device__ __forceinline__ void compute_tile(const SweepArgs<R> &A, const TileCoord &c, const R *buf,
                                             unsigned char *smem, int lp, int cc) {
  const int m = A.m, nlb = A.nlb, n = A.n, te = A.sp.tile_elems;
  const int cp = m * L + 1;
  const int tid = threadIdx.x;
  const bool thr_ok = tid < nlb * m;
  const int l = thr_ok ? tid % nlb : 0;
  const int j = thr_ok ? tid / nlb : 0;
  const bool lvalid = thr_ok && l < c.nvalid;
  ChunkPos<R> p;
  p.l = l;
  p.j = j;
  p.i0 = j * L;
  p.cnt = lvalid ? max(0, min(L, n - j * L)) : 0;
  p.thr_ok = thr_ok;
  p.jt = j;
  p.sc = whole_lines(A.m);
  p.qbase = source_base<R, CONTIG>(A, c, l);
  const int off0 = CONTIG ? l * cp + j * L : (j * L) * nlb + l;
  const int pstep = CONTIG ? 1 : nlb;
  R *outs = reinterpret_cast<R *>(smem + A.sp.off_out);
  const int cnt = p.cnt;
  auto load = [&](int f, int s, R (&v)[L]) {
    const R *src = buf + (size_t)(KIND == SWEEP_FIRST ? s : f * S + s) * te + off0;
#pragma unroll
    for (int t = 0; t < L; ++t) v[t] = src[t * pstep];
  };
  auto store = [&](int f, int s, const R (&v)[L]) {
    if constexpr (CONTIG) {
      R *o = outs + (size_t)(f * S + s) * te + off0;  // padding positions are never written back
#pragma unroll
      for (int t = 0; t < L; ++t) o[t] = v[t];
    } else if (lvalid) {
      R *po = A.out[f] + (long long)s * A.N + c.gbase + l + (long long)(j * L) * A.st;
#pragma unroll
      for (int t = 0; t < L; ++t)
        if (t < cnt) po[(long long)t * A.st] = v[t];
    }
  };
  chunk_sweep<R, S, L, KIND, 1>(A, p, smem + A.sp.off_sum, load, store);
  if constexpr (CONTIG) {
    // coalesced write-back: thread (lp, cc) writes elements cc + k m of line lp
    constexpr int NOUT = (KIND == SWEEP_LAST) ? S : 3 * S;
    __syncthreads();
    if (lp < nlb && lp < c.nvalid) {
#pragma unroll
      for (int f = 0; f < NOUT; ++f) {
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
