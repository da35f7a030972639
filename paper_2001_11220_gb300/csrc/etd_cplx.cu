// etd_cplx.cu -- ETD-RDP-IF sweeps for the coupled two-species systems of
// Section 8 (complex Ginzburg-Landau with D = 1 + i alpha, cubic
// Schrodinger): complex line solves.
//
// The state is the usual species-major layout: species 0 = Re u, species 1 =
// Im u, N points each.  One sweep per axis, as in the flow charts of Section 7
// (Figs. flow2d / flow3d):
//   FIRST  (x):  f0 = F(U_n); w* = U_n + k f0; c_U = R_x U_n, c_f = R_x f0,
//                w = P_x w*                                   (5 complex solves)
//   MIDDLE (y, 3D): c_U <- R_y c_U, c_f <- R_y c_f, w <- P_y w  (5 solves)
//   LAST   (last axis): U* = P w; f* = F(U*); U_{n+1} = T f1 - S f2 with
//                f1 = 9 c_U + 2k c_f + k f*, f2 = 8 c_U + 1.5k c_f + 0.5k f*
// with R = 9T - 8S and P, T, S the inverses of I + (k/gamma) A_a for
// gamma = 1, 3, 4 (Section 6), A_a = (p + i q) B_p / h^2 on the complex field.
//
// Kernel: a block stages NL whole lines (complex, 4 slots of p nodes) in
// shared memory with coalesced loads -- along x a line is a contiguous row;
// along y / z the NL lines are neighbouring x columns, so each node row is an
// NL-element contiguous run.  One warp then solves a line: lane j owns nodes
// [j c, (j+1) c), c = ceil(p/32).  Forward elimination y_i = b_i - l_i y_{i-1}
// and back substitution x_i = y_i / piv_i - mu_i x_{i+1} are first-order
// complex recurrences: each lane reduces its chunk to an affine map, a
// 5-step warp-shuffle scan composes the maps, and each lane re-runs its chunk
// from the true carry.  Periodic lines use the circulant factorisation of
// the cyclic matrix instead (two cyclic first-order recurrences, below).
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <new>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_context.h"
#include "etd_internal.h"
#include "etd_tables.h"

namespace etd {
etd_status validate_problem(const etd_grid *grid, const double *D, const etd_reaction *rx, double k,
                            int32_t precision);
cudaError_t prof_begin(etd_ctx *ctx, cudaStream_t s, cudaEvent_t &ev);
cudaError_t prof_end(etd_ctx *ctx, cudaStream_t s, int kind, cudaEvent_t ev0);
}  // namespace etd

namespace {

using namespace etd;

// d = 1: the frame without splitting, one sweep that loads U_n, forms F(U_n)
// and w* = U_n + k F, and continues as the last-axis sweep with c_U = U_n,
// c_f = F(U_n)
constexpr int CPLX_ONLY = 3;

template <typename R> struct C2 { R x, y; };

template <typename R> __device__ __forceinline__ C2<R> cmk(R x, R y) { return C2<R>{x, y}; }
template <typename R> __device__ __forceinline__ C2<R> cadd(C2<R> a, C2<R> b) { return {a.x + b.x, a.y + b.y}; }
template <typename R> __device__ __forceinline__ C2<R> csub(C2<R> a, C2<R> b) { return {a.x - b.x, a.y - b.y}; }
template <typename R> __device__ __forceinline__ C2<R> cscale(R s, C2<R> a) { return {s * a.x, s * a.y}; }
template <typename R> __device__ __forceinline__ C2<R> cmul(C2<R> a, C2<R> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename R> __device__ __forceinline__ C2<R> cneg(C2<R> a) { return {-a.x, -a.y}; }

__device__ __forceinline__ C2<float> ldt(const C2<float> *p) {
  const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
  return {v.x, v.y};
}
__device__ __forceinline__ C2<double> ldt(const C2<double> *p) {
  const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
  return {v.x, v.y};
}

template <typename R> __device__ __forceinline__ C2<R> shfl_up_c(C2<R> a, int off) {
  return {__shfl_up_sync(0xffffffffu, a.x, off), __shfl_up_sync(0xffffffffu, a.y, off)};
}
template <typename R> __device__ __forceinline__ C2<R> shfl_down_c(C2<R> a, int off) {
  return {__shfl_down_sync(0xffffffffu, a.x, off), __shfl_down_sync(0xffffffffu, a.y, off)};
}
template <typename R> __device__ __forceinline__ C2<R> shfl_c(C2<R> a, int src) {
  return {__shfl_sync(0xffffffffu, a.x, src), __shfl_sync(0xffffffffu, a.y, src)};
}

template <typename R> struct CTab {
  const C2<R> *ell, *ipv, *mu;  // Dirichlet / Neumann lines: Thomas factors
  const C2<R> *af, *ab;         // [32] per-lane chunk products of -l_i and of -mu_i
  // periodic lines: circulant factorisation alpha (I - lam E)(I - lam E^-1)
  const C2<R> *cpre, *csuf, *cchunk;  // [32] lam^(before lane), lam^(after lane), lam^(lane's nodes)
  C2<R> lam, ialpha, inv1m;           // lam, 1/alpha, 1/(1 - lam^p)
};

template <typename R> struct CplxArgs {
  const R *in[3];
  R *out[3];
  long long N;      // points per species
  long long st;     // element stride of the swept axis
  long long nlines; // lines of the axis
  long long nx, ny; // grid extents (point index -> node indices)
  int p, nl, nlo_blocks, periodic;
  CTab<R> tab[3];   // P, T, S (gamma = 1, 3, 4)
  const R *cos2[3]; // Schrodinger position term per axis (null: none)
  int dim;
  int rkind;
  R k;
  R rp[3];
};

// F at one node (Section 8): CGL  F = u - (1 + i p0) u |u|^2;
// Schrodinger  F = q J u, J = [[0, 1], [-1, 0]], q = p0 + p1 |u|^2 + p2 (1 - prod cos^2);
// LINEAR  F_i = p0 u_i + p1; ZERO.
template <typename R>
__device__ __forceinline__ C2<R> reaction_c(const CplxArgs<R> &A, C2<R> u, long long g) {
  switch (A.rkind) {
    case ETD_REACTION_LINEAR: return {A.rp[0] * u.x + A.rp[1], A.rp[0] * u.y + A.rp[1]};
    case ETD_REACTION_CGL: {
      const R r = u.x * u.x + u.y * u.y;
      const R ca = u.x - A.rp[0] * u.y, cb = A.rp[0] * u.x + u.y;
      return {u.x - r * ca, u.y - r * cb};
    }
    case ETD_REACTION_NLS: {
      R q = A.rp[0] + A.rp[1] * (u.x * u.x + u.y * u.y);
      if (A.cos2[0]) {
        const long long ix = g % A.nx, iy = (g / A.nx) % A.ny, iz = g / (A.nx * A.ny);
        R c = A.cos2[0][ix];
        if (A.dim >= 2) c *= A.cos2[1][iy];
        if (A.dim == 3) c *= A.cos2[2][iz];
        q += A.rp[2] * (R(1) - c);
      }
      return {q * u.y, -q * u.x};
    }
    default: return {R(0), R(0)};
  }
}

// Warp scans of the chunk recurrences.  Forward: chunk j maps its incoming
// y to y_out = A_j y_in + B_j; lane j needs y_in = the composition of the
// maps of lanes 0 .. j-1 applied to 0.  Backward: x_lo = A_j x_hi + B_j, lane j
// needs x_hi = the composition of lanes j+1 .. 31.  (A_j are the chunk products
// of -l_i and -mu_i, precomputed per axis and pole.)
template <typename R>
__device__ __forceinline__ C2<R> scan_fwd(C2<R> A, C2<R> B, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const C2<R> Ap = shfl_up_c(A, off), Bp = shfl_up_c(B, off);
    if (lane >= off) {
      B = cadd(cmul(A, Bp), B);
      A = cmul(A, Ap);
    }
  }
  C2<R> y = shfl_up_c(B, 1);
  return lane == 0 ? cmk<R>(0, 0) : y;
}
template <typename R>
__device__ __forceinline__ C2<R> scan_bwd(C2<R> A, C2<R> B, int lane) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const C2<R> An = shfl_down_c(A, off), Bn = shfl_down_c(B, off);
    if (lane + off < 32) {
      B = cadd(cmul(A, Bn), B);
      A = cmul(A, An);
    }
  }
  C2<R> x = shfl_down_c(B, 1);
  return lane == 31 ? cmk<R>(0, 0) : x;
}

// Nodes per lane: c = ceil(p/32) rounded up to an odd number, so that the
// 8- or 16-byte slot accesses of the 32 lanes (stride c entries) fall in
// distinct shared-memory banks.
__host__ __device__ __forceinline__ int lane_chunk(int p) { return ((p + 31) >> 5) | 1; }

// C > 0: compile-time bound on the chunk length (loops unrolled, so the table
// and slot loads of a pass issue ahead of the recurrence); C = 0: any length.
#define CHUNK_FWD(t, i) \
  _Pragma("unroll") for (int t = 0; t < (C ? C : c); ++t) \
    if (const int i = lo + t; i < hi)
#define CHUNK_BWD(t, i) \
  _Pragma("unroll") for (int t = (C ? C : c) - 1; t >= 0; --t) \
    if (const int i = lo + t; i < hi)

// Periodic lines on the circulant factorisation M = alpha (I - lam E)(I - lam E^-1)
// (E the cyclic shift, |lam| < 1): M^{-1} b = (1/alpha) z with y_i = b_i + lam y_{i-1}
// and z_i = y_i + lam z_{i+1}, indices cyclic.  Each lane reduces its chunk with a zero
// carry; a warp scan gives the zero-carry prefix and the line's total, and the cyclic
// carry closes it: y_{p-1} = total / (1 - lam^p), so the value entering lane j is
// prefix_j + lam^(nodes before lane j) y_{p-1}; backwards likewise with z_0.
template <typename R>
__device__ __forceinline__ void circ_scan_fwd(C2<R> A, C2<R> B, int lane, C2<R> &ex, C2<R> &tot) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const C2<R> Ap = shfl_up_c(A, off), Bp = shfl_up_c(B, off);
    if (lane >= off) {
      B = cadd(cmul(A, Bp), B);
      A = cmul(A, Ap);
    }
  }
  tot = shfl_c(B, 31);
  ex = shfl_up_c(B, 1);
  if (lane == 0) ex = cmk<R>(0, 0);
}
template <typename R>
__device__ __forceinline__ void circ_scan_bwd(C2<R> A, C2<R> B, int lane, C2<R> &ex, C2<R> &tot) {
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const C2<R> An = shfl_down_c(A, off), Bn = shfl_down_c(B, off);
    if (lane + off < 32) {
      B = cadd(cmul(A, Bn), B);
      A = cmul(A, An);
    }
  }
  tot = shfl_c(B, 0);
  ex = shfl_down_c(B, 1);
  if (lane == 31) ex = cmk<R>(0, 0);
}

// out = ca MA^{-1} srcA + cb MB^{-1} srcB on periodic lines (one chain when NCH = 1:
// out = MA^{-1} srcA, cb and the B arguments unused); st* hold the first recurrence
template <int C, int NCH, typename R>
__device__ __forceinline__ void circ_solve(const CTab<R> &TA, const CTab<R> &TB, int p, const C2<R> *srcA,
                                           C2<R> *stA, const C2<R> *srcB, C2<R> *stB, C2<R> *out, R ca, R cb,
                                           int lane) {
  using CT = C2<R>;
  __syncwarp();
  const int c = lane_chunk(p);
  const int lo = min(p, lane * c), hi = min(p, lo + c);
  const CT lA = TA.lam, lB = TB.lam;
  CT BA = cmk<R>(0, 0), BB = cmk<R>(0, 0);
  CHUNK_FWD(t, i) {
    BA = cadd(srcA[i], cmul(lA, BA));
    if (NCH == 2) BB = cadd(srcB[i], cmul(lB, BB));
  }
  CT ex, tot, yA, yB = cmk<R>(0, 0);
  circ_scan_fwd(ldt(TA.cchunk + lane), BA, lane, ex, tot);
  yA = cadd(ex, cmul(ldt(TA.cpre + lane), cmul(tot, TA.inv1m)));
  if (NCH == 2) {
    circ_scan_fwd(ldt(TB.cchunk + lane), BB, lane, ex, tot);
    yB = cadd(ex, cmul(ldt(TB.cpre + lane), cmul(tot, TB.inv1m)));
  }
  CHUNK_FWD(t, i) {
    const CT a = srcA[i];
    const CT b = NCH == 2 ? srcB[i] : a;
    yA = cadd(a, cmul(lA, yA));
    stA[i] = yA;
    if (NCH == 2) {
      yB = cadd(b, cmul(lB, yB));
      stB[i] = yB;
    }
  }
  BA = cmk<R>(0, 0);
  BB = cmk<R>(0, 0);
  CHUNK_BWD(t, i) {
    BA = cadd(stA[i], cmul(lA, BA));
    if (NCH == 2) BB = cadd(stB[i], cmul(lB, BB));
  }
  CT zA, zB = cmk<R>(0, 0);
  circ_scan_bwd(ldt(TA.cchunk + lane), BA, lane, ex, tot);
  zA = cadd(ex, cmul(ldt(TA.csuf + lane), cmul(tot, TA.inv1m)));
  if (NCH == 2) {
    circ_scan_bwd(ldt(TB.cchunk + lane), BB, lane, ex, tot);
    zB = cadd(ex, cmul(ldt(TB.csuf + lane), cmul(tot, TB.inv1m)));
  }
  const CT sA = cscale(ca, TA.ialpha), sB = cscale(cb, TB.ialpha);
  CHUNK_BWD(t, i) {
    zA = cadd(stA[i], cmul(lA, zA));
    if (NCH == 2) {
      zB = cadd(stB[i], cmul(lB, zB));
      out[i] = cadd(cmul(sA, zA), cmul(sB, zB));
    } else {
      out[i] = cmul(sA, zA);
    }
  }
  __syncwarp();
}

// One complex line solve by one warp, in place: buf = M^{-1} buf.  Lane j
// owns nodes [j c, (j+1) c), c = lane_chunk(p).
template <int C, typename R>
__device__ __forceinline__ void solve1(const CTab<R> &T, int p, int periodic, C2<R> *buf, int lane) {
  using CT = C2<R>;
  if (periodic) {
    circ_solve<C, 1>(T, T, p, buf, buf, buf, buf, buf, R(1), R(0), lane);
    return;
  }
  __syncwarp();
  const int c = lane_chunk(p);
  const int lo = min(p, lane * c), hi = min(p, lo + c);
  CT B = cmk<R>(0, 0);
  CHUNK_FWD(t, i) B = csub(buf[i], cmul(ldt(T.ell + i), B));
  CT y = scan_fwd(ldt(T.af + lane), B, lane);
  CHUNK_FWD(t, i) {
    y = csub(buf[i], cmul(ldt(T.ell + i), y));
    buf[i] = y;
  }
  B = cmk<R>(0, 0);
  CHUNK_BWD(t, i) B = csub(cmul(buf[i], ldt(T.ipv + i)), cmul(ldt(T.mu + i), B));
  CT x = scan_bwd(ldt(T.ab + lane), B, lane);
  CHUNK_BWD(t, i) {
    x = csub(cmul(buf[i], ldt(T.ipv + i)), cmul(ldt(T.mu + i), x));
    buf[i] = x;
  }
  __syncwarp();
}

// Two solves run together (independent chains side by side):
//   out = ca * MA^{-1} srcA + cb * MB^{-1} srcB
// stA / stB hold each chain's intermediate values (stA = srcA and stB = srcB
// allowed, srcA = srcB allowed with distinct stores); out = stA allowed.
// Used for R = 9T - 8S on one right-hand side and for T f1 - S f2.
template <int C, typename R>
__device__ __forceinline__ void solve_pair(const CTab<R> &TA, const CTab<R> &TB, int p, int periodic,
                                           const C2<R> *srcA, C2<R> *stA, const C2<R> *srcB, C2<R> *stB,
                                           C2<R> *out, R ca, R cb, int lane) {
  using CT = C2<R>;
  if (periodic) {
    circ_solve<C, 2>(TA, TB, p, srcA, stA, srcB, stB, out, ca, cb, lane);
    return;
  }
  __syncwarp();
  const int c = lane_chunk(p);
  const int lo = min(p, lane * c), hi = min(p, lo + c);
  CT BA = cmk<R>(0, 0), BB = cmk<R>(0, 0);
  CHUNK_FWD(t, i) {
    BA = csub(srcA[i], cmul(ldt(TA.ell + i), BA));
    BB = csub(srcB[i], cmul(ldt(TB.ell + i), BB));
  }
  CT yA = scan_fwd(ldt(TA.af + lane), BA, lane);
  CT yB = scan_fwd(ldt(TB.af + lane), BB, lane);
  CHUNK_FWD(t, i) {
    const CT a = srcA[i], b = srcB[i];
    yA = csub(a, cmul(ldt(TA.ell + i), yA));
    yB = csub(b, cmul(ldt(TB.ell + i), yB));
    stA[i] = yA;
    stB[i] = yB;
  }
  BA = cmk<R>(0, 0);
  BB = cmk<R>(0, 0);
  CHUNK_BWD(t, i) {
    BA = csub(cmul(stA[i], ldt(TA.ipv + i)), cmul(ldt(TA.mu + i), BA));
    BB = csub(cmul(stB[i], ldt(TB.ipv + i)), cmul(ldt(TB.mu + i), BB));
  }
  CT xA = scan_bwd(ldt(TA.ab + lane), BA, lane);
  CT xB = scan_bwd(ldt(TB.ab + lane), BB, lane);
  CHUNK_BWD(t, i) {
    const CT a = stA[i], b = stB[i];
    xA = csub(cmul(a, ldt(TA.ipv + i)), cmul(ldt(TA.mu + i), xA));
    xB = csub(cmul(b, ldt(TB.ipv + i)), cmul(ldt(TB.mu + i), xB));
    out[i] = cadd(cscale(ca, xA), cscale(cb, xB));
  }
  __syncwarp();
}

template <typename R, int KIND, bool CONTIG, int C>
__global__ void __launch_bounds__(256) cplx_sweep_kernel(const CplxArgs<R> A) {
  using CT = C2<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CT *slot = reinterpret_cast<CT *>(smem_raw);
  const int p = A.p, NL = A.nl;
  const long long N = A.N, st = A.st;
  const int NLp = NL * p;
  // the block's lines: CONTIG rows blockIdx.x * NL + l; strided columns lo0 + l of plane hi
  long long row0 = 0, lo0 = 0, hi = 0;
  if (CONTIG) {
    row0 = (long long)blockIdx.x * NL;
  } else {
    lo0 = (long long)(blockIdx.x % A.nlo_blocks) * NL;
    hi = blockIdx.x / A.nlo_blocks;
  }
  auto base_of = [&](int l, bool &ok) -> long long {
    if (CONTIG) {
      ok = row0 + l < A.nlines;
      return (row0 + l) * p;
    }
    ok = lo0 + l < st;
    return lo0 + l + hi * st * p;
  };
  // staging walk over the block's (line, node) pairs: along x each line's
  // nodes are consecutive threads (one division by p); along y / z the NL (a
  // power of two) neighbouring columns of one node row are (shifts)
  const int lgnl = __ffs(NL) - 1;
  constexpr bool LOADS_U = KIND == SWEEP_FIRST || KIND == CPLX_ONLY;
  constexpr bool ENDS_STEP = KIND == SWEEP_LAST || KIND == CPLX_ONLY;
  const int nin = LOADS_U ? 1 : 3;
  for (int idx = threadIdx.x; idx < NLp; idx += blockDim.x) {
    int l, i;
    if (CONTIG) {
      l = idx / p;
      i = idx - l * p;
    } else {
      l = idx & (NL - 1);
      i = idx >> lgnl;
    }
    bool ok;
    const long long g = base_of(l, ok) + i * st;
    for (int f = 0; f < nin; ++f)
      slot[f * NLp + l * p + i] = ok ? cmk<R>(A.in[f][g], A.in[f][g + N]) : cmk<R>(0, 0);
    if (LOADS_U) {
      // f0 = F(U_n) into slot 1, w* = U_n + k f0 into slot 2
      const CT u = slot[l * p + i];
      const CT f0 = ok ? reaction_c(A, u, g) : cmk<R>(0, 0);
      slot[NLp + l * p + i] = f0;
      slot[2 * NLp + l * p + i] = cadd(u, cscale(A.k, f0));
    }
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const R k = A.k;
  for (int l = warp; l < NL; l += nwarps) {
    bool ok;
    const long long base = base_of(l, ok);
    if (!ok) continue;
    CT *s0 = slot + l * p, *s1 = s0 + NLp, *s2 = s1 + NLp, *s3 = s2 + NLp;
    if (ENDS_STEP) {
      solve1<C>(A.tab[0], p, A.periodic, s2, lane);  // U* = P w
      for (int i = lane; i < p; i += 32) {
        const CT fs = reaction_c(A, s2[i], base + i * st);
        const CT cu = s0[i], cf = s1[i];
        s3[i] = cadd(cadd(cscale(R(9), cu), cscale(R(2) * k, cf)), cscale(k, fs));
        s0[i] = cadd(cadd(cscale(R(8), cu), cscale(R(1.5) * k, cf)), cscale(R(0.5) * k, fs));
      }
      // U_{n+1} = T f1 - S f2 into slot 3
      solve_pair<C>(A.tab[1], A.tab[2], p, A.periodic, s3, s3, s0, s0, s3, R(1), R(-1), lane);
    } else {
      solve1<C>(A.tab[0], p, A.periodic, s2, lane);                                       // w <- P w
      solve_pair<C>(A.tab[1], A.tab[2], p, A.periodic, s0, s0, s0, s3, s0, R(9), R(-8), lane);  // c_U <- R c_U
      solve_pair<C>(A.tab[1], A.tab[2], p, A.periodic, s1, s1, s1, s3, s1, R(9), R(-8), lane);  // c_f <- R c_f
    }
    __syncwarp();
  }
  __syncthreads();
  const int nout = ENDS_STEP ? 1 : 3;
  for (int idx = threadIdx.x; idx < NLp; idx += blockDim.x) {
    int l, i;
    if (CONTIG) {
      l = idx / p;
      i = idx - l * p;
    } else {
      l = idx & (NL - 1);
      i = idx >> lgnl;
    }
    bool ok;
    const long long g = base_of(l, ok) + i * st;
    if (!ok) continue;
    for (int f = 0; f < nout; ++f) {
      const CT v = slot[(ENDS_STEP ? 3 : f) * NLp + l * p + i];
      A.out[f][g] = v.x;
      A.out[f][g + N] = v.y;
    }
  }
}

// ------------------------------------------------------------------ host

using cd = std::complex<double>;

// Complex Thomas tables of M = I + c B (h^2 B_p of Example 1) for a Dirichlet
// or Neumann line, Section 7's LU without pivoting.
struct HostCplxTab {
  std::vector<cd> ell, ipv, mu;
};

HostCplxTab cplx_tables(int p, int bc, cd c) {
  std::vector<cd> sub(p, -c), dg(p, 1.0 + 2.0 * c), sup(p, -c);
  sub[0] = 0;
  sup[p - 1] = 0;
  if (bc == ETD_BC_NEUMANN) {
    sup[0] = -2.0 * c;
    sub[p - 1] = -2.0 * c;
  }
  HostCplxTab T;
  T.ell.assign(p, 0);
  T.ipv.assign(p, 0);
  T.mu.assign(p, 0);
  cd piv = dg[0];
  for (int i = 0; i < p; ++i) {
    if (i > 0) {
      T.ell[i] = sub[i] / piv;
      piv = dg[i] - T.ell[i] * sup[i - 1];
    }
    T.ipv[i] = 1.0 / piv;
    T.mu[i] = sup[i] / piv;
  }
  return T;
}

template <typename R>
const void *upload_c(Instance &I, const std::vector<cd> &v, cudaError_t &err) {
  std::vector<R> h(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    h[2 * i] = (R)v[i].real();
    h[2 * i + 1] = (R)v[i].imag();
  }
  return I.arena.put(h.data(), h.size() * sizeof(R), err);
}

template <typename R>
etd_status build_cplx_axis(etd_ctx *ctx, Instance &I, int a) {
  CplxAxis &X = I.cax[a];
  const int p = (int)I.n[a];
  const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
  static const double gammas[3] = {1.0, 3.0, 4.0};
  cudaError_t err = cudaSuccess;
  for (int gi = 0; gi < 3; ++gi) {
    const cd c = (I.k / gammas[gi]) * cd(I.dcp, I.dcq) / (h * h);
    CplxTabDev &D = X.tab[gi];
    const int cc = lane_chunk(p);  // nodes per lane (lane j: [j cc, (j+1) cc))
    if (I.bc[a] != ETD_BC_PERIODIC) {
      const HostCplxTab T = cplx_tables(p, I.bc[a], c);
      D.ell = upload_c<R>(I, T.ell, err);
      D.ipv = upload_c<R>(I, T.ipv, err);
      D.mu = upload_c<R>(I, T.mu, err);
      // chunk products of the warp scans
      std::vector<cd> af(32, 1.0), ab(32, 1.0);
      for (int j = 0; j < 32; ++j)
        for (int i = j * cc; i < std::min(p, (j + 1) * cc); ++i) {
          af[j] *= -T.ell[i];
          ab[j] *= -T.mu[i];
        }
      D.af = upload_c<R>(I, af, err);
      D.ab = upload_c<R>(I, ab, err);
    } else {
      // circulant factorisation of the cyclic line matrix (1 + 2c) I - c (E + E^-1):
      // alpha (1 + lam^2) = 1 + 2c, alpha lam = c, i.e. lam + 1/lam = 2 + 1/c, |lam| < 1.
      // The two roots multiply to 1: take the larger one without cancellation
      // (b + sqrt(b^2 - 4) with the root's sign aligned to b) and invert it.
      const cd bq = 2.0 + 1.0 / c;
      cd disc = std::sqrt(bq * bq - 4.0);
      if (std::abs(bq - disc) > std::abs(bq + disc)) disc = -disc;
      const cd lam = 2.0 / (bq + disc);
      const cd alpha = c / lam;
      std::vector<cd> pre(32, 1.0), suf(32, 1.0), chk(32, 1.0);
      for (int j = 0; j < 32; ++j) {
        const int lo = std::min(p, j * cc), hi = std::min(p, lo + cc);
        pre[j] = std::pow(lam, lo);
        suf[j] = std::pow(lam, p - hi);
        chk[j] = std::pow(lam, hi - lo);
      }
      D.cpre = upload_c<R>(I, pre, err);
      D.csuf = upload_c<R>(I, suf, err);
      D.cchunk = upload_c<R>(I, chk, err);
      const cd ia = 1.0 / alpha, i1m = 1.0 / (1.0 - std::pow(lam, p));
      D.lam[0] = lam.real();
      D.lam[1] = lam.imag();
      D.ialpha[0] = ia.real();
      D.ialpha[1] = ia.imag();
      D.inv1m[0] = i1m.real();
      D.inv1m[1] = i1m.imag();
    }
  }
  if (I.rkind == ETD_REACTION_NLS && I.rp[2] != 0.0) {
    std::vector<R> c2(p);
    for (int i = 0; i < p; ++i) {
      const double x = (I.bc[a] == ETD_BC_DIRICHLET ? i + 1 : i) * h;
      const double cv = std::cos(M_PI * x / I.length[a]);
      c2[i] = (R)(cv * cv);
    }
    X.cos2 = I.arena.put(c2.data(), c2.size() * sizeof(R), err);
  }
  if (err != cudaSuccess) return cuda_fail(ctx, err, "complex line tables");
  return ETD_OK;
}

constexpr size_t kCplxSmemCap = 200 * 1024;

// Lines per block (a power of two): at most what fits the shared-memory cap
// and 8 (one line per warp of a 256-thread block, so that 4 blocks -- 32
// warps -- share an SM when their slots fit; along y / z the 8 columns are
// 8-node contiguous runs); then halved while the sweep would have fewer than 2 blocks per SM
// (each line is one warp's serial work, so small grids need small blocks to
// spread over the SMs), and along y / z while a partial last column group
// would leave more than 1/8 of its lines idle.
bool plan_cplx_axis(Instance &I, int a) {
  CplxAxis &X = I.cax[a];
  const int p = (int)I.n[a];
  const size_t per_line = 4 * (size_t)p * 2 * I.real_bytes;
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  const long long nlines = I.N / p;
  const int cap_lines = 8;
  const size_t fit = kCplxSmemCap / per_line;
  if (fit < 1) return false;
  int nl = 1;
  while (nl * 2 <= cap_lines && (size_t)(nl * 2) <= fit) nl *= 2;
  auto blocks_of = [&](int v) -> long long {
    return a == 0 ? (nlines + v - 1) / v : ((st + v - 1) / v) * (nlines / st);
  };
  while (nl > 1 && blocks_of(nl) < 2 * 152) nl /= 2;
  if (a > 0)
    while (nl > 1 && ((st + nl - 1) / nl) * nl - st > st / 8) nl /= 2;
  X.nl = nl;
  X.nthreads = 32 * std::min(nl, 8);
  X.chunk = lane_chunk(p);
  X.smem = per_line * nl;
  if (a == 0) {
    X.nlo_blocks = 1;
    X.nblocks = (int)((nlines + nl - 1) / nl);
  } else {
    X.nlo_blocks = (int)((st + nl - 1) / nl);
    X.nblocks = (int)(X.nlo_blocks * (nlines / st));
  }
  return true;
}

// compile-time chunk bound of a plan: the smallest of 4, 8, 16 that holds
// ceil(p/32) nodes, else 0 (runtime loops)
int chunk_bound(int c) { return c <= 4 ? 4 : c <= 8 ? 8 : c <= 16 ? 16 : 0; }

template <typename R, int KIND, bool CONTIG>
cudaError_t set_cplx_smem_attr() {
  const int mx = 227 * 1024;
  cudaError_t e = cudaFuncSetAttribute(cplx_sweep_kernel<R, KIND, CONTIG, 4>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cplx_sweep_kernel<R, KIND, CONTIG, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cplx_sweep_kernel<R, KIND, CONTIG, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(cplx_sweep_kernel<R, KIND, CONTIG, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  return e;
}

template <typename R>
cudaError_t set_cplx_attrs() {
  cudaError_t e = set_cplx_smem_attr<R, SWEEP_FIRST, true>();
  if (e == cudaSuccess) e = set_cplx_smem_attr<R, SWEEP_MIDDLE, false>();
  if (e == cudaSuccess) e = set_cplx_smem_attr<R, SWEEP_LAST, false>();
  if (e == cudaSuccess) e = set_cplx_smem_attr<R, CPLX_ONLY, true>();
  return e;
}

template <typename R, int KIND, bool CONTIG>
void launch_cplx(const CplxArgs<R> &A, const CplxAxis &X, cudaStream_t s) {
  const dim3 grid(X.nblocks), block(X.nthreads);
  switch (chunk_bound(X.chunk)) {
    case 4: cplx_sweep_kernel<R, KIND, CONTIG, 4><<<grid, block, X.smem, s>>>(A); break;
    case 8: cplx_sweep_kernel<R, KIND, CONTIG, 8><<<grid, block, X.smem, s>>>(A); break;
    case 16: cplx_sweep_kernel<R, KIND, CONTIG, 16><<<grid, block, X.smem, s>>>(A); break;
    default: cplx_sweep_kernel<R, KIND, CONTIG, 0><<<grid, block, X.smem, s>>>(A); break;
  }
}

template <typename R>
cudaError_t cplx_step_t(const Instance &I, R *U, double t, cudaStream_t s, etd_ctx *prof) {
  (void)t;  // the coupled reactions are autonomous
  R *cu = (R *)I.scratch[0], *cf = (R *)I.scratch[1], *w = (R *)I.scratch[2];
  for (int a = 0; a < I.dim; ++a) {
    const CplxAxis &X = I.cax[a];
    const int kind = I.dim == 1 ? CPLX_ONLY : a == 0 ? SWEEP_FIRST : (a == I.dim - 1 ? SWEEP_LAST : SWEEP_MIDDLE);
    CplxArgs<R> A{};
    if (kind == CPLX_ONLY) {
      A.in[0] = U;
      A.out[0] = U;
    } else if (kind == SWEEP_FIRST) {
      A.in[0] = U;
      A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
    } else if (kind == SWEEP_MIDDLE) {
      A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
      A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
    } else {
      A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
      A.out[0] = U;
    }
    A.N = I.N;
    long long st = 1;
    for (int b = 0; b < a; ++b) st *= I.n[b];
    A.st = st;
    A.nlines = I.N / I.n[a];
    A.nx = I.n[0];
    A.ny = I.n[1];
    A.p = (int)I.n[a];
    A.nl = X.nl;
    A.nlo_blocks = X.nlo_blocks;
    A.periodic = I.bc[a] == ETD_BC_PERIODIC;
    for (int g = 0; g < 3; ++g) {
      const CplxTabDev &D = X.tab[g];
      A.tab[g] = CTab<R>{(const C2<R> *)D.ell, (const C2<R> *)D.ipv, (const C2<R> *)D.mu,
                         (const C2<R> *)D.af, (const C2<R> *)D.ab,
                         (const C2<R> *)D.cpre, (const C2<R> *)D.csuf, (const C2<R> *)D.cchunk,
                         C2<R>{(R)D.lam[0], (R)D.lam[1]}, C2<R>{(R)D.ialpha[0], (R)D.ialpha[1]},
                         C2<R>{(R)D.inv1m[0], (R)D.inv1m[1]}};
    }
    for (int b = 0; b < 3; ++b) A.cos2[b] = (const R *)I.cax[b].cos2;
    for (int b = 0; b < I.dim; ++b)
      if (!A.cos2[b]) A.cos2[0] = nullptr;  // no position term
    A.dim = I.dim;
    A.rkind = I.rkind;
    A.k = (R)I.k;
    for (int j = 0; j < 3; ++j) A.rp[j] = (R)I.rp[j];
    cudaEvent_t ev0;
    cudaError_t e = prof_begin(prof, s, ev0);
    if (e != cudaSuccess) return e;
    if (kind == CPLX_ONLY) launch_cplx<R, CPLX_ONLY, true>(A, X, s);
    else if (kind == SWEEP_FIRST) launch_cplx<R, SWEEP_FIRST, true>(A, X, s);
    else if (kind == SWEEP_MIDDLE) launch_cplx<R, SWEEP_MIDDLE, false>(A, X, s);
    else launch_cplx<R, SWEEP_LAST, false>(A, X, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = prof_end(prof, s, kind == CPLX_ONLY ? SWEEP_LAST : kind, ev0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace

namespace etd {

cudaError_t cplx_step(const Instance &I, void *U, double t, cudaStream_t s, etd_ctx *prof) {
  if (I.real_bytes == 8) return cplx_step_t<double>(I, (double *)U, t, s, prof);
  return cplx_step_t<float>(I, (float *)U, t, s, prof);
}

}  // namespace etd

extern "C" etd_status etd_create_coupled(const etd_grid *grid, const double *Dm, const etd_reaction *reaction,
                                         double k, int32_t precision, void *stream, etd_ctx **out) {
  if (!out) return fail(nullptr, ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!grid || !Dm || !reaction) return fail(nullptr, ETD_ERR_INVALID_ARG, "null grid, Dm or reaction");
  for (int j = 0; j < 4; ++j)
    if (!std::isfinite(Dm[j])) return fail(nullptr, ETD_ERR_INVALID_ARG, "Dm[%d] not finite", j);
  if (reaction->nspecies != 2) return fail(nullptr, ETD_ERR_INVALID_ARG, "coupled diffusion needs nspecies = 2");
  if (!(Dm[0] >= 0)) return fail(nullptr, ETD_ERR_INVALID_ARG, "Dm[0] (the real part p) must be >= 0");
  if (Dm[0] != Dm[3] || Dm[1] != -Dm[2])
    return fail(nullptr, ETD_ERR_UNSUPPORTED, "the kernels take Dm = [[p, -q], [q, p]] (complex p + i q) only");
  const int kind = reaction->kind;
  if (kind != ETD_REACTION_ZERO && kind != ETD_REACTION_LINEAR && kind != ETD_REACTION_CGL &&
      kind != ETD_REACTION_NLS)
    return fail(nullptr, ETD_ERR_UNSUPPORTED, "coupled diffusion takes the ZERO, LINEAR, CGL or NLS reaction");
  // grid, k, precision and parameters as for etd_create; d = 1 is taken here
  // too (one line: the frame without splitting)
  etd_reaction rz = *reaction;
  rz.kind = ETD_REACTION_ZERO;
  const double Dd[2] = {Dm[0], Dm[0]};
  etd_grid g2 = *grid;
  if (grid->dim == 1) {  // validate axis 0 inside a 2D grid with a minimal second axis
    g2.dim = 2;
    g2.n[1] = 3;
    g2.bc[1] = ETD_BC_NEUMANN;
    g2.length[1] = 1.0;
  }
  etd_status st = validate_problem(&g2, Dd, &rz, k, precision);
  if (st != ETD_OK) return st;
  etd_ctx *ctx = new (std::nothrow) etd_ctx();
  if (!ctx) return fail(nullptr, ETD_ERR_OOM, "host allocation failed");
  ctx->stream = (cudaStream_t)stream;
  ctx->precision = precision;
  ctx->inst.resize(1);
  Instance &I = ctx->inst[0];
  auto abort_create = [&](etd_status s2) {
    std::string msg = ctx->err;
    etd_destroy(ctx);
    return fail(nullptr, s2, "%s", msg.c_str());
  };
  I.dim = grid->dim;
  I.N = 1;
  for (int a = 0; a < 3; ++a) {
    I.n[a] = a < I.dim ? grid->n[a] : 1;
    I.bc[a] = a < I.dim ? grid->bc[a] : 0;
    I.length[a] = a < I.dim ? grid->length[a] : 1.0;
    I.N *= I.n[a];
  }
  I.S = 2;
  I.D[0] = I.D[1] = Dm[0];
  I.k = k;
  I.rkind = kind;
  for (int j = 0; j < 8; ++j) I.rp[j] = reaction->params[j];
  I.real_bytes = precision == ETD_FP64 ? 8 : 4;
  I.coupled = true;
  I.dcp = Dm[0];
  I.dcq = Dm[2];
  for (int a = 0; a < I.dim; ++a) {
    if (!plan_cplx_axis(I, a)) {
      fail(ctx, ETD_ERR_UNSUPPORTED, "axis %d: a complex line of %lld nodes does not fit shared memory", a,
           (long long)I.n[a]);
      return abort_create(ETD_ERR_UNSUPPORTED);
    }
    st = I.real_bytes == 8 ? build_cplx_axis<double>(ctx, I, a) : build_cplx_axis<float>(ctx, I, a);
    if (st != ETD_OK) return abort_create(st);
  }
  cudaError_t e = I.real_bytes == 8 ? set_cplx_attrs<double>() : set_cplx_attrs<float>();
  if (e != cudaSuccess) {
    cuda_fail(ctx, e, "complex kernel attributes");
    return abort_create(ETD_ERR_CUDA);
  }
  const size_t bytes = (size_t)2 * I.N * I.real_bytes;
  for (int f = 0; f < 3; ++f) {
    e = cudaMalloc(&I.scratch[f], bytes);
    if (e != cudaSuccess) {
      fail(ctx, ETD_ERR_OOM, "scratch allocation of %zu bytes failed", bytes);
      return abort_create(ETD_ERR_OOM);
    }
    I.owned.push_back(I.scratch[f]);
  }
  *out = ctx;
  return ETD_OK;
}
