// etd_adjoint.cuh -- reverse-mode (discrete adjoint) sweeps of one ETD-RDP-IF
// step and the misfit kernel.
//
// The forward step is a composition of line solves x = M^{-1} b with
// M = I + (k/gamma) D_s B (Section 7) and pointwise operations (Section 6
// frame).  Its adjoint, axis by axis in reverse order:
//   x = M^{-1} b         ->  bbar += M^{-T} xbar              (transposed tables)
//                            Dbar_s -= <M^{-T} xbar, b - x> / D_s
//                            (since (k/gamma) B x = (b - x) / D_s)
//   f = F(u)             ->  ubar += J_F(u)^T fbar, pbar += (dF/dp)^T fbar
//   linear combinations  ->  transposed combinations
// Each adjoint sweep recomputes the forward solves of its axis from the
// forward inputs of that sweep (kept by the caller), so every line solve of
// the step appears twice: forward (for the D-gradient) and transposed.
//
// Block layout: one block owns nlb complete lines; thread (l = tid % nlb,
// j = tid / nlb) owns chunk j of line l for every species in registers; all
// solves of a phase share one shared-memory exchange (etd_sweep.cuh).
#pragma once

#include "etd_sweep.cuh"

namespace etd {

// J_F(u)^T yb and (dF/dparams)^T yb at one point (q: manufactured-source
// factor e^{-t} prod sin(pi x/L) at the point, 0 if the source is off)
template <typename R, int S>
__device__ __forceinline__ void reaction_vjp(const SweepArgs<R> &A, const R (&u)[S], const R (&yb)[S], R (&out)[S],
                                             R (&pg)[8], R q) {
#pragma unroll
  for (int s = 0; s < S; ++s) out[s] = R(0);
  switch (A.rkind) {
    case 1: {  // F_i = p0 u_i + p1
      const R p0 = (R)A.rp[0];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        out[s] = p0 * yb[s];
        pg[0] = fma(u[s], yb[s], pg[0]);
        pg[1] += yb[s];
      }
      return;
    }
    case 2:
      if constexpr (S == 2) {  // Brusselator
        const R b = (R)A.rp[1], U = u[0], V = u[1];
        const R uv2 = R(2) * U * V, uu = U * U;
        out[0] = (uv2 - (b + R(1))) * yb[0] + (b - uv2) * yb[1];
        out[1] = uu * (yb[0] - yb[1]);
        pg[0] += yb[0];
        pg[1] = fma(U, yb[1] - yb[0], pg[1]);
      }
      return;
    case 3:
      if constexpr (S == 2) {  // Schnakenberg
        const R a = (R)A.rp[0], b = (R)A.rp[1], g = (R)A.rp[2], U = u[0], V = u[1];
        const R uv2 = R(2) * U * V, uu = U * U, uuv = uu * V;
        out[0] = g * ((uv2 - R(1)) * yb[0] - uv2 * yb[1]);
        out[1] = g * uu * (yb[0] - yb[1]);
        pg[0] = fma(g, yb[0], pg[0]);
        pg[1] = fma(g, yb[1], pg[1]);
        pg[2] += (a - U + uuv) * yb[0] + (b - uuv) * yb[1];
      }
      return;
    case 4:
      if constexpr (S == 2) {  // Gray-Scott
        const R F = (R)A.rp[0], kap = (R)A.rp[1], U = u[0], V = u[1];
        const R vv = V * V, uv2 = R(2) * U * V;
        out[0] = (-vv - F) * yb[0] + vv * yb[1];
        out[1] = -uv2 * yb[0] + (uv2 - (F + kap)) * yb[1];
        pg[0] += (R(1) - U) * yb[0] - V * yb[1];
        pg[1] -= V * yb[1];
      }
      return;
    case 6:
      if constexpr (S == 2) {  // CGL (alpha = 0): F = u - (1 + i beta) u |u|^2, r = |u|^2
        const R beta = (R)A.rp[0], a = u[0], b = u[1];
        const R r = a * a + b * b, ca = a - beta * b, cb = beta * a + b;
        out[0] = (R(1) - r - R(2) * a * ca) * yb[0] + (-beta * r - R(2) * a * cb) * yb[1];
        out[1] = (beta * r - R(2) * b * ca) * yb[0] + (R(1) - r - R(2) * b * cb) * yb[1];
        pg[0] += r * (b * yb[0] - a * yb[1]);
      }
      return;
    case 5: {  // enzyme kinetics + manufactured source
      const R d = R(1) + u[0];
      out[0] = -rdiv(yb[0], d * d);
      if (q != R(0)) {
        const R lf = (R)A.src_lf;
        pg[0] += (((R)A.rp[1] * lf - R(1)) * q + rdiv(q, R(1) + q)) * yb[0];
        pg[1] += (R)A.rp[0] * lf * q * yb[0];
      }
      return;
    }
    default:
      return;
  }
}

// manufactured-source factor q at grid point pidx
template <typename R>
__device__ __forceinline__ R mms_q(const SweepArgs<R> &A, long long pidx) {
  const long long x = pidx % A.nx;
  const long long r = pidx / A.nx;
  const long long y = r % A.ny;
  const long long z = r / A.ny;
  R q = (R)A.exp_mt * A.phi[0][x] * A.phi[1][y];
  if (A.phi[2]) q *= A.phi[2][z];
  return q;
}

// chain the chunk summaries of solves q0 .. q0+nq-1; mat(q) gives the solve's tables
// Line-solve passes of the adjoint sweeps: FP64 keeps the operation order of
// Section 7 (pass1 / pass2), FP32 uses the coefficient rows and the one-FMA
// forward chain of the forward sweeps (pass1v / pass2v).
template <typename R, int L>
__device__ __forceinline__ void apass1(const MatTab<R> &M, int m, int j, const R (&b)[L], R &F, R &Y) {
  if constexpr (sizeof(R) == 8) pass1<R, L>(M, m, j, b, F, Y);
  else pass1v<R, L>(M, m, j, b, F, Y);
}
template <typename R, int L>
__device__ __forceinline__ void apass1x2(const MatTab<R> &M, int m, int j, const R (&b0)[L], const R (&b1)[L], R &F0,
                                         R &Y0, R &F1, R &Y1) {
  if constexpr (sizeof(R) == 8) pass1x2<R, L>(M, m, j, b0, b1, F0, Y0, F1, Y1);
  else pass1x2v<R, L>(M, m, j, b0, b1, F0, Y0, F1, Y1);
}
template <typename R, int L>
__device__ __forceinline__ void apass2(const MatTab<R> &M, int m, int j, const R (&b)[L], R G, R X, R sg, R (&x)[L]) {
  if constexpr (sizeof(R) == 8) {
    pass2<R, L>(M, m, j, b, G, X, sg, x);
  } else {
    Carry<R> c;
    c.G = G;
    c.X = X;
    c.ns = -sg;
    pass2v<R, L>(M, m, j, b, c, x, [&](int t, R v) { x[t] = v; });
  }
}
// (the Sherman-Morrison scalars are formed in FP64 and stored in the sweep's precision)
template <typename R, typename GetMat>
__device__ __forceinline__ void scan_solves(const SweepArgs<R> &A, R *sF, R *sY, R *sSig, int q0, int nq,
                                            GetMat mat) {
  const int m = A.m, nlb = A.nlb, pitch = A.pitch;
  if (m > 32) {
    scan_lines_warp<R, R, 1, R>(A, sF, sY, sSig, q0, nq, mat);
    return;
  }
  for (int u = threadIdx.x; u < nlb * nq; u += blockDim.x) {
    const int l = u % nlb;
    const int q = q0 + u / nlb;
    const MatTab<R> &M = mat(q);
    R *F = sF + (q * nlb + l) * pitch;  // 32-bit shared-memory offsets
    R *Y = sY + (q * nlb + l) * pitch;
    R G, X;
    chain_line<R, R>(M, F, Y, m, 0, R(0), R(0), G, X);
    put_sigma(sSig + q * nlb + l, M, X, G);
  }
}

// block-wide sum of NV per-thread values, written to this block's slot
// part[blockIdx.x * NV + i] (reduce_partials adds the slots to the
// accumulators in a fixed order, so repeated runs give identical sums)
template <int NV>
__device__ __forceinline__ void block_accumulate(double (&v)[NV], double *part, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_xor_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[warp * NV + i] = v[i];
  __syncthreads();
  if (threadIdx.x < NV) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += red[w * NV + threadIdx.x];
    part[(size_t)blockIdx.x * NV + threadIdx.x] = s;
  }
}

// acc[i] += sum_b part[b * nv + i] for i < nv: warp i adds the slots in a
// fixed order (lane-strided partial sums, then a fixed shuffle tree)
static __global__ void __launch_bounds__(32 * (MAX_SPECIES + 8)) reduce_partials_kernel(const double *__restrict__ part,
                                                                                 int nblocks, int nv, double *acc) {
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (i >= nv) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += part[(size_t)b * nv + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) acc[i] += s;
}

// CIRC: periodic axis on the circulant factorisation (A.cl), else the line tables
template <typename R, int S, int L, bool CONTIG, int KIND, bool CIRC = false>
__global__ void __launch_bounds__(ETD_MAX_THREADS) adjoint_kernel(const __grid_constant__ SweepArgs<R> A) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int NQ = (KIND == ADJ_LAST) ? 6 * S : 10 * S;
  const int m = A.m, nlb = A.nlb, pitch = A.pitch, n = A.n;
  const int tid = threadIdx.x;
  const int l = tid % nlb, j = tid / nlb;
  long long base;
  bool line_ok;
  if constexpr (CONTIG) {
    const long long line = (long long)blockIdx.x * nlb + l;
    line_ok = line < A.nlines;
    base = line * n;
  } else {
    const long long lo = (long long)(blockIdx.x % A.nlo_blocks) * nlb + l;
    const long long hi = blockIdx.x / A.nlo_blocks;
    line_ok = lo < A.st;
    base = lo + hi * A.st * n;
  }
  const long long st = CONTIG ? 1 : A.st;
  const int i0 = j * L;
  const int cnt = line_ok ? max(0, min(L, n - i0)) : 0;
  const long long off0 = base + (long long)i0 * st;
  const long long N = A.N;
  const R k = (R)A.k;

  R *sF = reinterpret_cast<R *>(smem);
  R *sY = sF + NQ * nlb * pitch;
  unsigned char *sig_base = smem + ((2 * NQ * nlb * pitch * (int)sizeof(R) + 15) & ~15);
  R *sSig = reinterpret_cast<R *>(sig_base);  // NQ * nlb scalars (8-byte slots reserved)
  double *red = reinterpret_cast<double *>(sig_base) + NQ * nlb;
  const int myidx = l * pitch + j;  // 32-bit shared-memory offsets
  const int qstride = nlb * pitch;
  auto put = [&](int q, R F, R Y) {
    sF[q * qstride + myidx] = F;
    sY[q * qstride + myidx] = Y;
  };
  auto carries = [&](int q, R &G, R &X, R &sg) {
    G = sF[q * qstride + myidx];
    X = sY[q * qstride + myidx];
    sg = sSig[q * nlb + l];
  };
  // solve q with table M (CIRC: the circulant coefficients cl(q)): summaries,
  // and the solution from the carries
  auto pass1q = [&](int q, const MatTab<R> &M, const typename SweepArgs<R>::CircLine &C, const R (&b)[L]) {
    R F, Y;
    if constexpr (CIRC) cpass1<R, L>(C, b, F, Y);
    else apass1<R, L>(M, m, j, b, F, Y);
    put(q, F, Y);
  };
  auto pass1x2q = [&](int q0, int q1, const MatTab<R> &M, const typename SweepArgs<R>::CircLine &C,
                      const R (&b0)[L], const R (&b1)[L]) {
    R F0, Y0, F1, Y1;
    if constexpr (CIRC) {
      cpass1<R, L>(C, b0, F0, Y0);
      cpass1<R, L>(C, b1, F1, Y1);
    } else {
      apass1x2<R, L>(M, m, j, b0, b1, F0, Y0, F1, Y1);
    }
    put(q0, F0, Y0);
    put(q1, F1, Y1);
  };
  auto pass2q = [&](int q, const MatTab<R> &M, const typename SweepArgs<R>::CircLine &C, const R (&b)[L],
                    R (&x)[L]) {
    R G, X, sg;
    carries(q, G, X, sg);
    if constexpr (CIRC) cpass2<R, L>(C, b, G, X, x);
    else apass2<R, L>(M, m, j, b, G, X, sg, x);
  };
  auto qsrc = [&](int t) -> R {
    return (A.phi[0] != nullptr && t < cnt) ? mms_q(A, off0 + (long long)t * st) : R(0);
  };
  R dD[S];
  R pg[8];
#pragma unroll
  for (int s = 0; s < S; ++s) dD[s] = R(0);
#pragma unroll
  for (int i = 0; i < 8; ++i) pg[i] = R(0);
  // -<lam, b - x>: contribution of one solve to D_s (times 1/D_s at the end)
  auto dterm = [&](int s, const R (&lam)[L], const R (&b)[L], const R (&x)[L], R scale) {
    R acc = R(0);
#pragma unroll
    for (int t = 0; t < L; ++t) acc = fma(lam[t], b[t] - x[t], acc);
    dD[s] = fma(-scale, acc, dD[s]);
  };

  if constexpr (KIND == ADJ_LAST) {
    // forward inputs of the last sweep: c_U, c_f, w (fin); adjoint input: Ubar_{n+1} (in[0])
    // solves: phase A  q = 3s: P w ; 3s+1: T^T Ub ; 3s+2: S^T Ub
    //         phase B  q = 3S+3s: T f1 ; +1: S f2 ; +2: P^T Ustar_bar
    auto mat = [&](int q) -> const MatTab<R> & {
      const int qq = q < 3 * S ? q : q - 3 * S;
      const int s = qq / 3, r = qq - 3 * (qq / 3);
      if (q < 3 * S) return r == 0 ? A.mat[s][0] : A.matT[s][r];
      return r == 2 ? A.matT[s][0] : A.mat[s][r + 1];
    };
    auto cid = [&](int q) -> int {  // species * 3 + (0: P, 1: T, 2: S) of solve q
      const int qq = q < 3 * S ? q : q - 3 * S;
      const int s = qq / 3, r = qq - 3 * (qq / 3);
      return s * 3 + (q < 3 * S ? r : (r == 2 ? 0 : r + 1));
    };
    R w[S][L], Us[S][L], a1[S][L], a2[S][L];
    {
      R ub[S][L];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        load_chunk<R, L, CONTIG>(w[s], A.fin[2] + s * N, off0, st, cnt);
        load_chunk<R, L, CONTIG>(ub[s], A.in[0] + s * N, off0, st, cnt);
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        pass1q(3 * s, A.mat[s][0], A.cl[s][0], w[s]);
        pass1q(3 * s + 1, A.matT[s][1], A.cl[s][1], ub[s]);
        pass1q(3 * s + 2, A.matT[s][2], A.cl[s][2], ub[s]);
      }
      __syncthreads();
      if constexpr (CIRC) circ_chains<R>(A, sF, sY, 0, 3 * S, cid);
      else scan_solves<R>(A, sF, sY, sSig, 0, 3 * S, mat);
      __syncthreads();
#pragma unroll
      for (int s = 0; s < S; ++s) {
        pass2q(3 * s, A.mat[s][0], A.cl[s][0], w[s], Us[s]);
        pass2q(3 * s + 1, A.matT[s][1], A.cl[s][1], ub[s], a1[s]);
        pass2q(3 * s + 2, A.matT[s][2], A.cl[s][2], ub[s], a2[s]);
#pragma unroll
        for (int t = 0; t < L; ++t) a2[s][t] = -a2[s][t];  // f2bar = S^T (-Ubar)
      }
    }
    // pointwise: fstar_bar = k f1bar + k/2 f2bar, Ustar_bar = J^T fstar_bar,
    // c_U_bar = 9 f1bar + 8 f2bar, c_f_bar = 2k f1bar + 3k/2 f2bar, f1, f2 for the D-gradient
    R f1[S][L], f2[S][L], usb[S][L];
    {
      R cu[S][L], cf[S][L];
#pragma unroll
      for (int s = 0; s < S; ++s) {
        load_chunk<R, L, CONTIG>(cu[s], A.fin[0] + s * N, off0, st, cnt);
        load_chunk<R, L, CONTIG>(cf[s], A.fin[1] + s * N, off0, st, cnt);
      }
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], f[S], yb[S], ob[S];
        const R q = qsrc(t);
        const R src = (q != R(0)) ? (R)A.rp[0] * (((R)A.rp[1] * (R)A.src_lf - R(1)) * q + rdiv(q, R(1) + q)) : R(0);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          u[s] = Us[s][t];
          yb[s] = (t < cnt) ? fma(k, a1[s][t], R(0.5) * k * a2[s][t]) : R(0);
        }
        reaction_point<R, S>(A, u, f, src);
        reaction_vjp<R, S>(A, u, yb, ob, pg, q);
#pragma unroll
        for (int s = 0; s < S; ++s) {
          usb[s][t] = (t < cnt) ? ob[s] : R(0);
          const R fs = (t < cnt) ? f[s] : R(0);
          f1[s][t] = fma(R(9), cu[s][t], fma(R(2) * k, cf[s][t], k * fs));
          f2[s][t] = fma(R(8), cu[s][t], fma(R(1.5) * k, cf[s][t], R(0.5) * k * fs));
          cu[s][t] = fma(R(9), a1[s][t], R(8) * a2[s][t]);
          cf[s][t] = fma(R(2) * k, a1[s][t], R(1.5) * k * a2[s][t]);
        }
      }
#pragma unroll
      for (int s = 0; s < S; ++s) {
        store_chunk<R, L, CONTIG>(cu[s], A.out[0] + s * N, off0, st, cnt);
        store_chunk<R, L, CONTIG>(cf[s], A.out[1] + s * N, off0, st, cnt);
      }
    }
#pragma unroll
    for (int s = 0; s < S; ++s) {
      pass1q(3 * S + 3 * s, A.mat[s][1], A.cl[s][1], f1[s]);
      pass1q(3 * S + 3 * s + 1, A.mat[s][2], A.cl[s][2], f2[s]);
      pass1q(3 * S + 3 * s + 2, A.matT[s][0], A.cl[s][0], usb[s]);
    }
    __syncthreads();
    if constexpr (CIRC) circ_chains<R>(A, sF, sY, 3 * S, 3 * S, cid);
    else scan_solves<R>(A, sF, sY, sSig, 3 * S, 3 * S, mat);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R x[L];
      pass2q(3 * S + 3 * s, A.mat[s][1], A.cl[s][1], f1[s], x);
      dterm(s, a1[s], f1[s], x, R(1));
      pass2q(3 * S + 3 * s + 1, A.mat[s][2], A.cl[s][2], f2[s], x);
      dterm(s, a2[s], f2[s], x, R(1));
      pass2q(3 * S + 3 * s + 2, A.matT[s][0], A.cl[s][0], usb[s], x);  // wbar
      dterm(s, x, w[s], Us[s], R(1));
      store_chunk<R, L, CONTIG>(x, A.out[2] + s * N, off0, st, cnt);
    }
  } else {
    // FIRST / MIDDLE: adjoint inputs cbar_U, cbar_f, wbar (in); forward inputs
    // (fin): MIDDLE c_U, c_f, w of the previous axis; FIRST U_n (F(U_n) and
    // w* = U_n + k F(U_n) recomputed here)
    // solves q = 10s + {0: T^T cUb, 1: S^T cUb, 2: T^T cfb, 3: S^T cfb, 4: P^T wb,
    //                   5: T xu, 6: S xu, 7: T xf, 8: S xf, 9: P xw}
    auto mat = [&](int q) -> const MatTab<R> & {
      const int s = q / 10, r = q - 10 * (q / 10);
      if (r == 4) return A.matT[s][0];          // P^T
      if (r == 9) return A.mat[s][0];           // P
      if (r < 4) return A.matT[s][1 + (r & 1)];  // 0, 2: T^T ; 1, 3: S^T
      return A.mat[s][1 + ((r - 5) & 1)];       // 5, 7: T ; 6, 8: S
    };
    auto cid = [&](int q) -> int {  // species * 3 + (0: P, 1: T, 2: S) of solve q
      const int s = q / 10, r = q - 10 * (q / 10);
      return s * 3 + ((r == 4 || r == 9) ? 0 : (r < 4 ? 1 + (r & 1) : 1 + ((r - 5) & 1)));
    };
    R cb[S][L], fb[S][L], wb[S][L], xu[S][L], xf[S][L];
#pragma unroll
    for (int s = 0; s < S; ++s) {
      load_chunk<R, L, CONTIG>(cb[s], A.in[0] + s * N, off0, st, cnt);
      load_chunk<R, L, CONTIG>(fb[s], A.in[1] + s * N, off0, st, cnt);
      load_chunk<R, L, CONTIG>(wb[s], A.in[2] + s * N, off0, st, cnt);
      load_chunk<R, L, CONTIG>(xu[s], A.fin[0] + s * N, off0, st, cnt);
    }
    if constexpr (KIND == ADJ_MIDDLE) {
#pragma unroll
      for (int s = 0; s < S; ++s) load_chunk<R, L, CONTIG>(xf[s], A.fin[1] + s * N, off0, st, cnt);
    } else {
#pragma unroll
      for (int t = 0; t < L; ++t) {  // F(U_n, t_n)
        R u[S], f[S];
#pragma unroll
        for (int s = 0; s < S; ++s) u[s] = xu[s][t];
        const R q = qsrc(t);
        const R src = (q != R(0)) ? (R)A.rp[0] * (((R)A.rp[1] * (R)A.src_lf - R(1)) * q + rdiv(q, R(1) + q)) : R(0);
        reaction_point<R, S>(A, u, f, src);
#pragma unroll
        for (int s = 0; s < S; ++s) xf[s][t] = (t < cnt) ? f[s] : R(0);
      }
    }
    auto xw_at = [&](int s, R (&xw)[L]) {
      if constexpr (KIND == ADJ_MIDDLE) {
        load_chunk<R, L, CONTIG>(xw, A.fin[2] + s * N, off0, st, cnt);
      } else {
#pragma unroll
        for (int t = 0; t < L; ++t) xw[t] = fma(k, xf[s][t], xu[s][t]);
      }
    };
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R xw[L];
      pass1x2q(10 * s + 0, 10 * s + 2, A.matT[s][1], A.cl[s][1], cb[s], fb[s]);
      pass1x2q(10 * s + 1, 10 * s + 3, A.matT[s][2], A.cl[s][2], cb[s], fb[s]);
      pass1q(10 * s + 4, A.matT[s][0], A.cl[s][0], wb[s]);
      pass1x2q(10 * s + 5, 10 * s + 7, A.mat[s][1], A.cl[s][1], xu[s], xf[s]);
      pass1x2q(10 * s + 6, 10 * s + 8, A.mat[s][2], A.cl[s][2], xu[s], xf[s]);
      xw_at(s, xw);
      pass1q(10 * s + 9, A.mat[s][0], A.cl[s][0], xw);
    }
    __syncthreads();
    if constexpr (CIRC) circ_chains<R>(A, sF, sY, 0, NQ, cid);
    else scan_solves<R>(A, sF, sY, sSig, 0, NQ, mat);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < S; ++s) {
      R aT[L], aS[L], x[L];
      // cbar_U: lambda_T = 9 T^T cb, lambda_S = -8 S^T cb
      pass2q(10 * s + 0, A.matT[s][1], A.cl[s][1], cb[s], aT);
      pass2q(10 * s + 5, A.mat[s][1], A.cl[s][1], xu[s], x);
      dterm(s, aT, xu[s], x, R(9));
      pass2q(10 * s + 1, A.matT[s][2], A.cl[s][2], cb[s], aS);
      pass2q(10 * s + 6, A.mat[s][2], A.cl[s][2], xu[s], x);
      dterm(s, aS, xu[s], x, R(-8));
#pragma unroll
      for (int t = 0; t < L; ++t) cb[s][t] = fma(R(9), aT[t], R(-8) * aS[t]);
      // cbar_f
      pass2q(10 * s + 2, A.matT[s][1], A.cl[s][1], fb[s], aT);
      pass2q(10 * s + 7, A.mat[s][1], A.cl[s][1], xf[s], x);
      dterm(s, aT, xf[s], x, R(9));
      pass2q(10 * s + 3, A.matT[s][2], A.cl[s][2], fb[s], aS);
      pass2q(10 * s + 8, A.mat[s][2], A.cl[s][2], xf[s], x);
      dterm(s, aS, xf[s], x, R(-8));
#pragma unroll
      for (int t = 0; t < L; ++t) fb[s][t] = fma(R(9), aT[t], R(-8) * aS[t]);
      // wbar
      R xw[L];
      xw_at(s, xw);
      pass2q(10 * s + 4, A.matT[s][0], A.cl[s][0], wb[s], aT);
      pass2q(10 * s + 9, A.mat[s][0], A.cl[s][0], xw, x);
      dterm(s, aT, xw, x, R(1));
#pragma unroll
      for (int t = 0; t < L; ++t) wb[s][t] = aT[t];
    }
    if constexpr (KIND == ADJ_MIDDLE) {
#pragma unroll
      for (int s = 0; s < S; ++s) {
        store_chunk<R, L, CONTIG>(cb[s], A.out[0] + s * N, off0, st, cnt);
        store_chunk<R, L, CONTIG>(fb[s], A.out[1] + s * N, off0, st, cnt);
        store_chunk<R, L, CONTIG>(wb[s], A.out[2] + s * N, off0, st, cnt);
      }
    } else {
      // c_U = U_n, c_f = F(U_n), w* = U_n + k F(U_n):
      // f0bar = cbar_f + k wbar*, Ubar_n = cbar_U + wbar* + J_F(U_n)^T f0bar
#pragma unroll
      for (int t = 0; t < L; ++t) {
        R u[S], yb[S], ob[S];
#pragma unroll
        for (int s = 0; s < S; ++s) {
          u[s] = xu[s][t];
          yb[s] = (t < cnt) ? fma(k, wb[s][t], fb[s][t]) : R(0);
        }
        reaction_vjp<R, S>(A, u, yb, ob, pg, qsrc(t));
#pragma unroll
        for (int s = 0; s < S; ++s) cb[s][t] = cb[s][t] + wb[s][t] + ob[s];
      }
#pragma unroll
      for (int s = 0; s < S; ++s) store_chunk<R, L, CONTIG>(cb[s], A.out[0] + s * N, off0, st, cnt);
    }
  }
  // accumulate dL/dD and dL/dparams
  double v[MAX_SPECIES + 8];
#pragma unroll
  for (int s = 0; s < MAX_SPECIES; ++s) v[s] = (s < S && line_ok) ? (double)dD[s] * A.invD[s] : 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) v[MAX_SPECIES + i] = line_ok ? (double)pg[i] : 0.0;
  block_accumulate<MAX_SPECIES + 8>(v, A.part, red);
}

// L = 1/2 sum (U - target)^2, Ubar = U - target
// (per-block partial sums to part[blockIdx.x], added by reduce_partials_kernel)
template <typename R>
__global__ void __launch_bounds__(256) misfit_kernel(const R *__restrict__ U, const R *__restrict__ T,
                                                      R *__restrict__ Ub, long long n, double *part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const R r = U[i] - T[i];
    Ub[i] = r;
    acc += 0.5 * (double)r * (double)r;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    part[blockIdx.x] = s;
  }
}

}  // namespace etd
