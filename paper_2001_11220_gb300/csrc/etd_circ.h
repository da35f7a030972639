// etd_circ.h -- circulant line solves for periodic axes: host-side
// coefficients and the kernel argument block.  Library-internal.
//
// On a periodic axis every line matrix M = I + c B_p (c = (k/gamma) D_s / h^2,
// B_p the cyclic second difference of Section 3) is circulant with constant
// coefficients, and factors exactly as
//     M = alpha (I - lambda E)(I - lambda E^{-1}),   (E y)_i = y_{i-1 mod p},
//     lambda = 2c / (1 + 2c + sqrt(1 + 4c)) in [0, 1),  alpha = (1 + 2c) / (1 + lambda^2),
// (lambda + 1/lambda = 2 + 1/c matches the diagonal and off-diagonals).  So
// x = M^{-1} b is two cyclic first-order recurrences with one constant
// multiplier:
//     y_i = b_i + lambda y_{i-1},   z_i = y_i + lambda z_{i+1},   x = z / alpha.
// Split into chunks of L positions, chunk j's zero-carry values are
//     F_j = (forward value at the chunk end),
//     W_j = sum_t lambda^t ytilde_t (backward value at the chunk start),
// and with Yc_j = y before the chunk and Zc_j = z after it,
//     Yc_{j+1} = Lambda Yc_j + F_j,   Zc_{j-1} = W_j + kappa Yc_j + Lambda Zc_j,
//     Lambda = lambda^L,  kappa = sum_{s<L} lambda^{2s+1},
// closed cyclically by Yc_0 = (sum_j Lambda^{m-1-j} F_j) / (1 - lambda^p) and
// the same for Zc.  Every coefficient is the same for all chunks and lines:
// the kernels read no per-position tables.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime)

#include <cmath>
#include <cstdint>
#include <vector>

#include "etd_internal.h"

namespace etd {

constexpr int CIRC_MAX_L = 16;

// one circulant matrix (species s, gamma) in the sweep's precision
template <typename R> struct CircMat {
  R lam;              // lambda
  R lamL;             // Lambda = lambda^L
  R kap;              // kappa = sum_{s<L} lambda^{2s+1}
  R inv1m;            // 1 / (1 - lambda^p)
  R pw[CIRC_MAX_L];   // lambda^t, t < L
  R sc[5];            // Lambda^(2^k): multipliers of the lane scans
  R sw[5];            // Lambda^(32 * 2^k): multipliers of the warp scans
};

// Arguments of one circulant sweep launch.
template <typename R> struct CircArgs {
  // strided sweeps with 32 lines per block: tensor maps of the three input
  // fields as 3D tensors {st, N / st, species} (box: 32 lines x the block's
  // rows x 1 species), loaded by TMA (cp.async.bulk.tensor)
  CUtensorMap tmap[3];
  const R *in[3];     // FIRST: U_n.  MIDDLE / LAST: c_U, c_f, w
  R *out[3];          // FIRST / MIDDLE: c_U, c_f, w.  LAST: U_{n+1}
  long long N;        // points per species
  long long st;       // element stride of the swept axis
  long long nlines;   // lines of the axis
  long long nlo;      // strided axes: the contiguous line index runs over [0, nlo) (= st)
  int p;              // nodes per line
  int m;              // chunks per line (p = m L)
  int lpb;            // contiguous sweeps: lines per block
  int ncol;           // strided sweeps: lines (columns) per block
  int nlo_blocks;     // strided sweeps: blocks along the contiguous line index
  int cs;             // strided sweeps: blocks per line (thread-block cluster size; 1: whole lines)
  int wb;             // strided sweeps: chunks (warps) per block
  int ngroups;        // strided sweeps: groups of 32 neighbouring lines
  long long lst;      // strided sweeps: st * p, the stride of the slow line index
  int rkind;          // reaction kind
  R kR;               // k
  R rpR[8];           // reaction parameters
  R half_kR;          // k / 2
  R cT[MAX_SPECIES], cS[MAX_SPECIES], cP[MAX_SPECIES];  // 9/alpha_T, 8/alpha_S, 1/alpha_P
  R iaT[MAX_SPECIES], iaS[MAX_SPECIES];                  // 1/alpha_T, 1/alpha_S (last sweep: T f1 - S f2)
  CircMat<R> mat[MAX_SPECIES][3];                        // [species][0: P, 1: T, 2: S]
  const R *lpow[MAX_SPECIES][3];                         // Lambda^i, i = 0 .. m + 32 (device)
  const R *kch[MAX_SPECIES][3];                          // K_{nL} = sum_{s<nL} lambda^{2s+1}, n = 0 .. m
  const R *tabg;      // strided sweeps: the exchange tables in global memory, or NULL (a shared copy)
};

// host-side coefficients of one matrix (FP64)
struct CircHost {
  double lam = 0, alpha = 1, lamL = 0, kap = 0, inv1m = 1;
  std::vector<double> pw, lpow, kch, sc, sw;
};

inline void circ_coeffs(double c, int p, int L, CircHost &H) {
  const int m = p / L;
  H.lam = (c > 0.0) ? 2.0 * c / ((1.0 + 2.0 * c) + std::sqrt(1.0 + 4.0 * c)) : 0.0;
  H.alpha = (1.0 + 2.0 * c) / (1.0 + H.lam * H.lam);
  H.pw.assign(CIRC_MAX_L, 0.0);
  double q = 1.0, kap = 0.0;
  for (int t = 0; t < L; ++t) {
    H.pw[t] = q;
    kap += q * q * H.lam;
    q *= H.lam;
  }
  H.lamL = q;
  H.kap = kap;
  H.inv1m = 1.0 / (1.0 - std::pow(H.lam, (double)p));
  H.lpow.assign((size_t)m + 33, 0.0);
  double r = 1.0;
  for (size_t i = 0; i < H.lpow.size(); ++i) {
    H.lpow[i] = r;
    r *= H.lamL;
  }
  // K_{nL}: effect of the forward carry entering n chunks on the backward
  // value at their start (K_{(a+b)L} = K_{aL} + Lambda^{2a} K_{bL})
  H.kch.assign((size_t)m + 1, 0.0);
  for (int n = 1; n <= m; ++n) H.kch[n] = H.kch[n - 1] + H.kap * std::pow(H.lamL, 2.0 * (n - 1));
  H.sc.assign(5, 0.0);
  H.sw.assign(5, 0.0);
  for (int k = 0; k < 5; ++k) {
    H.sc[k] = std::pow(H.lamL, (double)(1 << k));
    H.sw[k] = std::pow(H.lamL, (double)(32 << k));
  }
}

template <typename R> inline void circ_to_args(const CircHost &H, CircMat<R> &M) {
  M.lam = (R)H.lam;
  M.lamL = (R)H.lamL;
  M.kap = (R)H.kap;
  M.inv1m = (R)H.inv1m;
  for (int t = 0; t < CIRC_MAX_L; ++t) M.pw[t] = (R)H.pw[t];
  for (int k = 0; k < 5; ++k) {
    M.sc[k] = (R)H.sc[k];
    M.sw[k] = (R)H.sw[k];
  }
}

// Tensor maps of the strided sweep's three input fields (32 lines x rows per
// box); false if the CUDA driver's tensor-map encoder is unavailable or refuses the layout
bool circ_encode_maps(CircArgs<float> &a, int nspecies, int rows);
bool circ_encode_maps(CircArgs<double> &a, int nspecies, int rows);
// set to non-zero by a kernel whose wait for a TMA copy gave up (bounded
// wait); read and cleared by circ_take_status
int circ_take_status();

// launchers (one per element type); kind: SweepKind
cudaError_t launch_circ(const CircArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                        int nblocks, cudaStream_t s);
cudaError_t launch_circ(const CircArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                        int nblocks, cudaStream_t s);

// strided sweeps: NC lines x WB chunks per block (WB NC threads); the tile
// holds the 3 input fields of every species for the block's WB L rows, then
// two exchange buffers of up to 2 s solves (receive / compose, alternating),
// the block carries and the exchange coefficient tables
inline size_t circ_strided_smem(int nspecies, int L, int WB, int NC, size_t real_bytes, bool lean = false) {
  const size_t tile = (size_t)3 * nspecies * WB * L * NC * real_bytes;
  const size_t exch = (size_t)2 * 2 * nspecies * (WB > 16 ? WB : 16) * NC * real_bytes;
  const size_t car = (size_t)2 * 2 * nspecies * NC * real_bytes;
  const size_t tab = lean ? 0 : (size_t)nspecies * 3 * (2 * (WB + 1) + 35) * real_bytes;
  return tile + 2 * exch + car + tab;
}
// the exchange tables of one strided plan: [nspecies * 3][2 (WB + 1) + 35]
inline int circ_tab_entries(int nspecies, int WB) { return nspecies * 3 * (2 * (WB + 1) + 35); }
// static shared memory of the strided kernels (mbarriers)
constexpr size_t CIRC_STRIDED_STATIC_SMEM = 128;
cudaError_t circ_cluster_capacity(const CircArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters);
cudaError_t circ_cluster_capacity(const CircArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                  int &nclusters);

cudaError_t circ_first_capacity(int real_bytes, int nspecies, int L, int nthreads, int rkind, size_t smem,
                                int &blocks_per_sm);

// kernels of one element type share this signature
template <typename R> using CircKernel = void (*)(CircArgs<R>);
// FP32 two-species kernels with the reaction kind (2, 3, 4) fixed at compile
// time, for the shapes the planner prefers; nullptr where none is compiled
CircKernel<float> circ_first_kernel_rk(int L, int nthreads, int rkind);
CircKernel<float> circ_strided_kernel_rk(int kind, int wb, int nc, int rkind);
int circ_take_status_rk_first();
int circ_take_status_rk_strided();

// shared memory of a contiguous circulant sweep block of nthreads threads
inline size_t circ_first_smem(int nspecies, int L, int nthreads, int m, int lpb, size_t real_bytes) {
  const size_t stage = (size_t)2 * nspecies * nthreads * L * real_bytes;  // double buffer
  const int nw = m > 32 ? m / 32 : 1;
  const size_t tot = (size_t)2 * lpb * nw * 5 * nspecies * real_bytes;
  return stage + ((tot + 15) & ~(size_t)15);
}

}  // namespace etd
