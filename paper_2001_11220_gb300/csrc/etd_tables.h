// etd_tables.h -- host-side (FP64) factorisation of the line matrices and the
// chunk tables the sweep kernels read.  Library-internal.
#pragma once

#include <algorithm>
#include <cmath>
#include <vector>

namespace etd {

enum { BC_DIRICHLET = 0, BC_NEUMANN = 1, BC_PERIODIC = 2 };

// One line matrix prepared for a chunk length L (see MatTab in etd_internal.h
// for the meaning of every entry).  Arrays are interleaved as the kernels
// read them: pos = 4 per entry, sum = 2 per entry, chunk = 4 per chunk.
struct HostTab {
  int p = 0, L = 0, m = 0;
  std::vector<double> pos, sum, chunk;
  // interior-chunk arrays (chunk-major, one value per position): pivot
  // reciprocal e, summary weights v and w, Sherman-Morrison vector z
  std::vector<double> e1, v1, w1, z1;
  // segmented sweeps: per segment of mx chunks (A_seg, K_seg, B_seg, 0)
  std::vector<double> segc;
  double r = 0.0;  // interior off-diagonal magnitude: l_i = u_i = -r
  double sm_c = 0.0, sm_inv = 0.0;
};

// M = I + r h^2 B_p (Section 3, Example 1): diagonal 1 + 2r, off-diagonals -r;
// Neumann first row (1+2r, -2r) and last row (-2r, 1+2r); periodic corners -r.
// transpose: the matrix of the adjoint solve.  Periodic lines are split as
// M = M' + u v^T with u = (g, 0, .., 0, bl), v = (1, 0, .., 0, tr/g), g = -d_0
// (Sherman-Morrison); M' is tridiagonal and is what the tables factorise.
// mx, nseg > 1: the line is split into nseg segments of mx chunks (segmented
// sweeps); the chunk table is then padded to nseg * mx entries and segc holds
// the segment coefficients.
inline void build_tab(int p, int bc, double r, bool transpose, int L, HostTab &T, int mx = 0, int nseg = 1) {
  std::vector<double> lo(p), di(p), up(p);
  for (int i = 0; i < p; ++i) {
    di[i] = 1.0 + 2.0 * r;
    lo[i] = (i > 0) ? -r : 0.0;
    up[i] = (i < p - 1) ? -r : 0.0;
  }
  double tr = 0.0, bl = 0.0;
  if (bc == BC_NEUMANN) {
    up[0] = -2.0 * r;
    lo[p - 1] = -2.0 * r;
  }
  if (bc == BC_PERIODIC) tr = bl = -r;
  if (transpose) {
    std::vector<double> nlo(p), nup(p);
    for (int i = 0; i < p; ++i) {
      nlo[i] = (i > 0) ? up[i - 1] : 0.0;
      nup[i] = (i < p - 1) ? lo[i + 1] : 0.0;
    }
    lo.swap(nlo);
    up.swap(nup);
    std::swap(tr, bl);
  }
  std::vector<double> u;
  double g = 0.0;
  if (bc == BC_PERIODIC) {
    g = -di[0];
    di[0] -= g;
    di[p - 1] -= bl * tr / g;
    u.assign(p, 0.0);
    u[0] = g;
    u[p - 1] = bl;
  }
  // LU without pivoting, in the operation order of the Thomas variant of
  // Section 7: alpha_0 = u_0/d_0, den_i = d_i - alpha_{i-1} l_i,
  // alpha_i = u_i / den_i.  The kernels run beta_i = (b_i - l_i beta_{i-1}) / den_i
  // as (b_i + nl_i beta_{i-1}) * e_i with nl = -l and e = 1/den.
  std::vector<double> a(p), e(p), al(p), nl(p), z(p, 0.0);
  double den = di[0];
  for (int i = 0; i < p; ++i) {
    if (i > 0) den = di[i] - al[i - 1] * lo[i];
    e[i] = 1.0 / den;
    al[i] = up[i] / den;
    nl[i] = -lo[i];
    a[i] = -lo[i] * e[i];
  }
  T.sm_c = 0.0;
  T.sm_inv = 0.0;
  if (bc == BC_PERIODIC) {
    double gg = 0.0;
    for (int i = 0; i < p; ++i) {
      gg = (u[i] + nl[i] * gg) * e[i];
      z[i] = gg;
    }
    for (int i = p - 2; i >= 0; --i) z[i] -= al[i] * z[i + 1];
    T.sm_c = tr / g;
    T.sm_inv = 1.0 / (1.0 + z[0] + T.sm_c * z[p - 1]);
  }
  // chunking
  const int m = (p + L - 1) / L;
  T.p = p;
  T.L = L;
  T.m = m;
  T.pos.assign((size_t)4 * L * m, 0.0);
  T.sum.assign((size_t)2 * L * m, 0.0);
  // zero entries pad to a multiple of 8 chunks (and to whole segments)
  T.chunk.assign((size_t)4 * std::max((m + 7) & ~7, nseg > 1 ? nseg * mx : 0), 0.0);
  T.e1.assign((size_t)L * m, 1.0);
  T.v1.assign((size_t)L * m, 0.0);
  T.w1.assign((size_t)L * m, 0.0);
  T.z1.assign((size_t)L * m, 0.0);
  T.r = r;
  std::vector<double> ca(L), ce(L), cal(L), cnl(L), A(L), V(L), Wt(L), Sx(L);
  for (int j = 0; j < m; ++j) {
    const int tl = std::min(L, p - j * L) - 1;  // last real position of the chunk
    for (int t = 0; t < L; ++t) {
      const int i = j * L + t;
      const bool real = t <= tl;
      ca[t] = real ? a[i] : 0.0;
      ce[t] = real ? e[i] : 1.0;
      cal[t] = real ? al[i] : 0.0;
      cnl[t] = real ? nl[i] : 0.0;
      const size_t q = (size_t)j * L + t;
      T.pos[4 * q + 0] = cnl[t];
      T.pos[4 * q + 1] = ce[t];
      T.pos[4 * q + 2] = cal[t];
      T.pos[4 * q + 3] = real ? z[i] : 0.0;
      T.e1[q] = ce[t];
      T.z1[q] = real ? z[i] : 0.0;
    }
    // A_t = prod_{r<=t} a_r ; W_t = prod_{r<t} (-alpha_r)
    double acc = 1.0;
    for (int t = 0; t <= tl; ++t) {
      acc *= ca[t];
      A[t] = acc;
    }
    Wt[0] = 1.0;
    for (int t = 1; t <= tl; ++t) Wt[t] = Wt[t - 1] * (-cal[t - 1]);
    // v_t = e_t prod_{t<r<=tl} a_r ; w_t = e_t S_t, S_t = W_t + a_{t+1} S_{t+1}
    V[tl] = 1.0;
    for (int t = tl - 1; t >= 0; --t) V[t] = ca[t + 1] * V[t + 1];
    Sx[tl] = Wt[tl];
    for (int t = tl - 1; t >= 0; --t) Sx[t] = Wt[t] + ca[t + 1] * Sx[t + 1];
    double kap = 0.0, bst = 1.0;
    for (int t = 0; t <= tl; ++t) {
      kap += Wt[t] * A[t];
      bst *= -cal[t];
      const size_t q = (size_t)j * L + t;
      T.sum[2 * q + 0] = ce[t] * V[t];
      T.sum[2 * q + 1] = ce[t] * Sx[t];
      T.v1[q] = ce[t] * V[t];
      T.w1[q] = ce[t] * Sx[t];
    }
    T.chunk[4 * j + 0] = A[tl];
    T.chunk[4 * j + 1] = kap;
    T.chunk[4 * j + 2] = bst;
    T.chunk[4 * j + 3] = 0.0;
  }
  // Segment of chunks j0 .. j1-1 with forward carry G in and solution value
  // X_end after it: G_in[j] = P_j G + p_j (P_j = prod_{j0<=i<j} A_i), so
  //   G_out   = A_seg G + F_seg,                A_seg = prod A_j,
  //   X_start = Y_seg + K_seg G + B_seg X_end,  B_seg = prod B_j,
  //   K_seg   = sum_j (prod_{j0<=i<j} B_i) kappa_j P_j,
  // where F_seg, Y_seg are the zero-carry values of the block's chain.
  T.segc.clear();
  if (nseg > 1) {
    T.segc.assign((size_t)4 * nseg, 0.0);
    for (int sg = 0; sg < nseg; ++sg) {
      const int j0 = sg * mx, j1 = std::min(m, j0 + mx);
      double Pp = 1.0, Bp = 1.0, K = 0.0;
      for (int j = j0; j < j1; ++j) {
        K += Bp * T.chunk[4 * j + 1] * Pp;
        Bp *= T.chunk[4 * j + 2];
        Pp *= T.chunk[4 * j + 0];
      }
      T.segc[4 * sg + 0] = Pp;
      T.segc[4 * sg + 1] = K;
      T.segc[4 * sg + 2] = Bp;
    }
  }
}

// FP32 coefficient rows of the forward sweeps (MatTab::rows1): row k at k m L
// holds ne = nl e, e, -alpha, z, v, w for every position, products in FP64
inline std::vector<float> fp32_rows(const HostTab &T) {
  const size_t ml = T.e1.size();
  std::vector<float> r1(6 * ml);
  for (size_t q = 0; q < ml; ++q) {
    r1[q] = (float)(T.pos[4 * q] * T.pos[4 * q + 1]);
    r1[ml + q] = (float)T.pos[4 * q + 1];
    r1[2 * ml + q] = -(float)T.pos[4 * q + 2];
    r1[3 * ml + q] = (float)T.pos[4 * q + 3];
    r1[4 * ml + q] = (float)T.sum[2 * q];
    r1[5 * ml + q] = (float)T.sum[2 * q + 1];
  }
  return r1;
}

inline double grid_h(int bc, long long p, double len) {
  if (bc == BC_DIRICHLET) return len / (double)(p + 1);
  if (bc == BC_NEUMANN) return len / (double)(p - 1);
  return len / (double)p;
}

}  // namespace etd
