// etd_cplx.h -- host-side plan of the coupled two-species sweeps.
//
// Section 8's complex Ginzburg-Landau equation (D = 1 + i alpha) and cubic
// Schrodinger equation (D = [[0, 1], [-1, 0]] in the paper's form
// u_t + D Lap u = q D u) couple the two real species (Re u, Im u) inside the
// diffusion term: u_t = Dm Lap u + F(u) with Dm = [[p, -q], [q, p]], which
// acts on u = u_0 + i u_1 as multiplication by the complex number p + i q.
// The line systems of Section 7 then become complex tridiagonal systems
// I + (k/gamma)(p + i q)/h^2 B_p, one per (axis, pole), factorised on the host
// (Thomas LU without pivoting: every row is strictly diagonally dominant in
// modulus for p >= 0, since |1 + 2c| > 2|c| when Re c >= 0); periodic lines
// are factored exactly as alpha (I - lam E)(I - lam E^-1), E the cyclic shift,
// |lam| < 1 (two cyclic first-order recurrences, no tables).
#pragma once

#include <cstddef>

namespace etd {

// device line coefficients of one axis and pole: complex (re, im) pairs in the
// context's real type (Dirichlet / Neumann: Thomas factors, p entries each;
// periodic: the circulant factorisation)
struct CplxTabDev {
  const void *ell = nullptr;  // l_i = a_i / piv_{i-1} (l_0 = 0)
  const void *ipv = nullptr;  // 1 / piv_i
  const void *mu = nullptr;   // e_i / piv_i (mu_{p-1} = 0)
  const void *af = nullptr;   // [32] products of -l_i over each lane's chunk of nodes
  const void *ab = nullptr;   // [32] products of -mu_i over each lane's chunk
  // periodic lines on the circulant factorisation M = alpha (I - lam E)(I - lam E^-1)
  // (E the cyclic shift, |lam| < 1): per-lane powers of lam and the scalars
  const void *cpre = nullptr;   // [32] lam^(nodes before lane j)
  const void *csuf = nullptr;   // [32] lam^(nodes after lane j)
  const void *cchunk = nullptr; // [32] lam^(nodes of lane j)
  double lam[2] = {0, 0}, ialpha[2] = {0, 0}, inv1m[2] = {0, 0};  // lam, 1/alpha, 1/(1 - lam^p)
};

// launch plan of one axis sweep of the complex kernel: NL lines per block
// staged in shared memory (4 complex slots of p nodes per line), one warp per
// line for the solves (a chunk of ceil(p/32) nodes per lane, warp-shuffle
// scans of the chunk recurrences)
struct CplxAxis {
  int nl = 1;            // lines per block
  int nthreads = 32;
  int nblocks = 1;
  int nlo_blocks = 1;    // strided axes: blocks along the contiguous line index
  int chunk = 1;         // nodes per lane
  size_t smem = 0;
  CplxTabDev tab[3];     // gamma = 1, 3, 4
  const void *cos2 = nullptr;  // cos^2(pi x_i / L) at this axis's nodes (Schrodinger q), or null
};

}  // namespace etd
