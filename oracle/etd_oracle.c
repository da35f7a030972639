/*
 * etd_oracle.c -- plain FP64 CPU oracle for the ETD-RDP-IF scheme
 * (arXiv 2001.11220).  TEST INFRASTRUCTURE ONLY: see etd_oracle.h.
 *
 * Written for a reader checking it against the paper: no blocking, no fusion,
 * one line at a time, every intermediate of the framed scheme stored in its
 * own array.  Citations name the paper's section / equation / figure.
 */
#include "etd_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------ grid -- */

/* Section 3, Example 1: h = L/(p+1) (Dirichlet, p interior nodes),
 * h = L/(p-1) (Neumann, both boundary nodes counted), h = L/p (periodic). */
double oracle_h(const oracle_problem *P, int a) {
  int p = P->n[a];
  double L = P->length[a];
  if (P->bc[a] == OR_DIRICHLET) return L / (double)(p + 1);
  if (P->bc[a] == OR_NEUMANN) return L / (double)(p - 1);
  return L / (double)p;
}

/* coordinate of node i on axis a (x_i = (i+1) h for Dirichlet, i h otherwise) */
static double node_x(const oracle_problem *P, int a, int i) {
  double h = oracle_h(P, a);
  return P->bc[a] == OR_DIRICHLET ? (i + 1) * h : i * h;
}

static long npoints(const oracle_problem *P) {
  long N = 1;
  for (int a = 0; a < P->dim; ++a) N *= P->n[a];
  return N;
}

/* stride of axis a in the x-fastest layout */
static long axis_stride(const oracle_problem *P, int a) {
  long st = 1;
  for (int b = 0; b < a; ++b) st *= P->n[b];
  return st;
}

static int check_problem(const oracle_problem *P) {
  if (!P || P->dim < 1 || P->dim > 3) return -1;
  if (P->nspecies < 1 || P->nspecies > 4) return -1;
  if (!(P->k > 0)) return -1;
  for (int a = 0; a < P->dim; ++a) {
    if (P->n[a] < 3) return -1;
    if (P->bc[a] < 0 || P->bc[a] > 2) return -1;
    if (!(P->length[a] > 0)) return -1;
  }
  if (P->coupled) {
    if (P->nspecies != 2) return -1;
    for (int j = 0; j < 4; ++j)
      if (!isfinite(P->Dc[j])) return -1;
  } else {
    for (int s = 0; s < P->nspecies; ++s)
      if (!(P->D[s] >= 0)) return -1;
  }
  if ((P->reaction == OR_BRUSSELATOR || P->reaction == OR_SCHNAKENBERG ||
       P->reaction == OR_GRAY_SCOTT || P->reaction == OR_CGL || P->reaction == OR_NLS) &&
      P->nspecies != 2) return -1;
  if (P->reaction == OR_ENZYME && P->nspecies != 1) return -1;
  if (P->reaction < 0 || P->reaction > OR_NLS) return -1;
  return 0;
}

/* ---------------------------------------------------- line matrix (Ex. 1) -- */

/* The p x p matrix M = I + r * (h^2 B_p), B_p of Section 3 Example 1:
 * diagonal 1 + 2r, off-diagonals -r; Neumann first row (1+2r, -2r) and last
 * row (-2r, 1+2r); periodic corners -r.  lo[i] = M[i][i-1], up[i] = M[i][i+1],
 * tr = M[0][p-1], bl = M[p-1][0].  transpose != 0 returns M^T. */
static void line_matrix(int p, int bc, double r, int transpose, double *lo, double *di,
                        double *up, double *tr, double *bl) {
  for (int i = 0; i < p; ++i) {
    di[i] = 1.0 + 2.0 * r;
    lo[i] = (i > 0) ? -r : 0.0;
    up[i] = (i < p - 1) ? -r : 0.0;
  }
  *tr = 0.0;
  *bl = 0.0;
  if (bc == OR_NEUMANN) {
    up[0] = -2.0 * r;
    lo[p - 1] = -2.0 * r;
  }
  if (bc == OR_PERIODIC) {
    *tr = -r;
    *bl = -r;
  }
  if (transpose) {
    /* (M^T)[i][i-1] = M[i-1][i] = up[i-1];  (M^T)[i][i+1] = M[i+1][i] = lo[i+1] */
    double *nlo = (double *)malloc(sizeof(double) * p);
    double *nup = (double *)malloc(sizeof(double) * p);
    for (int i = 0; i < p; ++i) {
      nlo[i] = (i > 0) ? up[i - 1] : 0.0;
      nup[i] = (i < p - 1) ? lo[i + 1] : 0.0;
    }
    memcpy(lo, nlo, sizeof(double) * p);
    memcpy(up, nup, sizeof(double) * p);
    free(nlo);
    free(nup);
    double t = *tr;
    *tr = *bl;
    *bl = t;
  }
}

/* Thomas algorithm as written in Section 7 (offset w = 1 for one line):
 * alpha_0 = u_0/d_0, beta_0 = b_0/d_0; for i >= 1
 * alpha_i = u_i/(d_i - alpha_{i-1} l_i), beta_i = (b_i - beta_{i-1} l_i)/(d_i - alpha_{i-1} l_i);
 * x_{p-1} = beta_{p-1}, x_i = beta_i - alpha_i x_{i+1}.  No pivoting (the
 * matrices are diagonally dominant, Section 7). */
static void thomas(int p, const double *lo, const double *di, const double *up, const double *b,
                   double *x, double *alpha, double *beta) {
  alpha[0] = up[0] / di[0];
  beta[0] = b[0] / di[0];
  for (int i = 1; i < p; ++i) {
    double den = di[i] - alpha[i - 1] * lo[i];
    alpha[i] = up[i] / den;
    beta[i] = (b[i] - beta[i - 1] * lo[i]) / den;
  }
  x[p - 1] = beta[p - 1];
  for (int i = p - 2; i >= 0; --i) x[i] = beta[i] - alpha[i] * x[i + 1];
}

int oracle_line_solve(int p, int bc, double r, int transpose, const double *b, double *x) {
  if (p < 3 || bc < 0 || bc > 2) return -1;
  double *lo = (double *)malloc(sizeof(double) * p);
  double *di = (double *)malloc(sizeof(double) * p);
  double *up = (double *)malloc(sizeof(double) * p);
  double *al = (double *)malloc(sizeof(double) * p);
  double *be = (double *)malloc(sizeof(double) * p);
  double *bb = (double *)malloc(sizeof(double) * p);
  double tr, bl;
  line_matrix(p, bc, r, transpose, lo, di, up, &tr, &bl);
  memcpy(bb, b, sizeof(double) * p); /* b and x may alias */
  if (bc != OR_PERIODIC) {
    thomas(p, lo, di, up, bb, x, al, be);
  } else {
    /* Cyclic line: M = M' + u v^T with u = (g, 0, ..., 0, bl)^T and
     * v = (1, 0, ..., 0, tr/g)^T, g = -d_0; M' is tridiagonal with
     * d'_0 = d_0 - g and d'_{p-1} = d_{p-1} - bl tr / g.  Sherman-Morrison:
     * x = y - (v.y)/(1 + v.z) z with M' y = b and M' z = u. */
    double g = -di[0];
    double *y = (double *)malloc(sizeof(double) * p);
    double *z = (double *)malloc(sizeof(double) * p);
    double *u = (double *)calloc(p, sizeof(double));
    di[0] -= g;
    di[p - 1] -= bl * tr / g;
    u[0] = g;
    u[p - 1] = bl;
    thomas(p, lo, di, up, bb, y, al, be);
    thomas(p, lo, di, up, u, z, al, be);
    double vy = y[0] + (tr / g) * y[p - 1];
    double vz = z[0] + (tr / g) * z[p - 1];
    double sigma = vy / (1.0 + vz);
    for (int i = 0; i < p; ++i) x[i] = y[i] - sigma * z[i];
    free(y);
    free(z);
    free(u);
  }
  free(lo);
  free(di);
  free(up);
  free(al);
  free(be);
  free(bb);
  return 0;
}

/* ------------------------------------- coupled lines (Section 8, 2 x 2 D) -- */

/* Gaussian elimination with partial pivoting, A = P L U in place (row-major
 * m x m; piv[i] = the row swapped into position i at step i).  Returns -1 on
 * a zero pivot. */
static int dense_lu(int m, double *A, int *piv) {
  for (int c = 0; c < m; ++c) {
    int r = c;
    for (int i = c + 1; i < m; ++i)
      if (fabs(A[(long)i * m + c]) > fabs(A[(long)r * m + c])) r = i;
    piv[c] = r;
    if (A[(long)r * m + c] == 0.0) return -1;
    if (r != c)
      for (int j = 0; j < m; ++j) {
        double t = A[(long)c * m + j];
        A[(long)c * m + j] = A[(long)r * m + j];
        A[(long)r * m + j] = t;
      }
    for (int i = c + 1; i < m; ++i) {
      double l = A[(long)i * m + c] / A[(long)c * m + c];
      A[(long)i * m + c] = l;
      for (int j = c + 1; j < m; ++j) A[(long)i * m + j] -= l * A[(long)c * m + j];
    }
  }
  return 0;
}

/* solve with the factors of dense_lu: x = A^{-1} b in place */
static void dense_lu_solve(int m, const double *LU, const int *piv, double *x) {
  for (int c = 0; c < m; ++c) {
    double t = x[c];
    x[c] = x[piv[c]];
    x[piv[c]] = t;
  }
  for (int i = 1; i < m; ++i)
    for (int j = 0; j < i; ++j) x[i] -= LU[(long)i * m + j] * x[j];
  for (int i = m - 1; i >= 0; --i) {
    for (int j = i + 1; j < m; ++j) x[i] -= LU[(long)i * m + j] * x[j];
    x[i] /= LU[(long)i * m + i];
  }
}

/* The 2p x 2p matrix of one coupled line, unknowns ordered (node i, species s)
 * -> 2 i + s: I + rr (B (x) Dc) with B = h^2 B_p of Example 1 (read off
 * line_matrix at r = 1 minus the identity) and rr = (k/gamma)/h^2
 * (transpose != 0: its transpose).  A is m x m, m = 2p, row-major. */
static void coupled_line_matrix(const oracle_problem *P, int p, int bc, double rr, int transpose, double *A) {
  double *lo = (double *)malloc(sizeof(double) * p);
  double *di = (double *)malloc(sizeof(double) * p);
  double *up = (double *)malloc(sizeof(double) * p);
  double tr, bl;
  line_matrix(p, bc, 1.0, 0, lo, di, up, &tr, &bl);
  const long m = 2L * p;
  memset(A, 0, sizeof(double) * m * m);
  for (int i = 0; i < p; ++i) {
    for (int j = 0; j < p; ++j) {
      double b = 0.0;
      if (j == i) b = di[i] - 1.0;
      else if (j == i - 1) b = lo[i];
      else if (j == i + 1) b = up[i];
      if (i == 0 && j == p - 1) b += tr;
      if (i == p - 1 && j == 0) b += bl;
      if (b == 0.0) continue;
      for (int s = 0; s < 2; ++s)
        for (int t = 0; t < 2; ++t) {
          long row = 2L * i + s, col = 2L * j + t;
          double v = rr * b * P->Dc[2 * s + t];
          if (transpose) A[col * m + row] += v;
          else A[row * m + col] += v;
        }
    }
  }
  for (long q = 0; q < m; ++q) A[q * m + q] += 1.0;
  free(lo);
  free(di);
  free(up);
}

/* 2 x 2 helpers, row-major */
static void m2_mul(const double *A, const double *B, double *C) {
  double c0 = A[0] * B[0] + A[1] * B[2], c1 = A[0] * B[1] + A[1] * B[3];
  double c2 = A[2] * B[0] + A[3] * B[2], c3 = A[2] * B[1] + A[3] * B[3];
  C[0] = c0; C[1] = c1; C[2] = c2; C[3] = c3;
}
static int m2_inv(const double *A, double *X) {
  double det = A[0] * A[3] - A[1] * A[2];
  if (det == 0.0) return -1;
  double a0 = A[3] / det, a1 = -A[1] / det, a2 = -A[2] / det, a3 = A[0] / det;
  X[0] = a0; X[1] = a1; X[2] = a2; X[3] = a3;
  return 0;
}

/* The Thomas algorithm of Section 7 in 2 x 2 block form, for a coupled
 * Dirichlet or Neumann line: blocks L_i = rr lo_i Dc, G_i = I + rr (d_i - 1) Dc,
 * U_i = rr up_i Dc of I + rr (B (x) Dc) (lo, d, up read off line_matrix at r = 1;
 * transpose: B^T and Dc^T).  alpha_0 = G_0^{-1} U_0, beta_0 = G_0^{-1} b_0;
 * alpha_i = (G_i - L_i alpha_{i-1})^{-1} U_i, beta_i = (G_i - L_i alpha_{i-1})^{-1}
 * (b_i - L_i beta_{i-1}); x_{p-1} = beta_{p-1}, x_i = beta_i - alpha_i x_{i+1}.
 * b and x hold node i's two species at 2 i, 2 i + 1 (may alias).  Returns -1 on
 * a singular pivot block. */
static int block_thomas(const oracle_problem *P, int p, int bc, double rr, int transpose, const double *b,
                        double *x) {
  double *lo = (double *)malloc(sizeof(double) * p);
  double *di = (double *)malloc(sizeof(double) * p);
  double *up = (double *)malloc(sizeof(double) * p);
  double *al = (double *)malloc(sizeof(double) * 4 * p);
  double *be = (double *)malloc(sizeof(double) * 2 * p);
  double tr, bl, D[4];
  line_matrix(p, bc, 1.0, transpose, lo, di, up, &tr, &bl);
  D[0] = P->Dc[0]; D[3] = P->Dc[3];
  D[1] = transpose ? P->Dc[2] : P->Dc[1];
  D[2] = transpose ? P->Dc[1] : P->Dc[2];
  int bad = 0;
  for (int i = 0; i < p && !bad; ++i) {
    double G[4], L[4], Uu[4], Gi[4], r[2];
    for (int j = 0; j < 4; ++j) {
      G[j] = rr * (di[i] - 1.0) * D[j] + (j == 0 || j == 3 ? 1.0 : 0.0);
      L[j] = rr * lo[i] * D[j];
      Uu[j] = rr * up[i] * D[j];
    }
    r[0] = b[2 * i];
    r[1] = b[2 * i + 1];
    if (i > 0) {
      double La[4];
      m2_mul(L, al + 4 * (i - 1), La);
      for (int j = 0; j < 4; ++j) G[j] -= La[j];
      const double *bp = be + 2 * (i - 1);
      r[0] -= L[0] * bp[0] + L[1] * bp[1];
      r[1] -= L[2] * bp[0] + L[3] * bp[1];
    }
    if (m2_inv(G, Gi)) {
      bad = 1;
      break;
    }
    m2_mul(Gi, Uu, al + 4 * i);
    be[2 * i] = Gi[0] * r[0] + Gi[1] * r[1];
    be[2 * i + 1] = Gi[2] * r[0] + Gi[3] * r[1];
  }
  if (!bad) {
    x[2 * (p - 1)] = be[2 * (p - 1)];
    x[2 * (p - 1) + 1] = be[2 * (p - 1) + 1];
    for (int i = p - 2; i >= 0; --i) {
      const double *a = al + 4 * i;
      double x0 = x[2 * (i + 1)], x1 = x[2 * (i + 1) + 1];
      x[2 * i] = be[2 * i] - (a[0] * x0 + a[1] * x1);
      x[2 * i + 1] = be[2 * i + 1] - (a[2] * x0 + a[3] * x1);
    }
  }
  free(lo);
  free(di);
  free(up);
  free(al);
  free(be);
  return bad ? -1 : 0;
}

/* ------------------------------------------------ axis operators (Eq. Ai) -- */

/* out = (I + (k/gamma) A_a)^{-1} in, one line of axis a at a time.  A_a acts
 * on species s as D_s B_p along axis a (Eq. Ai), so each line of each species
 * is an independent system with r = (k/gamma) D_s / h_a^2 (Section 7). */
int oracle_axis_solve(const oracle_problem *P, int a, double gamma, int transpose,
                      const double *in, double *out) {
  if (check_problem(P) || a < 0 || a >= P->dim) return -1;
  long N = npoints(P);
  int p = P->n[a];
  long st = axis_stride(P, a);
  long nhigh = N / (st * p);
  double h = oracle_h(P, a);
  if (P->coupled && P->bc[a] != OR_PERIODIC) {
    /* both species of a line form one block-tridiagonal system (Section 8: D
     * not diagonal), solved by the block Thomas algorithm */
    const double rr = (P->k / gamma) / (h * h);
    int bad = 0;
#pragma omp parallel
    {
      double *line = (double *)malloc(sizeof(double) * 2 * p);
#pragma omp for schedule(static) reduction(| : bad)
      for (long q = 0; q < nhigh * st; ++q) {
        long hi = q / st, lo = q % st;
        long base = lo + hi * st * p;
        for (int i = 0; i < p; ++i) {
          line[2 * i] = in[base + i * st];
          line[2 * i + 1] = in[N + base + i * st];
        }
        bad |= block_thomas(P, p, P->bc[a], rr, transpose, line, line) != 0;
        for (int i = 0; i < p; ++i) {
          out[base + i * st] = line[2 * i];
          out[N + base + i * st] = line[2 * i + 1];
        }
      }
      free(line);
    }
    return bad ? -1 : 0;
  }
  if (P->coupled) {
    /* periodic: both species of a line form one cyclic block system, solved
     * by dense LU (formed once per call) */
    const int m = 2 * p;
    double *LU = (double *)malloc(sizeof(double) * (size_t)m * m);
    int *piv = (int *)malloc(sizeof(int) * m);
    coupled_line_matrix(P, p, P->bc[a], (P->k / gamma) / (h * h), transpose, LU);
    int bad = dense_lu(m, LU, piv);
    if (!bad) {
#pragma omp parallel
      {
        double *line = (double *)malloc(sizeof(double) * m);
#pragma omp for schedule(static)
        for (long q = 0; q < nhigh * st; ++q) {
          long hi = q / st, lo = q % st;
          long base = lo + hi * st * p;
          for (int i = 0; i < p; ++i) {
            line[2 * i] = in[base + i * st];
            line[2 * i + 1] = in[N + base + i * st];
          }
          dense_lu_solve(m, LU, piv, line);
          for (int i = 0; i < p; ++i) {
            out[base + i * st] = line[2 * i];
            out[N + base + i * st] = line[2 * i + 1];
          }
        }
        free(line);
      }
    }
    free(LU);
    free(piv);
    return bad ? -1 : 0;
  }
  for (int s = 0; s < P->nspecies; ++s) {
    double r = (P->k / gamma) * P->D[s] / (h * h);
    const double *src = in + s * N;
    double *dst = out + s * N;
    /* lines are independent: with OpenMP they are shared among host threads
     * (each with its own line buffer); the arithmetic per line is unchanged */
#pragma omp parallel
    {
      double *line = (double *)malloc(sizeof(double) * p);
#pragma omp for schedule(static)
      for (long q = 0; q < nhigh * st; ++q) {
        long hi = q / st, lo = q % st;
        long base = lo + hi * st * p;
        for (int i = 0; i < p; ++i) line[i] = src[base + i * st];
        oracle_line_solve(p, P->bc[a], r, transpose, line, line);
        for (int i = 0; i < p; ++i) dst[base + i * st] = line[i];
      }
      free(line);
    }
  }
  return 0;
}

/* host threads for the line loops (OpenMP builds; ignored otherwise) */
void oracle_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int oracle_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* out = B_a in per species (no D): the -Laplacian along axis a, Example 1. */
static void axis_laplacian(const oracle_problem *P, int a, const double *in, double *out) {
  long N = npoints(P);
  int p = P->n[a];
  long st = axis_stride(P, a);
  long nhigh = N / (st * p);
  double h = oracle_h(P, a);
  double *lo = (double *)malloc(sizeof(double) * p);
  double *di = (double *)malloc(sizeof(double) * p);
  double *up = (double *)malloc(sizeof(double) * p);
  double tr, bl;
  /* M = I + r B h^2 with r = 1  =>  B h^2 = M - I */
  line_matrix(p, P->bc[a], 1.0, 0, lo, di, up, &tr, &bl);
  for (int s = 0; s < P->nspecies; ++s)
    for (long hi = 0; hi < nhigh; ++hi)
      for (long l0 = 0; l0 < st; ++l0) {
        long base = s * N + l0 + hi * st * p;
        for (int i = 0; i < p; ++i) {
          double acc = (di[i] - 1.0) * in[base + i * st];
          if (i > 0) acc += lo[i] * in[base + (i - 1) * st];
          if (i < p - 1) acc += up[i] * in[base + (i + 1) * st];
          if (i == 0) acc += tr * in[base + (p - 1) * st];
          if (i == p - 1) acc += bl * in[base];
          out[base + i * st] = acc / (h * h);
        }
      }
  free(lo);
  free(di);
  free(up);
}

int oracle_axis_apply(const oracle_problem *P, int a, const double *in, double *out) {
  if (check_problem(P) || a < 0 || a >= P->dim) return -1;
  long N = npoints(P);
  if (P->coupled) {
    double *lap = (double *)malloc(sizeof(double) * 2 * N);
    axis_laplacian(P, a, in, lap);
    for (long i = 0; i < N; ++i) {
      double l0 = lap[i], l1 = lap[N + i];
      out[i] = P->Dc[0] * l0 + P->Dc[1] * l1;
      out[N + i] = P->Dc[2] * l0 + P->Dc[3] * l1;
    }
    free(lap);
    return 0;
  }
  axis_laplacian(P, a, in, out);
  for (int s = 0; s < P->nspecies; ++s)
    for (long i = 0; i < N; ++i) out[s * N + i] *= P->D[s];
  return 0;
}

/* ---------------------------------------------------- reaction (Sec. 2) -- */

/* manufactured source of the enzyme model: with q = e^{-t} prod_a sin(pi x_a/L_a)
 * the exact solution u = q satisfies u_t = d Lap u - u/(1+u) + src. */
static double enzyme_q(const oracle_problem *P, const int *idx, double t) {
  double q = exp(-t);
  for (int a = 0; a < P->dim; ++a) q *= sin(OR_PI * node_x(P, a, idx[a]) / P->length[a]);
  return q;
}
static double enzyme_lap_factor(const oracle_problem *P) {
  double f = 0.0;
  for (int a = 0; a < P->dim; ++a) f += (OR_PI / P->length[a]) * (OR_PI / P->length[a]);
  return f;
}

static void point_index(const oracle_problem *P, long i, int *idx) {
  idx[0] = idx[1] = idx[2] = 0;
  for (int a = 0; a < P->dim; ++a) {
    idx[a] = (int)(i % P->n[a]);
    i /= P->n[a];
  }
}

/* F at one point: u[s] -> f[s]; also J[s][r] = dF_s/du_r and G[s][j] = dF_s/dparams_j */
static void reaction_point(const oracle_problem *P, const double *u, const int *idx, double t,
                           double *f, double J[4][4], double G[4][8]) {
  const double *p = P->params;
  int S = P->nspecies;
  for (int s = 0; s < 4; ++s) {
    f[s] = 0.0;
    for (int r = 0; r < 4; ++r) J[s][r] = 0.0;
    for (int j = 0; j < 8; ++j) G[s][j] = 0.0;
  }
  switch (P->reaction) {
  case OR_ZERO:
    break;
  case OR_LINEAR:
    for (int s = 0; s < S; ++s) {
      f[s] = p[0] * u[s] + p[1];
      J[s][s] = p[0];
      G[s][0] = u[s];
      G[s][1] = 1.0;
    }
    break;
  case OR_BRUSSELATOR: { /* config form: a constant feed, b the (A) of Section 8.2 */
    double a = p[0], b = p[1], U = u[0], V = u[1];
    f[0] = a + U * U * V - (b + 1.0) * U;
    f[1] = b * U - U * U * V;
    J[0][0] = 2.0 * U * V - (b + 1.0);
    J[0][1] = U * U;
    J[1][0] = b - 2.0 * U * V;
    J[1][1] = -U * U;
    G[0][0] = 1.0;
    G[0][1] = -U;
    G[1][1] = U;
    break;
  }
  case OR_SCHNAKENBERG: {
    double a = p[0], b = p[1], g = p[2], U = u[0], V = u[1];
    f[0] = g * (a - U + U * U * V);
    f[1] = g * (b - U * U * V);
    J[0][0] = g * (-1.0 + 2.0 * U * V);
    J[0][1] = g * U * U;
    J[1][0] = -g * 2.0 * U * V;
    J[1][1] = -g * U * U;
    G[0][0] = g;
    G[1][1] = g;
    G[0][2] = a - U + U * U * V;
    G[1][2] = b - U * U * V;
    break;
  }
  case OR_GRAY_SCOTT: {
    double F = p[0], kap = p[1], U = u[0], V = u[1];
    f[0] = -U * V * V + F * (1.0 - U);
    f[1] = U * V * V - (F + kap) * V;
    J[0][0] = -V * V - F;
    J[0][1] = -2.0 * U * V;
    J[1][0] = V * V;
    J[1][1] = 2.0 * U * V - (F + kap);
    G[0][0] = 1.0 - U;
    G[1][0] = -V;
    G[1][1] = -V;
    break;
  }
  case OR_CGL: { /* u = a + i b, r = |u|^2: F = u - (1 + i beta) u r (Section 8, CGL with alpha = 0) */
    double beta = p[0], a = u[0], b = u[1], r = a * a + b * b;
    double ca = a - beta * b, cb = beta * a + b; /* (1 + i beta) u */
    f[0] = a - r * ca;
    f[1] = b - r * cb;
    J[0][0] = 1.0 - r - 2.0 * a * ca;
    J[0][1] = beta * r - 2.0 * b * ca;
    J[1][0] = -beta * r - 2.0 * a * cb;
    J[1][1] = 1.0 - r - 2.0 * b * cb;
    G[0][0] = r * b;
    G[1][0] = -r * a;
    break;
  }
  case OR_NLS: { /* Section 8: F = q J u, J = [[0, 1], [-1, 0]], q = p0 + p1 |u|^2 + p2 bfac(x) */
    double v = u[0], w = u[1], r = v * v + w * w;
    double bfac = 1.0, cc = 1.0;
    for (int a = 0; a < P->dim; ++a) {
      double c = cos(OR_PI * node_x(P, a, idx[a]) / P->length[a]);
      cc *= c * c;
    }
    bfac -= cc;
    double q = p[0] + p[1] * r + p[2] * bfac;
    f[0] = q * w;
    f[1] = -q * v;
    J[0][0] = 2.0 * p[1] * v * w;
    J[0][1] = q + 2.0 * p[1] * w * w;
    J[1][0] = -q - 2.0 * p[1] * v * v;
    J[1][1] = -2.0 * p[1] * v * w;
    G[0][0] = w;
    G[1][0] = -v;
    G[0][1] = r * w;
    G[1][1] = -r * v;
    G[0][2] = bfac * w;
    G[1][2] = -bfac * v;
    break;
  }
  case OR_ENZYME: {
    double U = u[0];
    f[0] = -U / (1.0 + U);
    J[0][0] = -1.0 / ((1.0 + U) * (1.0 + U));
    if (p[0] != 0.0) {
      double q = enzyme_q(P, idx, t);
      double lf = enzyme_lap_factor(P);
      double src = (p[1] * lf - 1.0) * q + q / (1.0 + q);
      f[0] += p[0] * src;
      G[0][0] = src;
      G[0][1] = p[0] * lf * q;
    }
    break;
  }
  }
}

int oracle_reaction(const oracle_problem *P, const double *U, double t, double *F) {
  if (check_problem(P)) return -1;
  long N = npoints(P);
  int S = P->nspecies;
#pragma omp parallel for schedule(static)
  for (long i = 0; i < N; ++i) {
    int idx[3];
    double u[4], f[4], J[4][4], G[4][8];
    point_index(P, i, idx);
    for (int s = 0; s < S; ++s) u[s] = U[s * N + i];
    reaction_point(P, u, idx, t, f, J, G);
    for (int s = 0; s < S; ++s) F[s * N + i] = f[s];
  }
  return 0;
}

int oracle_reaction_vjp(const oracle_problem *P, const double *U, double t, const double *ybar,
                        double *out, double *pbar) {
  if (check_problem(P)) return -1;
  long N = npoints(P);
  int S = P->nspecies, idx[3];
  double u[4], f[4], J[4][4], G[4][8];
  for (long i = 0; i < N; ++i) {
    point_index(P, i, idx);
    for (int s = 0; s < S; ++s) u[s] = U[s * N + i];
    reaction_point(P, u, idx, t, f, J, G);
    for (int r = 0; r < S; ++r) {
      double acc = 0.0;
      for (int s = 0; s < S; ++s) acc += J[s][r] * ybar[s * N + i];
      out[r * N + i] = acc;
    }
    if (pbar)
      for (int j = 0; j < 8; ++j)
        for (int s = 0; s < S; ++s) pbar[j] += G[s][j] * ybar[s * N + i];
  }
  return 0;
}

/* ------------------------------------------------------------ the step -- */

/* Intermediates of one step, named after the flow charts of Section 7.
 * cU[a], cf[a], w[a] hold the three carried fields BEFORE axis a is applied
 * (a = 0 .. d-1); xT_U[a], xS_U[a], xT_f[a], xS_f[a] the four RDP solves of
 * axis a < d-1 (kept for the adjoint's D-derivative); Ustar, fstar, f1, f2,
 * d1, d2 the last-axis quantities. */
typedef struct {
  long M;
  double *f0;
  double *cU[3], *cf[3], *w[3];
  double *xT_U[3], *xS_U[3], *xT_f[3], *xS_f[3];
  double *Ustar, *fstar, *f1, *f2, *d1, *d2;
} step_work;

static double *dalloc(long M) { return (double *)calloc((size_t)M, sizeof(double)); }

static void work_alloc(step_work *W, long M, int dim) {
  memset(W, 0, sizeof(*W));
  W->M = M;
  W->f0 = dalloc(M);
  for (int a = 0; a < dim; ++a) {
    W->cU[a] = dalloc(M);
    W->cf[a] = dalloc(M);
    W->w[a] = dalloc(M);
    W->xT_U[a] = dalloc(M);
    W->xS_U[a] = dalloc(M);
    W->xT_f[a] = dalloc(M);
    W->xS_f[a] = dalloc(M);
  }
  W->Ustar = dalloc(M);
  W->fstar = dalloc(M);
  W->f1 = dalloc(M);
  W->f2 = dalloc(M);
  W->d1 = dalloc(M);
  W->d2 = dalloc(M);
}

static void work_free(step_work *W) {
  free(W->f0);
  for (int a = 0; a < 3; ++a) {
    free(W->cU[a]);
    free(W->cf[a]);
    free(W->w[a]);
    free(W->xT_U[a]);
    free(W->xS_U[a]);
    free(W->xT_f[a]);
    free(W->xS_f[a]);
  }
  free(W->Ustar);
  free(W->fstar);
  free(W->f1);
  free(W->f2);
  free(W->d1);
  free(W->d2);
}

/* The d-dimensional ETD-RDP-IF frame of Section 6, written with
 * T_a = (I + k/3 A_a)^{-1}, S_a = (I + k/4 A_a)^{-1}, P_a = (I + k A_a)^{-1},
 * R_a = 9 T_a - 8 S_a (partial fractions of R_RDP, Section 6):
 *   U*      = P_d ... P_1 (U_n + k f(U_n, t_n))
 *   U_{n+1} = T_d [ R_{d-1}..R_1 (9 U_n + 2k f(U_n)) + k f(U*, t_{n+1}) ]
 *           - S_d [ R_{d-1}..R_1 (8 U_n + 3k/2 f(U_n)) + k/2 f(U*, t_{n+1}) ]
 * evaluated as in Figs. flow2d/flow3d: c_U = R..R U_n and c_f = R..R f(U_n)
 * are carried separately (by linearity R(9U + 2kf) = 9 R U + 2k R f), then
 * f1 = 9 c_U + 2k c_f + k f*, f2 = 8 c_U + 3k/2 c_f + k/2 f*,
 * U_{n+1} = T_d f1 - S_d f2.  (The 3D chart prints the sign of f2 flipped
 * against its own frame and against the 2D chart; the frame is followed.) */
static void step_forward(const oracle_problem *P, const double *Un, double t, step_work *W,
                         double *Unext) {
  long M = W->M;
  int d = P->dim;
  double k = P->k;
  oracle_reaction(P, Un, t, W->f0);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < M; ++i) {
    W->cU[0][i] = Un[i];
    W->cf[0][i] = W->f0[i];
    W->w[0][i] = Un[i] + k * W->f0[i];
  }
  for (int a = 0; a < d - 1; ++a) {
    oracle_axis_solve(P, a, 3.0, 0, W->cU[a], W->xT_U[a]);
    oracle_axis_solve(P, a, 4.0, 0, W->cU[a], W->xS_U[a]);
    oracle_axis_solve(P, a, 3.0, 0, W->cf[a], W->xT_f[a]);
    oracle_axis_solve(P, a, 4.0, 0, W->cf[a], W->xS_f[a]);
    oracle_axis_solve(P, a, 1.0, 0, W->w[a], W->w[a + 1]);
#pragma omp parallel for schedule(static)
    for (long i = 0; i < M; ++i) {
      W->cU[a + 1][i] = 9.0 * W->xT_U[a][i] - 8.0 * W->xS_U[a][i];
      W->cf[a + 1][i] = 9.0 * W->xT_f[a][i] - 8.0 * W->xS_f[a][i];
    }
  }
  oracle_axis_solve(P, d - 1, 1.0, 0, W->w[d - 1], W->Ustar);
  oracle_reaction(P, W->Ustar, t + k, W->fstar);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < M; ++i) {
    W->f1[i] = 9.0 * W->cU[d - 1][i] + 2.0 * k * W->cf[d - 1][i] + k * W->fstar[i];
    W->f2[i] = 8.0 * W->cU[d - 1][i] + 1.5 * k * W->cf[d - 1][i] + 0.5 * k * W->fstar[i];
  }
  oracle_axis_solve(P, d - 1, 3.0, 0, W->f1, W->d1);
  oracle_axis_solve(P, d - 1, 4.0, 0, W->f2, W->d2);
#pragma omp parallel for schedule(static)
  for (long i = 0; i < M; ++i) Unext[i] = W->d1[i] - W->d2[i];
}

int oracle_step(const oracle_problem *P, double *U, double t) {
  if (check_problem(P)) return -1;
  step_work W;
  long M = npoints(P) * P->nspecies;
  work_alloc(&W, M, P->dim);
  step_forward(P, U, t, &W, U);
  work_free(&W);
  return 0;
}

int oracle_run(const oracle_problem *P, double *U, double t0, long nsteps) {
  if (check_problem(P) || nsteps < 0) return -1;
  step_work W;
  long M = npoints(P) * P->nspecies;
  work_alloc(&W, M, P->dim);
  for (long n = 0; n < nsteps; ++n) step_forward(P, U, t0 + n * P->k, &W, U);
  work_free(&W);
  return 0;
}

/* ---------------------------------------------------------- the adjoint -- */

/* dD_s += -(k/gamma) <lam_s, B_a x_s> for the solve x = (I + k/gamma A_a)^{-1} b
 * whose right-hand-side adjoint is lam = (I + k/gamma A_a)^{-T} xbar:
 * d x / d D_s = -(I + k/gamma A_a)^{-1} (k/gamma) B_a x on species s. */
static void accumulate_dD(const oracle_problem *P, int a, double gamma, const double *lam,
                          const double *x, double *tmp, double *Dbar) {
  long N = npoints(P);
  axis_laplacian(P, a, x, tmp);
  if (P->coupled) {
    /* A_a = (B (x) Dc) / h^2: d/dDc[s][t] of the solve enters species s through B x_t,
     * so dL/dDc[s][t] += -(k/gamma) <lam_s, B x_t> (Dbar row-major, 4 entries) */
    for (int s2 = 0; s2 < 2; ++s2)
      for (int t2 = 0; t2 < 2; ++t2) {
        double acc = 0.0;
        for (long i = 0; i < N; ++i) acc += lam[s2 * N + i] * tmp[t2 * N + i];
        Dbar[2 * s2 + t2] += -(P->k / gamma) * acc;
      }
    return;
  }
  for (int s = 0; s < P->nspecies; ++s) {
    double acc = 0.0;
    for (long i = 0; i < N; ++i) acc += lam[s * N + i] * tmp[s * N + i];
    Dbar[s] += -(P->k / gamma) * acc;
  }
}

/* Reverse mode of step_forward, transposing each line of the frame in turn. */
int oracle_step_adjoint(const oracle_problem *P, const double *Un, double t,
                        const double *Ubar_next, double *Ubar_n, double *Dbar, double *pbar) {
  if (check_problem(P)) return -1;
  long M = npoints(P) * P->nspecies;
  int d = P->dim;
  double k = P->k;
  step_work W;
  work_alloc(&W, M, d);
  double *Unext = dalloc(M), *tmp = dalloc(M);
  double *f1b = dalloc(M), *f2b = dalloc(M), *fsb = dalloc(M), *Usb = dalloc(M);
  double *cUb = dalloc(M), *cfb = dalloc(M), *wb = dalloc(M);
  double *lT = dalloc(M), *lS = dalloc(M), *f0b = dalloc(M), *g = dalloc(M);
  double Dloc[4] = {0, 0, 0, 0};
  step_forward(P, Un, t, &W, Unext);

  /* U_{n+1} = d1 - d2, d1 = T_d f1, d2 = S_d f2 */
  oracle_axis_solve(P, d - 1, 3.0, 1, Ubar_next, f1b);
  accumulate_dD(P, d - 1, 3.0, f1b, W.d1, tmp, Dloc);
  for (long i = 0; i < M; ++i) tmp[i] = -Ubar_next[i];
  oracle_axis_solve(P, d - 1, 4.0, 1, tmp, f2b);
  accumulate_dD(P, d - 1, 4.0, f2b, W.d2, tmp, Dloc);
  /* f1 = 9 cU + 2k cf + k f*, f2 = 8 cU + 1.5k cf + 0.5k f* */
  for (long i = 0; i < M; ++i) {
    cUb[i] = 9.0 * f1b[i] + 8.0 * f2b[i];
    cfb[i] = 2.0 * k * f1b[i] + 1.5 * k * f2b[i];
    fsb[i] = k * f1b[i] + 0.5 * k * f2b[i];
  }
  /* f* = F(U*, t+k) */
  oracle_reaction_vjp(P, W.Ustar, t + k, fsb, Usb, pbar);
  /* U* = P_d w */
  oracle_axis_solve(P, d - 1, 1.0, 1, Usb, wb);
  accumulate_dD(P, d - 1, 1.0, wb, W.Ustar, tmp, Dloc);
  /* earlier axes in reverse: cU' = 9 T cU - 8 S cU, cf likewise, w' = P w */
  for (int a = d - 2; a >= 0; --a) {
    for (long i = 0; i < M; ++i) g[i] = 9.0 * cUb[i];
    oracle_axis_solve(P, a, 3.0, 1, g, lT);
    accumulate_dD(P, a, 3.0, lT, W.xT_U[a], tmp, Dloc);
    for (long i = 0; i < M; ++i) g[i] = -8.0 * cUb[i];
    oracle_axis_solve(P, a, 4.0, 1, g, lS);
    accumulate_dD(P, a, 4.0, lS, W.xS_U[a], tmp, Dloc);
    for (long i = 0; i < M; ++i) cUb[i] = lT[i] + lS[i];

    for (long i = 0; i < M; ++i) g[i] = 9.0 * cfb[i];
    oracle_axis_solve(P, a, 3.0, 1, g, lT);
    accumulate_dD(P, a, 3.0, lT, W.xT_f[a], tmp, Dloc);
    for (long i = 0; i < M; ++i) g[i] = -8.0 * cfb[i];
    oracle_axis_solve(P, a, 4.0, 1, g, lS);
    accumulate_dD(P, a, 4.0, lS, W.xS_f[a], tmp, Dloc);
    for (long i = 0; i < M; ++i) cfb[i] = lT[i] + lS[i];

    oracle_axis_solve(P, a, 1.0, 1, wb, lT);
    accumulate_dD(P, a, 1.0, lT, W.w[a + 1], tmp, Dloc);
    memcpy(wb, lT, sizeof(double) * M);
  }
  /* cU_0 = U_n, cf_0 = f0, w_0 = U_n + k f0, f0 = F(U_n, t) */
  for (long i = 0; i < M; ++i) f0b[i] = cfb[i] + k * wb[i];
  oracle_reaction_vjp(P, Un, t, f0b, tmp, pbar);
  for (long i = 0; i < M; ++i) Ubar_n[i] = cUb[i] + wb[i] + tmp[i];
  if (Dbar)
    for (int s = 0; s < (P->coupled ? 4 : P->nspecies); ++s) Dbar[s] += Dloc[s];

  work_free(&W);
  free(Unext);
  free(tmp);
  free(f1b);
  free(f2b);
  free(fsb);
  free(Usb);
  free(cUb);
  free(cfb);
  free(wb);
  free(lT);
  free(lS);
  free(f0b);
  free(g);
  return 0;
}

int oracle_grad(const oracle_problem *P, const double *U0, double t0, const double *target,
                long nsteps, double *loss, double *dU0, double *dD, double *dparams) {
  if (check_problem(P) || nsteps < 0) return -1;
  long M = npoints(P) * P->nspecies;
  double *states = (double *)malloc(sizeof(double) * (size_t)M * (size_t)(nsteps + 1));
  if (!states) return -2;
  memcpy(states, U0, sizeof(double) * M);
  step_work W;
  work_alloc(&W, M, P->dim);
  for (long n = 0; n < nsteps; ++n)
    step_forward(P, states + n * M, t0 + n * P->k, &W, states + (n + 1) * M);
  work_free(&W);
  const double *UN = states + nsteps * M;
  double L = 0.0;
  double *bar = dalloc(M), *bar2 = dalloc(M);
  for (long i = 0; i < M; ++i) {
    double r = UN[i] - target[i];
    L += 0.5 * r * r;
    bar[i] = r;
  }
  for (int s = 0; s < 4; ++s) dD[s] = 0.0;
  for (int j = 0; j < 8; ++j) dparams[j] = 0.0;
  for (long n = nsteps - 1; n >= 0; --n) {
    oracle_step_adjoint(P, states + n * M, t0 + n * P->k, bar, bar2, dD, dparams);
    memcpy(bar, bar2, sizeof(double) * M);
  }
  memcpy(dU0, bar, sizeof(double) * M);
  *loss = L;
  free(bar);
  free(bar2);
  free(states);
  return 0;
}
