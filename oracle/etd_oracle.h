/*
 * etd_oracle.h -- plain FP64 CPU oracle for the ETD-RDP-IF scheme.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or table with the CUDA library and must never be called by
 * the product path.
 *
 * What it computes (paper: Asante-Asamani, Kleefeld, Wade, "A second-order
 * exponential time differencing scheme for non-linear reaction-diffusion
 * systems with dimensional splitting", arXiv 2001.11220):
 *   - the model u_t = D Lap u + F(u) of Section 2 (Eq. model), s species,
 *     diagonal D, homogeneous Dirichlet / Neumann / periodic boundaries;
 *   - the coupled two-species form of Section 8 (complex Ginzburg-Landau
 *     with D = 1 + i alpha, the cubic Schrodinger equation with a
 *     non-diagonal D): a full 2 x 2 diffusion matrix, whose line systems
 *     I + (k/gamma)/h^2 (B_p (x) D) are solved as one system per line: the
 *     Thomas algorithm in 2 x 2 block form (Dirichlet, Neumann), dense LU
 *     with partial pivoting of the 2p x 2p matrix (periodic);
 *   - d = 1 as well as 2 and 3 (the frame with no splitting: the last-axis
 *     step alone);
 *   - the 1D matrices B_p of Section 3, Example 1 and the Kronecker operator
 *     A_i of Eq. (Ai), applied line by line;
 *   - the fully discrete ETD-RDP-IF scheme of the framed box in Section 6
 *     (Eq. donedone for d = 3, the d-dimensional frame for d = 2), evaluated
 *     in the order of the flow charts of Section 7 (Figs. flow2d / flow3d);
 *   - line solves by the Thomas variant of Section 7, periodic lines by a
 *     per-line Sherman-Morrison correction (the rank-one form of the
 *     Sherman-Morrison-Woodbury formula mentioned in Section 7);
 *   - the discrete adjoint (reverse mode) of that exact iteration.
 *
 * Layout: species-major, x fastest: U[s][z][y][x]; axis 0 = x = the factor
 * B_p at the last spatial Kronecker position of Eq. (Ai).
 *
 * Every function is pinned by tests (dense LU of the Kronecker-assembled
 * matrices, eigenmode closed forms, Heun's method for D = 0, conservation
 * invariants, convergence order, finite differences for the adjoint).
 */
#ifndef ETD_ORACLE_H
#define ETD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_DIRICHLET = 0, OR_NEUMANN = 1, OR_PERIODIC = 2 };
enum {
  OR_ZERO = 0,         /* F = 0 */
  OR_LINEAR = 1,       /* F_i = p0 * u_i + p1 */
  OR_BRUSSELATOR = 2,  /* F_u = a + u^2 v - (b+1) u ; F_v = b u - u^2 v ; p = (a, b) */
  OR_SCHNAKENBERG = 3, /* F_u = g (a - u + u^2 v) ; F_v = g (b - u^2 v) ; p = (a, b, g) */
  OR_GRAY_SCOTT = 4,   /* F_u = -u v^2 + F (1-u) ; F_v = u v^2 - (F+kappa) v ; p = (F, kappa) */
  OR_ENZYME = 5,       /* F = -u/(1+u) + p0 * src(x,t; p1) (Section 8.1, plus manufactured source) */
  OR_CGL = 6,          /* complex Ginzburg-Landau (Section 8): species 0, 1 = Re, Im of u;
                          F = u - (1 + i beta) u |u|^2 ; p = (beta) */
  OR_NLS = 7           /* cubic Schrodinger (Section 8): species 0, 1 = v, w (Psi = v + i w);
                          F = q J u with J = [[0, 1], [-1, 0]] and
                          q = p0 + p1 |u|^2 + p2 (1 - prod_a cos^2(pi x_a / L_a)) */
};

typedef struct {
  int dim;           /* 1, 2 or 3 */
  int n[3];          /* p_a: grid nodes per axis (paper convention per boundary type) */
  double length[3];  /* domain length per axis */
  int bc[3];         /* OR_DIRICHLET / OR_NEUMANN / OR_PERIODIC per axis */
  int nspecies;      /* s, 1..4 */
  double D[4];       /* diffusion coefficients */
  int reaction;      /* OR_* reaction kind */
  double params[8];  /* reaction parameters */
  double k;          /* time step */
  int coupled;       /* 1: species 0 and 1 diffuse through the full matrix Dc (s = 2; D unused) */
  double Dc[4];      /* 2 x 2 diffusion matrix, row-major: u_t = Dc Lap u + F(u) */
} oracle_problem;

/* spacing h of axis a (Section 3, Example 1) */
double oracle_h(const oracle_problem *P, int axis);

/* one line: solve (I + r B) x = b with B = h^2 B_p of Example 1 for boundary
 * type bc (r = c / h^2).  transpose != 0 solves with the transposed matrix. */
int oracle_line_solve(int p, int bc, double r, int transpose, const double *b, double *x);

/* all lines of one axis, all species: out = (I + (k/gamma) A_axis)^{-1} in
 * (transpose: the transposed operator).  in and out may alias.  Coupled
 * problems solve both species of a line together (returns -1 if that
 * 2p x 2p matrix is singular). */
int oracle_axis_solve(const oracle_problem *P, int axis, double gamma, int transpose,
                      const double *in, double *out);

/* out = A_axis in  (the Kronecker operator of Eq. (Ai) for one axis, times D;
 * for coupled problems species r of the output sums Dc[r][s] B_p u_s) */
int oracle_axis_apply(const oracle_problem *P, int axis, const double *in, double *out);

/* pointwise reaction F(U, t) over the grid (Section 2) */
int oracle_reaction(const oracle_problem *P, const double *U, double t, double *F);

/* pointwise products with the reaction Jacobian: out = J_F(U,t)^T ybar;
 * pbar[j] += sum over points of (dF/dparams_j)^T ybar */
int oracle_reaction_vjp(const oracle_problem *P, const double *U, double t, const double *ybar,
                        double *out, double *pbar);

/* one ETD-RDP-IF step in place: U <- U_{n+1} given U = U_n at time t */
int oracle_step(const oracle_problem *P, double *U, double t);
int oracle_run(const oracle_problem *P, double *U, double t0, long nsteps);

/* reverse mode of one step: given U_n (at time t) and Ubar_{n+1}, return
 * Ubar_n and accumulate Dbar[s] (d/dD_s) and pbar[j] (d/dparams_j).
 * Coupled problems: Dbar holds 4 entries, d/dDc[s][t] row-major (the
 * transposed solves are those of B^T (x) Dc^T). */
int oracle_step_adjoint(const oracle_problem *P, const double *Un, double t,
                        const double *Ubar_next, double *Ubar_n, double *Dbar, double *pbar);

/* loss L = 1/2 sum (U_N - target)^2 after nsteps from U0 at t0, and its
 * gradients w.r.t. U0, D and the reaction parameters (all states stored). */
int oracle_grad(const oracle_problem *P, const double *U0, double t0, const double *target,
                long nsteps, double *loss, double *dU0, double *dD, double *dparams);

/* host threads for the line and point loops of an OpenMP build (each line and
 * each point is computed exactly as in the serial loop; set 1 for one core). */
void oracle_set_threads(int n);
int oracle_get_threads(void);

#ifdef __cplusplus
}
#endif
#endif