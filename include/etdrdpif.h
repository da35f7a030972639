/*
 * etdrdpif.h -- C ABI of libetdrdpif, a GB300 (sm_103a) implementation of the
 * second-order L-stable ETD-RDP-IF scheme of Asante-Asamani, Kleefeld and
 * Wade, "A second-order exponential time differencing scheme for non-linear
 * reaction-diffusion systems with dimensional splitting" (arXiv 2001.11220).
 *
 * Problem (Section 2, Eq. model): u_t = D Lap u + F(u) for s species on a
 * d-dimensional box (d = 2, 3), diagonal D, homogeneous Dirichlet, Neumann or
 * periodic boundaries, second-order central differences (Section 3, Example 1
 * and Eq. Ai).  One time step is the framed ETD-RDP-IF scheme of Section 6
 * (Eq. donedone and its d-dimensional frame):
 *     U*      = P_d ... P_1 (U_n + k F(U_n, t_n))
 *     U_{n+1} = T_d [R_{d-1}..R_1 (9 U_n + 2k F(U_n)) + k F(U*, t_{n+1})]
 *             - S_d [R_{d-1}..R_1 (8 U_n + 3k/2 F(U_n)) + k/2 F(U*, t_{n+1})]
 * with P_a = (I + k A_a)^{-1}, T_a = (I + k/3 A_a)^{-1}, S_a = (I + k/4 A_a)^{-1},
 * R_a = 9 T_a - 8 S_a.  Every inverse is a set of independent line solves
 * along one axis (Section 7); periodic lines are cyclic and are solved with a
 * per-line Sherman-Morrison correction whose scalar is formed in FP64.
 *
 * Conventions shared by every entry point
 *   - State layout: species-major, x fastest: U[s][z][y][x] (2D: U[s][y][x]),
 *     contiguous, element type double (ETD_FP64) or float (ETD_FP32).
 *     Axis 0 = x is the B_p factor at the last spatial Kronecker slot of
 *     Eq. (Ai); the last axis carries T_d / S_d and F(U*).
 *   - Grid nodes per axis follow Section 3, Example 1: Dirichlet n interior
 *     nodes, h = L/(n+1); Neumann n nodes including both ends, h = L/(n-1);
 *     periodic n nodes, h = L/n.  n >= 3 on every axis.
 *   - Device pointers are CUDA device (or managed) memory owned by the
 *     caller; the library never frees them.  Host pointers are plain host
 *     memory.  The context owns its coefficient tables and scratch.
 *   - All device work is ordered on the context's stream; entry points
 *     return without synchronising unless stated otherwise.
 *   - Every entry point returns an etd_status and never aborts the process;
 *     on failure etd_last_error(ctx) describes the cause.
 */
#ifndef ETDRDPIF_H
#define ETDRDPIF_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  ETD_OK = 0,
  ETD_ERR_INVALID_ARG = 1, /* bad pointer, size, boundary, coefficient, step or reaction */
  ETD_ERR_UNSUPPORTED = 2, /* valid problem outside what the kernels implement */
  ETD_ERR_OOM = 3,         /* device or host allocation failed */
  ETD_ERR_CUDA = 4,        /* a CUDA runtime call or kernel launch failed */
  ETD_ERR_TIMEOUT = 5,     /* a bounded device wait gave up */
  ETD_ERR_NONFINITE = 6    /* a non-finite value was detected where checked */
} etd_status;

typedef enum { ETD_BC_DIRICHLET = 0, ETD_BC_NEUMANN = 1, ETD_BC_PERIODIC = 2 } etd_bc;
typedef enum { ETD_FP64 = 0, ETD_FP32 = 1 } etd_precision;

/* Reactions F(u) evaluated pointwise (Section 2; systems of Section 8 and the
 * benchmark problems).  params[] per kind:
 *   ZERO          F = 0
 *   LINEAR        F_i = p0 u_i + p1                                 (any s)
 *   BRUSSELATOR   F_u = p0 + u^2 v - (p1+1) u, F_v = p1 u - u^2 v    (s = 2;
 *                 Section 8.2 with B = p0, A = p1)
 *   SCHNAKENBERG  F_u = p2 (p0 - u + u^2 v), F_v = p2 (p1 - u^2 v)  (s = 2)
 *   GRAY_SCOTT    F_u = -u v^2 + p0 (1-u), F_v = u v^2 - (p0+p1) v   (s = 2)
 *   ENZYME        F = -u/(1+u) + p0 src(x,t), src the manufactured source
 *                 (p1 Sum_a (pi/L_a)^2 - 1) q + q/(1+q),
 *                 q = e^{-t} Prod_a sin(pi x_a/L_a)                 (s = 1;
 *                 Section 8.1; p0 = 0 gives the paper's enzyme model)
 *   CGL           complex Ginzburg-Landau of Section 8: species 0, 1 = Re u,
 *                 Im u, F = u - (1 + i p0) u |u|^2 (s = 2).  With etd_create
 *                 the diffusion is real (alpha = 0, the paper's runs); with
 *                 etd_create_coupled it is 1 + i alpha.
 *   NLS           cubic Schrodinger of Section 8 (etd_create_coupled only):
 *                 species 0, 1 = v, w (Psi = v + i w), F = q (w, -v) with
 *                 q = p0 + p1 (v^2 + w^2) + p2 (1 - Prod_a cos^2(pi x_a/L_a))
 *                 (s = 2; the paper's 2D example: p0 = 0, p1 = p2 = 1 - 2 pi^2) */
typedef enum {
  ETD_REACTION_ZERO = 0,
  ETD_REACTION_LINEAR = 1,
  ETD_REACTION_BRUSSELATOR = 2,
  ETD_REACTION_SCHNAKENBERG = 3,
  ETD_REACTION_GRAY_SCOTT = 4,
  ETD_REACTION_ENZYME = 5,
  ETD_REACTION_CGL = 6,
  ETD_REACTION_NLS = 7
} etd_reaction_kind;

typedef struct {
  int32_t dim;       /* 2 or 3 */
  int32_t bc[3];     /* etd_bc per axis (axis 0 = x) */
  int64_t n[3];      /* nodes per axis, 3 <= n <= 16384 */
  double length[3];  /* domain length per axis, > 0 */
} etd_grid;

typedef struct {
  int32_t kind;      /* etd_reaction_kind */
  int32_t nspecies;  /* s: 1 or 2 */
  double params[8];  /* see etd_reaction_kind */
} etd_reaction;

typedef struct etd_ctx etd_ctx;

/* Bytes of the static device scratch array behind etd_step_noalloc. */
#define ETD_NOALLOC_BYTES (64u * 1024u * 1024u)

/* Static facts about a context (for measurement and tuning). */
typedef struct {
  int32_t dim, nspecies, precision;
  int64_t npoints;               /* points per species */
  int64_t state_bytes;           /* bytes of one state U */
  int64_t scratch_bytes;         /* device scratch the context owns */
  int64_t algorithmic_bytes;     /* HBM bytes one step must move (sweep floor: 6d-4 fields
                                    read or written per species per point: 8 in 2D, 14 in 3D) */
  int32_t launches_per_step;     /* kernels one etd_step enqueues */
  int32_t chunk[3];              /* chunk length per axis (elements per thread) */
  int32_t lines_per_block[3];    /* lines per tile / block per axis */
  int32_t staged[3];             /* 0: register kernel, 1: persistent shared-memory-staged kernel,
                                    2: FP32 tile kernel (lines_per_block then counts line units),
                                    3: segmented register kernel (long lines split over blocks;
                                    summary, carry and solve launches), 4: the same in one launch,
                                    the blocks of a line group forming a thread-block cluster,
                                    5: circulant kernel of a periodic axis (constant-coefficient
                                    factorisation, no line tables), 6: complex line kernel of a
                                    coupled context (etd_create_coupled) */
  int32_t pack[3];               /* 2: FP32 register kernel on pairs of neighbouring lines
                                    (lines_per_block then counts pairs), 1: one line per thread;
                                    segmented kernels: chunks per segment */
  int32_t grid_blocks[3];        /* blocks of each axis's sweep launch (persistent circulant
                                    sweeps: the blocks resident at once) */
} etd_info;

/* Create a context for one problem.  Validates every argument
 * (ETD_ERR_INVALID_ARG on dim not 2/3, n < 3, bad bc, length <= 0, D < 0 or
 * non-finite, k <= 0 or non-finite, reaction kind / species mismatch),
 * factorises the line matrices I + (k/gamma) D_s B_p for gamma in {1,3,4} in
 * FP64 on the host (LU without pivoting, Section 7; the matrices are
 * diagonally dominant for every k > 0, D >= 0), uploads the tables in the
 * context's precision and allocates 3 s N elements of device scratch.
 * D points to nspecies host doubles.  stream is a cudaStream_t (NULL = legacy
 * default stream).  On success *out owns everything; free with etd_destroy. */
etd_status etd_create(const etd_grid *grid, const double *D, const etd_reaction *reaction,
                      double k, int32_t precision, void *stream, etd_ctx **out);

/* Create a context for a coupled two-species problem of Section 8:
 * u_t = Dm Lap u + F(u) with the 2 x 2 diffusion matrix Dm (4 host doubles,
 * row-major) acting on (u_0, u_1).  The kernels take Dm = [[p, -q], [q, p]]
 * with p >= 0 -- the complex coefficient p + i q on u = u_0 + i u_1: the
 * complex Ginzburg-Landau equation (p = 1, q = alpha) and the cubic
 * Schrodinger equation, whose form u_t + J Lap u = q J u with
 * J = [[0, 1], [-1, 0]] is Dm = -J (p = 0, q = 1).  Every line system
 * I + (k/gamma)(p + i q)/h^2 B_p is a complex tridiagonal (cyclic) matrix:
 * Dirichlet / Neumann lines are LU-factorised in FP64 on the host (strictly
 * diagonally dominant in modulus, no pivoting), periodic lines are factored
 * exactly as alpha (I - lam E)(I - lam E^-1) (E the cyclic shift, |lam| < 1);
 * the coefficients are uploaded in the context's precision.  nspecies must be 2 and
 * the reaction ZERO, LINEAR, CGL or NLS (else ETD_ERR_UNSUPPORTED, as for
 * another Dm; ETD_ERR_INVALID_ARG for a non-finite Dm or p < 0, and for the
 * grid / k / precision checks of etd_create).  Lines longer than about
 * 3200 nodes (FP64) / 6400 (FP32) do not fit the kernel's shared memory:
 * ETD_ERR_UNSUPPORTED.  grid->dim may also be 1 here (one line, the frame
 * without splitting, as in the paper's 1D Schrodinger run; n[0] and
 * length[0] as for the other axes).  The context takes etd_step, etd_run, etd_run_host,
 * etd_profile*, etd_get_info (staged = 6) and etd_destroy; the adjoint and
 * gradient calls and etd_autotune return ETD_ERR_UNSUPPORTED. */
etd_status etd_create_coupled(const etd_grid *grid, const double *Dm, const etd_reaction *reaction,
                              double k, int32_t precision, void *stream, etd_ctx **out);

/* One ETD-RDP-IF step in place: U (device, layout above) holds U_n at time
 * t_n on entry and U_{n+1} on return (stream-ordered). */
etd_status etd_step(etd_ctx *ctx, void *U, double t_n);
/* State pointers (U, U0, targets) must be 16-byte aligned when an axis runs
 * an FP32 tile kernel (etd_info.staged == 2; only after etd_autotune or an
 * ETD_TILES override): ETD_ERR_INVALID_ARG otherwise.  cudaMalloc and torch
 * allocations are. */

/* nsteps steps from time t0, in place on device U. */
etd_status etd_run(etd_ctx *ctx, void *U, double t0, int64_t nsteps);

/* Same as etd_run for a HOST buffer U_host: copies it to a device state the
 * context owns, runs, copies back and synchronises the stream before
 * returning.  Pinned host memory gives the fastest copies. */
etd_status etd_run_host(etd_ctx *ctx, void *U_host, double t0, int64_t nsteps);

/* Reverse mode of one step (the discrete adjoint of the frame above): given
 * U_n (device) at t_n and Ubar_next = dL/dU_{n+1} (device), writes
 * Ubar_n = dL/dU_n (device, may alias Ubar_next) and ADDS dL/dD_s into dD[s]
 * and dL/dparams_j into dparams[j] (host arrays of nspecies and 8 doubles;
 * either may be NULL).  Synchronises the stream.  The adjoint sweeps take
 * lines of one block (at most 4096 nodes): longer axes, D_s = 0 and coupled
 * contexts return ETD_ERR_UNSUPPORTED (so do etd_grad and etd_run_vjp). */
etd_status etd_step_adjoint(etd_ctx *ctx, const void *Un, double t_n, const void *Ubar_next,
                            void *Ubar_n, double *dD, double *dparams);

/* Loss L = 1/2 sum (U_N - target)^2 after nsteps from U0 (device) at t0 and
 * its gradients: dU0 (device), dD[nspecies], dparams[8] (host), with the
 * forward states checkpointed every ckpt_every steps and recomputed segment
 * by segment in the reverse sweep.  loss is a host double.  Synchronises. */
etd_status etd_grad(etd_ctx *ctx, const void *U0, double t0, const void *target, int64_t nsteps,
                    int64_t ckpt_every, double *loss, void *dU0, double *dD, double *dparams);

/* Vector-Jacobian product of a run: given U0 (device) at t0 and a cotangent
 * Ubar_N = dL/dU_N (device) of the state after nsteps steps, writes
 * dU0 = dL/dU0 (device) and dD[nspecies], dparams[8] (host) for any
 * differentiable L of U_N (the reverse pass of etd_grad with the misfit
 * replaced by the caller's cotangent; same checkpointing).  Synchronises. */
etd_status etd_run_vjp(etd_ctx *ctx, const void *U0, double t0, int64_t nsteps, int64_t ckpt_every,
                       const void *Ubar_N, void *dU0, double *dD, double *dparams);

/* Batched ensemble: ninst independent problems (grids[i], D[i*nspecies ..],
 * reactions[i]; all instances share nspecies, dim and precision; k is
 * common; ninst < 2^24) advanced together.  Each time step is ONE persistent
 * kernel launch (Section 7's step on every instance): resident blocks take
 * (axis, instance, line block) work items from a device queue ordered so
 * that every item's dependencies -- all blocks of the previous sweep of the
 * same instance -- come earlier, and wait for them on per-instance
 * completion counters with a bounded wait.  Periodic axes whose lines are
 * whole chunks are solved on the circulant factorisation of each line
 * system (no tables read); other axes use the line tables.  Multi-step runs
 * are captured into a CUDA graph and replayed.  (In the environment at
 * create time, ETD_ENSEMBLE_PERSISTENT=0 selects one launch per sweep kind
 * instead, with tables on every axis; ETD_ENSEMBLE_CIRC=0 keeps the tables
 * in the persistent step too, which then gives the same bits as the
 * per-sweep launches.)
 * etd_batch_run takes an array of ninst device state pointers (host array),
 * synchronises the context's stream and returns ETD_ERR_TIMEOUT if a
 * dependency wait gave up (the states are then incomplete; the counters are
 * reset and the context stays usable).  Other entry points reject batched
 * contexts. */
etd_status etd_batch_create(int32_t ninst, const etd_grid *grids, const double *D,
                            const etd_reaction *reactions, double k, int32_t precision,
                            void *stream, etd_ctx **out);
etd_status etd_batch_run(etd_ctx *ctx, void *const *U, double t0, int64_t nsteps);

/* Non-finite detection: scans the state U (device, layout above, the
 * context's precision) for NaN or infinity on the context's stream and
 * synchronises.  Returns ETD_OK, or ETD_ERR_NONFINITE with *first_bad (may be
 * NULL) set to the smallest flat element index s N + point that is not finite
 * (-1 when all are finite); ETD_ERR_INVALID_ARG for a NULL ctx or U or a
 * batched context.  A run that diverges (k too large for an explicit
 * reaction term, a blow-up of the model itself) is caught by calling this on
 * its result. */
etd_status etd_check_finite(etd_ctx *ctx, const void *U, int64_t *first_bad);

/* Limit of each dependency wait of the persistent ensemble step, in seconds
 * (default 1; (0, 60]).  ETD_ERR_INVALID_ARG on a single-problem context or
 * a limit outside the range. */
etd_status etd_batch_set_wait_limit(etd_ctx *ctx, double seconds);

/* Test hook of the bounded waits.  Seeds the completion counter of sweep
 * `axis` (0 .. dim-2) of instance `instance` with a value the next step's
 * blocks cannot raise to its target, so the first wait on it runs out and
 * the next etd_batch_run returns ETD_ERR_TIMEOUT (naming instance and
 * axis + 1).  Synchronises.  ETD_ERR_INVALID_ARG on indices out of range or
 * a context without the persistent step. */
etd_status etd_batch_debug_hold(etd_ctx *ctx, int32_t instance, int32_t axis);

/* Choose the ensemble's line-block shapes (the chunk length of every axis,
 * shared by all instances; each instance then fills the common block size
 * with as many lines as fit) by timing every candidate on the context's
 * stream with CUDA events.  U_work: ninst device states of the instances'
 * shapes, used as scratch (overwritten).  Synchronises; captured graphs are
 * dropped.  ETD_ERR_INVALID_ARG on a single-problem context or null
 * pointers. */
etd_status etd_batch_autotune(etd_ctx *ctx, void *const *U_work);

/* Re-plan every axis by timing each candidate sweep on the context's stream
 * with CUDA events and keeping the fastest: the kernel family (register,
 * FP32 line pairs, staged, FP32 tile, segmented or cluster-segmented for
 * long lines), the chunk length, the lines per block and, for segmented
 * sweeps, the chunks per segment (etd_get_info reports the choice; every
 * candidate computes the same step).  U_work: a device state of the
 * context's shape, used as scratch (overwritten).  Synchronises; captured
 * graphs are dropped.  ETD_ERR_INVALID_ARG on a batched context or a null
 * pointer. */
etd_status etd_autotune(etd_ctx *ctx, void *U_work);

etd_status etd_set_stream(etd_ctx *ctx, void *stream);

/* Per-sweep timing for measurement.  While enabled, runs launch kernels
 * directly (no graph) and bracket every sweep launch with CUDA events on the
 * context's stream; etd_profile_read synchronises, adds the elapsed device
 * time of each sweep kind (0 = first axis, 1 = middle axis, 2 = last axis)
 * to ms[3] and the launch counts to launches[3], and clears the record. */
etd_status etd_profile(etd_ctx *ctx, int32_t enable);
etd_status etd_profile_read(etd_ctx *ctx, double *ms, int64_t *launches);
etd_status etd_get_info(const etd_ctx *ctx, etd_info *info);

/* One step without any device allocation.  The paper has no counterpart:
 * this exists for callers that cannot call cudaMalloc -- plugins whose host
 * application owns every device allocation through its own pool, and
 * real-time loops that must not touch the allocator after start-up.  Same
 * arguments as etd_create plus the state: U (device, layout above) holds U_n
 * at t_n on entry and U_{n+1} on return.  Scratch (the three carried fields
 * and the line tables) lives in one static __device__ array of
 * ETD_NOALLOC_BYTES (64 MiB) that every GPU loading the library keeps until
 * exit.  Limits, checked before any device work:
 *   - 3 s N elements plus the line tables must fit the array, else
 *     ETD_ERR_INVALID_ARG;
 *   - every axis must fit one block of whole lines (at most 512 chunks of
 *     16 positions: n <= 8192 per axis), else ETD_ERR_UNSUPPORTED (the
 *     segmented plans of etd_create need device buffers this call does not
 *     have).
 * Every call looks up the array's device address (cudaGetSymbolAddress) in
 * the CUDA context current on the calling thread, so a host that switches
 * contexts or resets the device gets the address valid for the current one.
 * Each call recomputes the line tables on the host, copies them into the
 * array on `stream` and synchronises that stream once before launching the
 * sweeps.  All calls share the one array and keep the last call's contents:
 * calls that overlap on the GPU (other streams, other host threads) race. */
etd_status etd_step_noalloc(const etd_grid *grid, const double *D, const etd_reaction *reaction, double k,
                            int32_t precision, void *U, double t_n, void *stream);

/* Description of the last failure on ctx (or of the last failed etd_create /
 * etd_batch_create when ctx is NULL).  Never NULL. */
const char *etd_last_error(const etd_ctx *ctx);

/* Frees everything the context owns; NULL is accepted. */
void etd_destroy(etd_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif
