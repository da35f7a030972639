// etd_internal.h -- types shared by the host side and the sweep kernels of
// libetdrdpif.  Nothing here is part of the public C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace etd {

// The three fused sweeps of one step (Section 7, Figs. flow2d / flow3d):
//  FIRST  (axis 0, contiguous lines): F(U_n, t_n), the five solves
//         T,S on U_n; T,S on F(U_n); P on U_n + k F(U_n)  -> c_U, c_f, w
//  MIDDLE (axis 1 of a 3D grid, strided lines): the same five solves applied
//         to (c_U, c_f, w) in place (R_2 on c_U and c_f, P_2 on w)
//  LAST   (axis d-1, strided lines): U* = P_d w, F(U*, t_{n+1}),
//         f1 = 9 c_U + 2k c_f + k F*, f2 = 8 c_U + 3k/2 c_f + k/2 F*,
//         U_{n+1} = T_d f1 - S_d f2
enum SweepKind { SWEEP_FIRST = 0, SWEEP_MIDDLE = 1, SWEEP_LAST = 2 };

constexpr int MAX_SPECIES = 2;

template <typename R> struct V4T;
template <> struct V4T<float> { using T = float4; };
template <> struct V4T<double> { using T = double4; };
template <typename R> struct V2T;
template <> struct V2T<float> { using T = float2; };
template <> struct V2T<double> { using T = double2; };

// Tables of one line matrix M = I + (k/gamma) D_s B_p (or its modified
// tridiagonal part M' for periodic lines), chunked into m chunks of L
// positions, stored chunk-major: entry (t, j) at index j*L + t, i.e. the
// t-th position of chunk j (a thread's L entries are contiguous).  Positions past the end of the line are identity
// rows (nl = 0, e = 1, alpha = 0, z = 0, v = w = 0).
//   pos[j*L+t]   = (nl, e, alpha, z): forward g_i = (b_i + nl_i g_{i-1}) e_i
//                  (nl = minus the sub-diagonal, e = 1 / pivot), backward
//                  x_i = g_i - alpha_i x_{i+1}, Sherman-Morrison vector z
//                  (periodic only)
//   sum[j*L+t]   = (v, w): chunk summaries F_j = sum v b (zero-carry forward
//                  value at the chunk end) and Y_j = sum w b (zero-carry
//                  backward value at the chunk start)
//   chunk[j]     = (Aend, kappa, Bst, 0): with a_i = -l_i e_i,
//                  G_in[j+1] = Aend G_in[j] + F_j;
//                  X[j] = Y_j + kappa G_in[j] + Bst X[j+1]
//   e1, v1, w1, z1 [j*L+t]: the same e, v, w, z as separate arrays, read four
//                  positions at a time in interior chunks (0 < j < m-1), where
//                  every row has l = u = -r: nl = r, alpha = -r e
//   rows1 (FP32 forward sweeps): six rows of m*L entries, row k at k*m*L:
//                  ne = nl e, e, -alpha, z, v, w at every position (the forward
//                  recurrence as g_i = ne_i g_{i-1} + e_i b_i)
//   rows2 (FP32 line pairs): the same rows with each value in both lanes of a float2
template <typename R> struct MatTab {
  const typename V4T<R>::T *pos;
  const typename V2T<R>::T *sum;
  const typename V4T<R>::T *chunk;
  const R *e1, *v1, *w1, *z1;
  const R *rows1;
  const typename V2T<R>::T *rows2;
  // segmented sweeps: per segment of mx chunks (A_seg, K_seg, B_seg, 0) with
  // G_out = A_seg G_in + F_seg and X_start = Y_seg + K_seg G_in + B_seg X_end
  const typename V4T<R>::T *segc;
  double r;       // interior off-diagonal magnitude
  double sm_c;    // v_{p-1} of the Sherman-Morrison rank-one term (periodic)
  double sm_inv;  // 1 / (1 + v.z)                                  (periodic)
};

// Shared-memory staging plan of the persistent sweep kernels (byte offsets
// into dynamic shared memory; every region 16-byte aligned).
struct StagePlan {
  int staged;       // 0: register kernel, 1: persistent shared-memory-staged kernel,
                    // 2: FP32 tile kernel (one tile of whole lines per block, compile-time geometry)
  int tile_elems;   // elements of one staged field tile
  int tile_pitch;   // tile kernel, x axis: row pitch (elements) of a field tile
  int nin;          // staged input fields per tile
  int nbuf;         // 1 or 2 tile buffers (2 = next tile prefetched during compute)
  int vec;          // strided tiles: 1 = 16-byte async copies per row segment
  int ntiles;       // tiles of this instance
  unsigned off_buf, off_f0, off_out, off_sum, off_sig, bytes;
};

// Everything one sweep launch needs for one problem instance.
template <typename R> struct SweepArgs {
  const R *in[3];  // FIRST: in[0] = U_n.  MIDDLE/LAST: c_U, c_f, w
  R *out[3];       // FIRST/MIDDLE: c_U, c_f, w.  LAST: out[0] = U_{n+1}
  long long N;     // points per species (species stride in elements)
  long long st;    // element stride of the swept axis
  long long nlines;  // lines of the swept axis = N / n
  int n;           // nodes on the swept axis
  int nlo_blocks;  // strided sweeps: blocks along the low (contiguous) line index
  int m;           // chunks per line
  int nlb;         // lines per block (blockDim.x = nlb * m)
  int pitch;       // shared-memory pitch of one line's chunk summaries
  int nblocks;     // blocks of this instance
  MatTab<R> mat[MAX_SPECIES][3];  // [species][0: P (gamma 1), 1: T (gamma 3), 2: S (gamma 4)]
  double k;        // time step
  double t_eval;   // time at which F is evaluated in this sweep
  double exp_mt;   // e^{-t_eval} (manufactured source)
  int rkind;       // etd_reaction_kind
  double rp[8];    // reaction parameters
  const R *phi[3]; // sin(pi x_a / L_a) per axis (manufactured source), NULL otherwise
  int nx, ny;      // grid extents of axes 0 and 1 (point -> coordinates)
  double src_lf;   // Sum_a (pi / L_a)^2
  // k, the reaction parameters, src_lf and e^{-t_eval} rounded to R once on
  // the host (the kernels never convert FP64 parameters per thread)
  R kR, src_lfR, exp_mtR;
  R rpR[8];
  int axis;        // swept axis
  int pk;          // 2: register kernel on line pairs (nlb counts pairs), else 1
  // Segmented sweeps: a line longer than one block's mx chunks is split over
  // nseg blocks.  Summary launches write each segment's zero-carry chunk-chain
  // values, a carry launch chains the segments of every line, and solve
  // launches start their chunk chains from those carries (SegPhase).
  int mx;          // chunks per block along the line (= m for whole-line blocks)
  int nseg;        // segments per line (1: whole lines)
  int segphase;    // SegPhase of this launch
  R *seg_sum;      // [solve][line][segment] (F_seg, Y_seg), zero carries
  R *seg_car;      // [solve][line][segment] (G_in, X_end)
  R *seg_sig;      // [solve][line] Sherman-Morrison scalar of the whole line
  StagePlan sp;    // staged-kernel plan
  // adjoint sweeps only
  MatTab<R> matT[MAX_SPECIES][3];  // tables of the transposed line matrices
  const R *fin[3];                 // forward quantities recomputed for this sweep
  double *acc;                     // device accumulators: dL/dD[MAX_SPECIES], dL/dparams[8]
  double *part;                    // per-block partial sums [nblocks][MAX_SPECIES + 8], added to acc
                                   // in a fixed order by a second launch (reproducible sums)
  double invD[MAX_SPECIES];        // 1 / D_s
  int circ_adj = 0;  // adjoint sweep on the circulant factorisation (cl below), else the tables
  int circ_fwd = 0;  // ensemble sweep of periodic whole-chunk lines on the circulant factorisation (cl)
  // adjoint sweeps of periodic axes on the circulant factorisation
  // M = alpha (I - lambda E)(I - lambda E^{-1}) (M is symmetric, so M^T = M):
  // per [species][0: P, 1: T, 2: S]
  struct CircLine {
    R lam, lamL, kap, inv1m, ialpha;  // lambda, lambda^L, sum_{s<L} lambda^{2s+1}, 1/(1 - lambda^p), 1/alpha
    R pw[16];                          // lambda^t, t < L
  } cl[MAX_SPECIES][3];
};

// Launch phases of a segmented sweep.  FIRST/MIDDLE: SEG_SUMMARY writes the
// segment summaries of all solves, SEG_SOLVE solves from the carries.  LAST:
// SEG_SUMMARY covers the P solves; SEG_SOLVE solves P from its carries, forms
// U*, F* and f1, f2 and writes the summaries of the T and S solves; SEG_FINAL
// solves everything from its carries.  SEG_WHOLE: lines are not split.
// SEG_CLUSTER: one launch; the nseg blocks of a line group form a thread-block
// cluster and exchange their segment summaries through distributed shared
// memory (one exchange per dependent group of solves: FIRST/MIDDLE one, LAST two).
enum SegPhase { SEG_WHOLE = 0, SEG_SUMMARY = 1, SEG_SOLVE = 2, SEG_FINAL = 3, SEG_CLUSTER = 4 };

// largest cluster of a cluster-segmented sweep (16 needs the non-portable size)
constexpr int ETD_MAX_CLUSTER = 16;

enum AdjKind { ADJ_FIRST = 0, ADJ_MIDDLE = 1, ADJ_LAST = 2 };

// host-side launchers (one translation unit per element type)
cudaError_t launch_sweep(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads,
                         size_t smem, cudaStream_t s);
cudaError_t launch_sweep(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads,
                         size_t smem, cudaStream_t s);
// batched: args[] in device memory, block_start[i] = first block of instance i (prefix, ninst+1)
cudaError_t launch_sweep_batched(const SweepArgs<float> *args_dev, const int *block_start_dev, int ninst,
                                 int total_blocks, int nspecies, int L, int kind, int nthreads,
                                 size_t smem, cudaStream_t s, double t_eval);
cudaError_t launch_sweep_batched(const SweepArgs<double> *args_dev, const int *block_start_dev, int ninst,
                                 int total_blocks, int nspecies, int L, int kind, int nthreads,
                                 size_t smem, cudaStream_t s, double t_eval);

// Persistent ensemble step (etd_ensemble.cuh): one launch advances every
// instance of a batched context by one step.
// status words: [0] non-zero once a dependency wait gave up, [1] instance,
// [2] axis of the first wait that gave up
constexpr int ENS_STATUS_WORDS = 4;

template <typename R> struct EnsArgs {
  const SweepArgs<R> *args[3];  // per axis: SweepArgs of every instance (device)
  const int2 *items;            // work list: x = axis << 24 | instance, y = block of that sweep
  int nitems;
  int ninst;
  unsigned *queue;              // [0] next item, [1] blocks that have left the loop
  int *done;                    // [axis][instance]: finished blocks (axes 0 .. dim - 2)
  int *status;                  // ENS_STATUS_WORDS words
  long long wait_ns;            // limit of one dependency wait (%globaltimer)
  double t_eval[3];             // time at which each sweep evaluates F
  R exp_mt[3];                  // e^{-t_eval} in R
};

// L0: chunk length of axis 0, LS: of axes 1 and 2.  resident != nullptr:
// only report the blocks resident at once (blocks per SM x SMs)
cudaError_t launch_ensemble_2d(const EnsArgs<float> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident);
cudaError_t launch_ensemble_3d(const EnsArgs<float> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident);
cudaError_t launch_ensemble_2d(const EnsArgs<double> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident);
cudaError_t launch_ensemble_3d(const EnsArgs<double> &E, int nspecies, int L0, int LS, int nthreads, size_t smem,
                               int grid, cudaStream_t s, int *resident);

// cluster-segmented register sweeps (a.segphase = SEG_CLUSTER; FP32 L = 8 or
// 16, FP64 L = 4 or 8): the launch, and the clusters that fit on the device
// at once (0: the configuration cannot launch)
cudaError_t launch_sweep_cluster(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                 cudaStream_t s);
cudaError_t launch_sweep_cluster(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads,
                                 size_t smem, cudaStream_t s);
cudaError_t sweep_cluster_capacity(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads,
                                   size_t smem, int &nclusters);
cudaError_t sweep_cluster_capacity(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads,
                                   size_t smem, int &nclusters);

// FP32 tile kernels: NLB lines per block, pk = 1 or 2 (line pairs, strided axes)
cudaError_t launch_tile(const SweepArgs<float> &a, int nspecies, int L, int NLB, int kind, int pk, int nthreads,
                        size_t smem, cudaStream_t s);
cudaError_t launch_tile_first(const SweepArgs<float> &a, int nspecies, int L, int NLB, int nthreads, size_t smem,
                              cudaStream_t s);
cudaError_t launch_tile_middle(const SweepArgs<float> &a, int nspecies, int L, int NLB, int pk, int nthreads,
                               size_t smem, cudaStream_t s);
cudaError_t launch_tile_last(const SweepArgs<float> &a, int nspecies, int L, int NLB, int pk, int nthreads,
                             size_t smem, cudaStream_t s);

// carries of the segments of every line for solves q0 .. q0+nq-1 (segmented sweeps)
cudaError_t launch_seg_carry(const SweepArgs<float> &a, int nspecies, int kind, int q0, int nq, cudaStream_t s);
cudaError_t launch_seg_carry(const SweepArgs<double> &a, int nspecies, int kind, int q0, int nq, cudaStream_t s);

cudaError_t launch_adjoint(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                           cudaStream_t s);
// the adjoint sweeps on the circulant factorisation (a.circ_adj; FP32 L = 8, FP64 L = 4)
cudaError_t launch_adjoint_circ(const SweepArgs<float> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                cudaStream_t s);
cudaError_t launch_adjoint_circ(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                                cudaStream_t s);
cudaError_t launch_adjoint(const SweepArgs<double> &a, int nspecies, int L, int kind, int nthreads, size_t smem,
                           cudaStream_t s);
// part: at least loss_blocks(n) doubles of per-block partial sums
int loss_blocks(long long n);
cudaError_t launch_loss(const float *U, const float *target, float *Ubar, long long n, double *loss, double *part,
                        cudaStream_t s);
cudaError_t launch_loss(const double *U, const double *target, double *Ubar, long long n, double *loss, double *part,
                        cudaStream_t s);

// shared-memory bytes of one adjoint sweep block
inline size_t adjoint_smem_bytes(int kind, int nspecies, int nlb, int pitch, size_t real_bytes) {
  int nq = (kind == ADJ_LAST) ? 6 * nspecies : 10 * nspecies;
  size_t sums = (size_t)2 * nq * nlb * pitch * real_bytes;
  sums = (sums + 15) & ~(size_t)15;
  return sums + (size_t)nq * nlb * sizeof(double) + 16 * sizeof(double) * 32;
}

// Row pitch of the chunk-summary exchange: odd (rows of neighbouring lines
// fall on different banks) and at least m rounded up to 8, so the carry
// chain can read whole batches of 8 chunks without bounds tests (chunk
// tables are padded with zeros to the same multiple of 8).
inline int exchange_pitch(int m) { return ((m + 7) & ~7) + 1; }

// shared-memory bytes of one sweep block (pk = 2: nlb line pairs); the
// Sherman-Morrison scalars take 8 bytes each (stored in the sweep's precision)
// chunk-table cache of a cluster-segmented sweep block: the chunk entries
// (A_j, kappa_j, B_j) of its chunks for the 3 matrices of every species
// (pitch - 1 entries each, the padded chunk count) and the nseg segment
// entries of each matrix
inline size_t chunk_cache_bytes(int nspecies, int pitch, size_t real_bytes, int nseg = 0) {
  return (size_t)3 * nspecies * ((size_t)(pitch - 1) + (size_t)nseg) * 4 * real_bytes;
}

// cluster-segmented sweeps add the segment summaries (G, X) of every
// (solve, line unit), read by the other blocks of the cluster
inline size_t sweep_smem_bytes(int kind, int nspecies, int nlb, int pitch, size_t real_bytes, int pk = 1,
                               bool cluster = false, int nseg = 1) {
  int nq = (kind == SWEEP_LAST) ? 3 * nspecies : 5 * nspecies;
  size_t sums = (size_t)2 * nq * nlb * pitch * real_bytes * pk;
  sums = (sums + 15) & ~(size_t)15;
  size_t sig = ((size_t)nq * nlb * pk * sizeof(double) + 15) & ~(size_t)15;
  size_t seg = cluster ? (((size_t)2 * nq * nlb * pk * real_bytes + 15) & ~(size_t)15) : 0;
  return sums + sig + seg + (cluster ? chunk_cache_bytes(nspecies, pitch, real_bytes, nseg) : 0);
}

}  // namespace etd
