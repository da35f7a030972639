// etd_api.cu -- C ABI of libetdrdpif: contexts, FP64 pre-factorisation,
// launch planning and the forward step.  See include/etdrdpif.h.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_circ.h"
#include "etd_context.h"
#include "etd_internal.h"
#include "etd_tables.h"

using namespace etd;

static thread_local std::string g_create_error = "no error";

const char *etd_last_error(const etd_ctx *ctx) {
  if (!ctx) return g_create_error.c_str();
  return ctx->err.c_str();
}

namespace etd {

etd_status fail(etd_ctx *ctx, etd_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_create_error = buf;
  return st;
}

etd_status cuda_fail(etd_ctx *ctx, cudaError_t e, const char *what) {
  return fail(ctx, ETD_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

// ------------------------------------------------------------ validation

etd_status validate_problem(const etd_grid *grid, const double *D, const etd_reaction *rx, double k,
                            int32_t precision) {
  if (!grid || !D || !rx) return fail(nullptr, ETD_ERR_INVALID_ARG, "null grid, D or reaction");
  if (grid->dim != 2 && grid->dim != 3) return fail(nullptr, ETD_ERR_INVALID_ARG, "dim must be 2 or 3 (got %d)", grid->dim);
  for (int a = 0; a < grid->dim; ++a) {
    if (grid->n[a] < 3 || grid->n[a] > 16384)
      return fail(nullptr, ETD_ERR_INVALID_ARG, "n[%d] = %lld outside [3, 16384]", a, (long long)grid->n[a]);
    if (grid->bc[a] < 0 || grid->bc[a] > 2) return fail(nullptr, ETD_ERR_INVALID_ARG, "bc[%d] = %d invalid", a, grid->bc[a]);
    if (!(grid->length[a] > 0) || !std::isfinite(grid->length[a]))
      return fail(nullptr, ETD_ERR_INVALID_ARG, "length[%d] must be finite and > 0", a);
  }
  if (!(k > 0) || !std::isfinite(k)) return fail(nullptr, ETD_ERR_INVALID_ARG, "k must be finite and > 0");
  if (precision != ETD_FP64 && precision != ETD_FP32) return fail(nullptr, ETD_ERR_INVALID_ARG, "precision %d invalid", precision);
  const int S = rx->nspecies;
  if (S < 1) return fail(nullptr, ETD_ERR_INVALID_ARG, "nspecies must be >= 1");
  if (S > MAX_SPECIES) return fail(nullptr, ETD_ERR_UNSUPPORTED, "nspecies %d > %d", S, MAX_SPECIES);
  for (int s = 0; s < S; ++s)
    if (!(D[s] >= 0) || !std::isfinite(D[s])) return fail(nullptr, ETD_ERR_INVALID_ARG, "D[%d] must be finite and >= 0", s);
  switch (rx->kind) {
    case ETD_REACTION_ZERO:
    case ETD_REACTION_LINEAR: break;
    case ETD_REACTION_BRUSSELATOR:
    case ETD_REACTION_SCHNAKENBERG:
    case ETD_REACTION_GRAY_SCOTT:
    case ETD_REACTION_CGL:
      if (S != 2) return fail(nullptr, ETD_ERR_INVALID_ARG, "reaction %d needs 2 species", rx->kind);
      break;
    case ETD_REACTION_ENZYME:
      if (S != 1) return fail(nullptr, ETD_ERR_INVALID_ARG, "enzyme reaction needs 1 species");
      break;
    case ETD_REACTION_NLS:
      return fail(nullptr, ETD_ERR_UNSUPPORTED, "the Schrodinger reaction needs etd_create_coupled");
    default: return fail(nullptr, ETD_ERR_INVALID_ARG, "unknown reaction kind %d", rx->kind);
  }
  for (int j = 0; j < 8; ++j)
    if (!std::isfinite(rx->params[j])) return fail(nullptr, ETD_ERR_INVALID_ARG, "params[%d] not finite", j);
  return ETD_OK;
}

// ------------------------------------------------------------ planning


static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

static int pow2_floor(long long v) {
  int p = 1;
  while ((long long)p * 2 <= v) p *= 2;
  return p;
}

// shared-memory plan of the staged kernel for nlb lines per tile and nbuf buffers
static StagePlan stage_plan(const Instance &I, const AxisPlan &P, int nlb, int nbuf) {
  StagePlan sp{};
  const bool contig = P.kind == SWEEP_FIRST;
  const int S = I.S, rb = I.real_bytes;
  const long long n = P.nlines > 0 ? I.N / P.nlines : 1;
  const int nin = contig ? S : 3 * S;
  const int nq = (P.kind == SWEEP_LAST) ? 3 * S : 5 * S;
  const int pitch = exchange_pitch(P.m);
  const long long mL = (long long)P.m * P.L;  // positions per line incl. zero padding
  long long te = contig ? (long long)nlb * (mL + 1) : mL * nlb;
  te = (te + 3) & ~3LL;
  sp.staged = 1;
  sp.tile_elems = (int)te;
  sp.nin = nin;
  sp.nbuf = nbuf;
  const int VW = 16 / rb;
  sp.vec = (!contig && P.st % VW == 0 && nlb % VW == 0) ? 1 : 0;
  sp.off_buf = 0;
  size_t off = align16((size_t)nbuf * nin * te * rb);
  sp.off_f0 = (unsigned)off;  // unused: F(U_n) stays in registers
  sp.off_out = (unsigned)off;
  if (contig) off = align16(off + (size_t)(P.kind == SWEEP_LAST ? 1 : 3) * S * te * rb);
  sp.off_sum = (unsigned)off;
  off = align16(off + (size_t)2 * nq * nlb * pitch * rb);
  sp.off_sig = (unsigned)off;
  off += (size_t)nq * nlb * sizeof(double);
  sp.bytes = (unsigned)off;
  if (contig) sp.ntiles = (int)((P.nlines + nlb - 1) / nlb);
  else sp.ntiles = (int)(((P.st + nlb - 1) / nlb) * (I.N / (P.st * n)));
  return sp;
}

static const size_t kStageSmemCap = 220 * 1024;      // one block per SM
static const size_t kStageSmemHalf = 110 * 1024;     // two blocks per SM

// lines-per-block and chunk count for one axis and chunk length L.  Lines
// short enough to stage go to the persistent double-buffered kernel; longer
// ones to the register kernel.  nlb_force > 0 asks for the staged kernel with
// that many lines per tile, reg_force for the register kernel (autotuning).
bool plan_axis_ex(Instance &I, int a, int L, int max_threads, int nlb_force, bool reg_force, int pack) {
  AxisPlan &P = I.plan[a];
  const long long n = I.n[a];
  P.L = L;
  P.m = (int)((n + L - 1) / L);
  if (P.m > max_threads) return false;
  P.kind = (a == 0) ? SWEEP_FIRST : (a == I.dim - 1 ? SWEEP_LAST : SWEEP_MIDDLE);
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  P.st = st;
  P.nlines = I.N / n;
  P.pitch = exchange_pitch(P.m);
  P.pk = 1;
  P.mx = P.m;
  P.nseg = 1;
  P.cluster = false;
  P.circ = false;
  if (pack == 2) {
    // register kernel on line pairs (lo, lo + 1) of a strided FP32 axis with an even stride
    if (I.real_bytes != 4 || a == 0 || st % 2 != 0 || L != 8) return false;
    const long long npairs = st / 2;
    int nlb = std::max(1, max_threads / P.m);
    if (nlb >= 32) nlb = (nlb / 32) * 32;
    nlb = (int)std::min<long long>(nlb, ((npairs + 31) / 32) * 32);
    nlb = std::max(1, nlb);
    if (nlb_force > 0 && nlb_force <= nlb) nlb = nlb_force;
    P.pk = 2;
    P.sp = StagePlan{};
    P.nlb = nlb;
    P.nlo_blocks = (int)((npairs + nlb - 1) / nlb);
    P.nblocks = (int)(P.nlo_blocks * (I.N / (st * n)));
    P.nthreads = nlb * P.m;
    P.smem = sweep_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes, 2);
    return P.smem <= 200 * 1024;
  }
  // staged plan: largest power-of-two lines per tile that fits with double buffering
  P.sp = StagePlan{};
  {
    const int cap = (a == 0) ? 64 : (I.real_bytes == 4 ? 32 : 16);
    const long long avail = (a == 0) ? P.nlines : st;
    int top = pow2_floor(std::min<long long>(std::min(cap, max_threads / P.m), std::max<long long>(1, avail)));
    if (top < avail && top * 2 <= std::min(cap, max_threads / P.m)) top *= 2;
    // prefer two resident blocks per SM (their exchange phases overlap), then one
    int chosen = 0;
    if (nlb_force > 0 && !reg_force) {
      if (nlb_force * P.m > max_threads || stage_plan(I, P, nlb_force, 2).bytes > kStageSmemCap) return false;
      chosen = nlb_force;
    }
    for (int nlb = top; nlb >= 8 && !chosen && !reg_force; nlb /= 2)
      if (stage_plan(I, P, nlb, 2).bytes <= kStageSmemHalf) chosen = nlb;
    for (int nlb = top; nlb >= 4 && !chosen && !reg_force; nlb /= 2)
      if (stage_plan(I, P, nlb, 2).bytes <= kStageSmemCap) chosen = nlb;
    if (chosen) {
      P.sp = stage_plan(I, P, chosen, 2);
      P.nlb = chosen;
      P.nthreads = chosen * P.m;
      P.nlo_blocks = (a == 0) ? 1 : (int)((st + chosen - 1) / chosen);
      P.nblocks = P.sp.ntiles;
      P.smem = P.sp.bytes;
      return true;
    }
  }
  if (a == 0) {
    int nlb = pow2_floor(std::min(32, std::max(1, max_threads / P.m)));
    if (reg_force && nlb_force > 0 && nlb_force <= nlb) nlb = nlb_force;
    while (nlb > 1 && nlb / 2 >= P.nlines) nlb /= 2;
    // short lines: many lines per block, but their exchange buffers must fit
    while (nlb > 1 && sweep_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes) > 200 * 1024) nlb /= 2;
    P.nlb = nlb;
    P.nlo_blocks = 1;
    P.nblocks = (int)((P.nlines + nlb - 1) / nlb);
  } else {
    int nlb = std::max(1, max_threads / P.m);
    if (nlb >= 32) nlb = (nlb / 32) * 32;
    nlb = (int)std::min<long long>(nlb, ((st + 31) / 32) * 32);
    nlb = std::max(1, nlb);
    if (reg_force && nlb_force > 0 && nlb_force <= nlb) nlb = nlb_force;
    while (nlb > 1 && sweep_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes) > 200 * 1024) nlb /= 2;
    P.nlb = nlb;
    P.nlo_blocks = (int)((st + nlb - 1) / nlb);
    const long long nhi = I.N / (st * n);
    P.nblocks = (int)(P.nlo_blocks * nhi);
  }
  P.nthreads = P.nlb * P.m;
  P.smem = sweep_smem_bytes(P.kind, I.S, P.nlb, P.pitch, I.real_bytes);
  return P.smem <= 200 * 1024;
}

bool plan_axis(Instance &I, int a, int L, int max_threads) { return plan_axis_ex(I, a, L, max_threads, 0, false, 1); }

// FP32 tile kernel: NLB lines per block (NLB / pk line units of L-position
// chunks), every input field of the block's lines staged in shared memory
// with 16-byte copies (strided axes: stride a multiple of 4 elements; x axis:
// line length a multiple of 4)
bool plan_axis_tile(Instance &I, int a, int L, int NLB, int pk) {
  AxisPlan &P = I.plan[a];
  const long long n = I.n[a];
  if (I.real_bytes != 4 || (L != 8 && L != 16) || (NLB != 16 && NLB != 32) || (pk != 1 && pk != 2)) return false;
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  const bool contig = (a == 0);
  if (contig ? (n % 4 != 0 || pk != 1) : (st % 4 != 0)) return false;
  const int m = (int)((n + L - 1) / L);
  const int W = NLB / pk;
  if ((long long)W * m > 512) return false;
  P.L = L;
  P.m = m;
  P.kind = contig ? SWEEP_FIRST : (a == I.dim - 1 ? SWEEP_LAST : SWEEP_MIDDLE);
  P.st = st;
  P.nlines = I.N / n;
  P.pitch = exchange_pitch(m);
  P.pk = pk;
  P.mx = m;
  P.nseg = 1;
  P.cluster = false;
  P.circ = false;
  const int S = I.S, nq = (P.kind == SWEEP_LAST) ? 3 * S : 5 * S;
  StagePlan sp{};
  sp.staged = 2;
  const long long mL = (long long)m * L;
  long long ft;
  if (contig) {
    sp.tile_pitch = (int)(((mL + 31) / 32) * 32 + 4);  // 4 (mod 32): conflict-free 16-byte reads
    ft = (long long)NLB * sp.tile_pitch;
  } else {
    const int padj = (W < 32) ? NLB : 0;
    ft = (long long)m * (L * NLB + padj);
  }
  ft = (ft + 3) & ~3LL;
  sp.tile_elems = (int)ft;
  sp.nin = contig ? S : 3 * S;
  sp.nbuf = 1;
  sp.vec = 1;
  size_t off = align16((size_t)3 * S * ft * 4);
  sp.off_sum = (unsigned)off;
  off = align16(off + (size_t)2 * nq * W * P.pitch * 4 * pk);
  sp.off_sig = (unsigned)off;
  off += (size_t)nq * W * pk * sizeof(double);
  sp.bytes = (unsigned)off;
  if (sp.bytes > 227 * 1024) return false;
  P.nlb = W;
  P.nthreads = W * m;
  P.smem = sp.bytes;
  if (contig) {
    P.nlo_blocks = 1;
    P.nblocks = (int)((P.nlines + NLB - 1) / NLB);
  } else {
    P.nlo_blocks = (int)((st + NLB - 1) / NLB);
    P.nblocks = (int)(P.nlo_blocks * (I.N / (st * n)));
  }
  sp.ntiles = P.nblocks;
  P.sp = sp;
  return true;
}

// Segmented register kernel for long lines: blocks of nlb lines x mx chunks
// (mx a multiple of 8, m > mx), nseg = ceil(m / mx) blocks along every line
// (summary, carry and solve launches, see SegPhase).  cluster: the nseg
// blocks of a line group form one thread-block cluster and the sweep is one
// launch (nseg <= ETD_MAX_CLUSTER; whether the device can hold such a cluster
// is checked by cluster_plan_fits).
bool plan_axis_seg(Instance &I, int a, int L, int nlb, int mx, bool cluster) {
  AxisPlan &P = I.plan[a];
  const long long n = I.n[a];
  const int m = (int)((n + L - 1) / L);
  if ((L != 4 && L != 8 && L != 16) || mx < 8 || mx % 8 != 0 || m <= mx || nlb < 1 || nlb * mx > ETD_MAX_BLOCK_THREADS)
    return false;
  if (cluster && (m + mx - 1) / mx > ETD_MAX_CLUSTER) return false;
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  P.L = L;
  P.m = m;
  P.kind = (a == 0) ? SWEEP_FIRST : (a == I.dim - 1 ? SWEEP_LAST : SWEEP_MIDDLE);
  P.st = st;
  P.nlines = I.N / n;
  P.pk = 1;
  P.sp = StagePlan{};
  P.circ = false;
  P.mx = mx;
  P.nseg = (m + mx - 1) / mx;
  P.pitch = exchange_pitch(mx);
  P.nlb = nlb;
  long long line_blocks;
  if (a == 0) {
    P.nlo_blocks = 1;
    line_blocks = (P.nlines + nlb - 1) / nlb;
  } else {
    P.nlo_blocks = (int)((st + nlb - 1) / nlb);
    line_blocks = (long long)P.nlo_blocks * (I.N / (st * n));
  }
  if (line_blocks * P.nseg > INT_MAX) return false;
  P.nblocks = (int)(line_blocks * P.nseg);
  P.nthreads = nlb * mx;
  P.cluster = cluster;
  P.smem = sweep_smem_bytes(P.kind, I.S, nlb, P.pitch, I.real_bytes, 1, cluster, P.nseg);
  return P.smem <= 200 * 1024;
}

// Circulant kernels (etd_circ.cuh) for a periodic axis.  First axis: p = m L
// with m a power of two, lanes along the line, one block of max(m, 256)
// threads holding 256 / m lines (m <= 512).  Strided axes: 32 lines (lanes)
// times wb chunks (warps) per block, p = cs wb L with cs <= 16 blocks per
// line forming a cluster; the stride a multiple of 32.  Problems with a
// manufactured source are left to the table kernels.
bool plan_axis_circ_strided(Instance &I, int a, int L, int wb, int nc);
bool plan_axis_circ(Instance &I, int a, int L, int wb, int nc) {
  if (a > 0) return plan_axis_circ_strided(I, a, L, wb, nc);
  AxisPlan &P = I.plan[a];
  const long long n = I.n[a];
  if (I.bc[a] != BC_PERIODIC) return false;
  if (I.rkind == ETD_REACTION_ENZYME && I.rp[0] != 0.0) return false;
  if (I.real_bytes == 4 ? (L != 8 && L != 16) : (L != 4 && L != 8)) return false;
  if (n % L != 0) return false;
  const long long m = n / L;
  if (m < 1 || m > 512 || (m & (m - 1)) != 0) return false;
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  P.L = L;
  P.m = (int)m;
  P.kind = SWEEP_FIRST;
  P.st = st;
  P.nlines = I.N / n;
  P.pitch = 1;
  P.pk = 1;
  P.sp = StagePlan{};
  P.mx = P.m;
  P.nseg = 1;
  P.cluster = false;
  P.circ = true;
  P.nthreads = (int)std::max<long long>(m, 256);
  P.nlb = P.nthreads / P.m;
  P.nlo_blocks = 1;
  P.smem = circ_first_smem(I.S, L, P.nthreads, P.m, P.nlb, I.real_bytes);
  if (P.smem > 200 * 1024) return false;
  // persistent: the blocks resident at once, each walking the line groups
  const long long ngroups = (P.nlines + P.nlb - 1) / P.nlb;
  int per_sm = 0, dev = 0, nsm = 0;
  if (circ_first_capacity(I.real_bytes, I.S, L, P.nthreads, I.rkind, P.smem, per_sm) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (per_sm < 1) return false;
  P.nblocks = (int)std::min<long long>(ngroups, (long long)per_sm * nsm);
  return true;
}

bool plan_axis_circ_strided(Instance &I, int a, int L, int wb, int nc) {
  AxisPlan &P = I.plan[a];
  const long long n = I.n[a];
  if (I.bc[a] != BC_PERIODIC || a == 0) return false;
  if (I.rkind == ETD_REACTION_ENZYME && I.rp[0] != 0.0) return false;
  // (chunks, lines) per block with compiled kernels
  const bool ok32 = L == 16 && ((wb == 16 && (nc == 16 || nc == 32)) || (wb == 8 && nc == 32) || (wb == 32 && nc == 16));
  const bool ok64 = L == 8 && ((wb == 8 && nc == 32) || (wb == 16 && nc == 16));
  if (I.real_bytes == 4 ? !ok32 : !ok64) return false;
  long long st = 1;
  for (int b = 0; b < a; ++b) st *= I.n[b];
  if (st % nc != 0 || n % ((long long)wb * L) != 0) return false;
  const long long cs = n / ((long long)wb * L);
  if (cs < 1 || cs > ETD_MAX_CLUSTER) return false;
  P.L = L;
  P.m = (int)(n / L);
  P.kind = (a == I.dim - 1) ? SWEEP_LAST : SWEEP_MIDDLE;
  P.st = st;
  P.nlines = I.N / n;
  P.pitch = 1;
  P.pk = 1;
  P.sp = StagePlan{};
  P.mx = wb;
  P.nseg = (int)cs;
  P.cluster = cs > 1;
  P.circ = true;
  P.nlb = nc;
  P.nthreads = wb * nc;
  P.nlo_blocks = (int)(st / nc);
  const long long ngroups = (long long)P.nlo_blocks * (I.N / (st * n));
  if (ngroups > INT_MAX / 2) return false;
  P.smem = circ_strided_smem(I.S, L, wb, nc, I.real_bytes);
  // lean: the exchange tables stay in global memory when that is what lets a
  // second block share the SM (228 KB per SM, 1 KB reserved per block);
  // ETD_CIRC_LEAN=0 / 1 forbids / forces it
  {
    const size_t lean = circ_strided_smem(I.S, L, wb, nc, I.real_bytes, true);
    const size_t per_sm = 228 * 1024, blk = CIRC_STRIDED_STATIC_SMEM + 1024;
    const char *lv = std::getenv("ETD_CIRC_LEAN");
    P.circ_lean = lv ? (lv[0] == '1') : (2 * (P.smem + blk) > per_sm && 2 * (lean + blk) <= per_sm);
    if (P.circ_lean) P.smem = lean;
  }
  if (P.smem + CIRC_STRIDED_STATIC_SMEM > 227 * 1024) return false;
  // persistent launch: as many clusters (cs > 1) or blocks as the device holds
  // at once, each walking the line groups
  int ncl = 0;
  cudaError_t e;
  if (I.real_bytes == 8) {
    CircArgs<double> C{};
    C.cs = (int)cs;
    C.wb = wb;
    C.ncol = nc;
    C.rkind = I.rkind;
    e = circ_cluster_capacity(C, I.S, L, P.kind, P.nthreads, P.smem, ncl);
  } else {
    CircArgs<float> C{};
    C.cs = (int)cs;
    C.wb = wb;
    C.ncol = nc;
    C.rkind = I.rkind;
    e = circ_cluster_capacity(C, I.S, L, P.kind, P.nthreads, P.smem, ncl);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (cs == 1) {  // the capacity query gave blocks per SM
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    ncl *= nsm;
  }
  if (ncl < 1) return false;
  P.nblocks = (int)(std::min<long long>(ncl, ngroups) * cs);
  return true;
}

// a cluster-segmented plan of axis a can launch on the current device
bool cluster_plan_fits(const Instance &I, int a) {
  const AxisPlan &P = I.plan[a];
  if (!P.cluster) return true;
  int nclusters = 0;
  cudaError_t e;
  if (I.real_bytes == 8) {
    SweepArgs<double> A;
    fill_args<double>(I, a, 0, A);
    A.segphase = SEG_CLUSTER;
    e = sweep_cluster_capacity(A, I.S, P.L, P.kind, P.nthreads, P.smem, nclusters);
  } else {
    SweepArgs<float> A;
    fill_args<float>(I, a, 0, A);
    A.segphase = SEG_CLUSTER;
    e = sweep_cluster_capacity(A, I.S, P.L, P.kind, P.nthreads, P.smem, nclusters);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();  // a refused configuration is not a sticky error
    return false;
  }
  return nclusters > 0;
}

// alignment in bytes the kernels need of the state pointer: tile kernels
// move U with 16-byte copies, circulant sweeps with 16-byte copies and
// 32-byte stores
size_t state_alignment(const Instance &I) {
  size_t al = 1;
  for (int a = 0; a < I.dim; ++a) {
    if (I.plan[a].sp.staged == 2) al = std::max<size_t>(al, 16);
    if (I.plan[a].circ) al = std::max<size_t>(al, 32);
  }
  return al;
}
bool misaligned_state(const Instance &I, const void *U) {
  return (reinterpret_cast<uintptr_t>(U) & (state_alignment(I) - 1)) != 0;
}

int default_chunk(const Instance &I, int a) {
  // staged kernels: 16 positions per thread (FP32) keeps the per-line chain of
  // chunk carries short; the register kernel for long x lines uses 8
  const long long n = I.n[a];
  if (I.real_bytes == 4) return (a == 0 && n > 1024) ? 8 : 16;
  return (a == 0 && n > 1024) ? 4 : 8;
}

// ------------------------------------------------------------ tables

// Places a set of tables in one device block: a sizing pass (no device
// block yet; the returned pointers are placeholders), then a pass with the
// block allocated, whose host image goes up in one copy.
struct StagedArena {
  unsigned char *dev = nullptr;
  std::vector<unsigned char> host;
  size_t used = 0;
  void *put(const void *src, size_t bytes, cudaError_t &) {
    const size_t off = used;
    used += (bytes + 255) & ~(size_t)255;
    if (host.size() < used) host.resize(used);
    memcpy(host.data() + off, src, bytes);
    return dev ? dev + off : nullptr;
  }
};

template <typename R, typename Arena>
static void upload_tab(Arena &arena, const HostTab &T, MatTab<R> &M, std::vector<void *> &owned,
                       cudaError_t &err) {
  std::vector<R> pos(T.pos.begin(), T.pos.end()), sum(T.sum.begin(), T.sum.end()),
      chunk(T.chunk.begin(), T.chunk.end());
  M.pos = (const typename V4T<R>::T *)arena.put(pos.data(), pos.size() * sizeof(R), err);
  M.sum = (const typename V2T<R>::T *)arena.put(sum.data(), sum.size() * sizeof(R), err);
  M.chunk = (const typename V4T<R>::T *)arena.put(chunk.data(), chunk.size() * sizeof(R), err);
  std::vector<R> e1(T.e1.begin(), T.e1.end()), v1(T.v1.begin(), T.v1.end()), w1(T.w1.begin(), T.w1.end()),
      z1(T.z1.begin(), T.z1.end());
  M.e1 = (const R *)arena.put(e1.data(), e1.size() * sizeof(R), err);
  M.v1 = (const R *)arena.put(v1.data(), v1.size() * sizeof(R), err);
  M.w1 = (const R *)arena.put(w1.data(), w1.size() * sizeof(R), err);
  M.z1 = (const R *)arena.put(z1.data(), z1.size() * sizeof(R), err);
  M.rows1 = nullptr;
  M.rows2 = nullptr;
  if constexpr (sizeof(R) == 4) {
    // FP32 coefficient rows, and the same rows with each value in both lanes for line pairs
    const std::vector<float> r1 = fp32_rows(T);
    std::vector<float> r2(2 * r1.size());
    for (size_t q = 0; q < r1.size(); ++q) r2[2 * q] = r2[2 * q + 1] = r1[q];
    M.rows1 = (const float *)arena.put(r1.data(), r1.size() * sizeof(float), err);
    M.rows2 = (const float2 *)arena.put(r2.data(), r2.size() * sizeof(float), err);
  }
  M.segc = nullptr;
  if (!T.segc.empty()) {
    std::vector<R> sc(T.segc.begin(), T.segc.end());
    M.segc = (const typename V4T<R>::T *)arena.put(sc.data(), sc.size() * sizeof(R), err);
  }
  M.r = T.r;
  M.sm_c = T.sm_c;
  M.sm_inv = T.sm_inv;
  (void)owned;
}

// factorise every (axis, species, gamma) line matrix of one instance, forward
// (and transposed for the adjoint), and upload in the instance's precision
etd_status build_axis_tables(etd_ctx *ctx, Instance &I, int a) {
  cudaError_t err = cudaSuccess;
  static const double gammas[3] = {1.0, 3.0, 4.0};
  {
    // every table of the axis in one device block (replaced when the axis is re-planned)
    const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
    std::vector<HostTab> tabs;
    for (int s = 0; s < I.S; ++s)
      for (int g = 0; g < 3; ++g)
        for (int tr = 0; tr < 2; ++tr) {
          const double r = (I.k / gammas[g]) * I.D[s] / (h * h);
          tabs.emplace_back();
          build_tab((int)I.n[a], I.bc[a], r, tr != 0, I.plan[a].L, tabs.back(), I.plan[a].mx, I.plan[a].nseg);
        }
    StagedArena st;
    for (int pass = 0; pass < 2; ++pass) {
      if (pass == 1) {
        if (I.axis_tables[a]) cudaFree(I.axis_tables[a]);
        I.axis_tables[a] = nullptr;
        err = cudaMalloc((void **)&I.axis_tables[a], st.used);
        if (err != cudaSuccess) return cuda_fail(ctx, err, "line table allocation");
        st.dev = (unsigned char *)I.axis_tables[a];
        st.used = 0;
      }
      int q = 0;
      for (int s = 0; s < I.S; ++s)
        for (int g = 0; g < 3; ++g)
          for (int tr = 0; tr < 2; ++tr, ++q) {
            if (I.real_bytes == 8) upload_tab<double>(st, tabs[q], I.tab64[tr][a][s][g], I.owned, err);
            else upload_tab<float>(st, tabs[q], I.tab32[tr][a][s][g], I.owned, err);
          }
    }
    err = cudaMemcpy(I.axis_tables[a], st.host.data(), st.used, cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "uploading line tables");
  }
  AxisPlan &P = I.plan[a];
  if (I.circ_tables[a]) {
    cudaFree(I.circ_tables[a]);
    I.circ_tables[a] = nullptr;
  }
  if (P.circ) {
    // circulant coefficients of every (species, gamma) and their power tables Lambda^i
    const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
    CircHost H[MAX_SPECIES][3];
    size_t per = 0;
    for (int s = 0; s < I.S; ++s)
      for (int g = 0; g < 3; ++g) {
        circ_coeffs((I.k / gammas[g]) * I.D[s] / (h * h), (int)I.n[a], P.L, H[s][g]);
        per = std::max(per, H[s][g].lpow.size() + H[s][g].kch.size());
      }
    const size_t rb = I.real_bytes;
    // lean strided plans: the exchange tables follow the power tables
    const int WBt = P.mx, TSt = 2 * (WBt + 1) + 35;
    const size_t tab_off = (size_t)I.S * 3 * per * rb;
    const size_t tab_n = (P.circ_lean && a > 0) ? (size_t)circ_tab_entries(I.S, WBt) : 0;
    std::vector<unsigned char> img(tab_off + tab_n * rb, 0);
    for (int s = 0; s < I.S; ++s)
      for (int g = 0; g < 3; ++g)
        for (size_t i = 0; i < H[s][g].lpow.size() + H[s][g].kch.size(); ++i) {
          const size_t nl = H[s][g].lpow.size();
          const double x = i < nl ? H[s][g].lpow[i] : H[s][g].kch[i - nl];
          unsigned char *d = img.data() + ((size_t)(s * 3 + g) * per + i) * rb;
          if (rb == 8) memcpy(d, &x, 8);
          else {
            const float v = (float)x;
            memcpy(d, &v, 4);
          }
        }
    for (size_t e = 0; e < tab_n; ++e) {  // the kernel's shared-memory table layout, per matrix
      const int mxi = (int)(e / TSt), o = (int)(e % TSt);
      const CircHost &Hm = H[mxi / 3][mxi % 3];
      double v;
      if (o <= WBt) v = Hm.kch[o];
      else if (o <= 2 * WBt + 1) v = Hm.lpow[o - (WBt + 1)];
      else if (o < 2 * WBt + 2 + 17) {
        const int b = o - (2 * WBt + 2);
        v = b * WBt <= P.m ? Hm.kch[b * WBt] : 0.0;
      } else if (o < 2 * WBt + 2 + 34) {
        const int b = o - (2 * WBt + 2 + 17);
        v = b * WBt <= P.m ? Hm.lpow[b * WBt] : 0.0;
      } else v = Hm.kch[P.m];
      unsigned char *d = img.data() + tab_off + e * rb;
      if (rb == 8) memcpy(d, &v, 8);
      else {
        const float f = (float)v;
        memcpy(d, &f, 4);
      }
    }
    err = cudaMalloc(&I.circ_tables[a], img.size());
    if (err != cudaSuccess) return cuda_fail(ctx, err, "circulant power tables");
    err = cudaMemcpy(I.circ_tables[a], img.data(), img.size(), cudaMemcpyHostToDevice);
    if (err != cudaSuccess) return cuda_fail(ctx, err, "uploading circulant power tables");
    auto fill = [&](auto &C, auto zero) {
      using R = decltype(zero);
      memset(&C, 0, sizeof(C));
      C.N = I.N;
      C.st = P.st;
      C.nlines = P.nlines;
      C.nlo = P.st;
      C.p = (int)I.n[a];
      C.m = P.m;
      C.lpb = P.nlb;
      C.ncol = P.nlb;
      C.nlo_blocks = P.nlo_blocks;
      C.cs = P.circ && a > 0 ? P.nseg : 1;
      C.wb = P.mx;
      C.ngroups = (int)((long long)P.nlo_blocks * (I.N / (P.st * I.n[a])));
      C.lst = P.st * I.n[a];
      C.rkind = I.rkind;
      C.kR = (R)I.k;
      C.half_kR = (R)(0.5 * I.k);
      for (int j = 0; j < 8; ++j) C.rpR[j] = (R)I.rp[j];
      for (int s = 0; s < I.S; ++s) {
        C.cP[s] = (R)(1.0 / H[s][0].alpha);
        C.cT[s] = (R)(9.0 / H[s][1].alpha);
        C.cS[s] = (R)(8.0 / H[s][2].alpha);
        C.iaT[s] = (R)(1.0 / H[s][1].alpha);
        C.iaS[s] = (R)(1.0 / H[s][2].alpha);
        for (int g = 0; g < 3; ++g) {
          circ_to_args<R>(H[s][g], C.mat[s][g]);
          C.lpow[s][g] = (const R *)((unsigned char *)I.circ_tables[a] + (size_t)(s * 3 + g) * per * rb);
          C.kch[s][g] = C.lpow[s][g] + H[s][g].lpow.size();
        }
      }
      C.tabg = tab_n ? (const R *)((unsigned char *)I.circ_tables[a] + tab_off) : nullptr;
    };
    if (rb == 8) fill(I.circ64[a], 0.0);
    else fill(I.circ32[a], 0.0f);
  }
  if (P.nseg > 1 && !P.cluster) {
    // segment summaries and carries (2 values per solve, line and segment) and scalars
    const int nq = (P.kind == SWEEP_LAST) ? 3 * I.S : 5 * I.S;
    const size_t need = ((size_t)4 * nq * P.nlines * P.nseg + (size_t)nq * P.nlines) * I.real_bytes;
    if (P.seg_bytes < need) {
      if (P.seg_buf) {
        cudaFree(P.seg_buf);
        for (auto &o : I.owned)
          if (o == P.seg_buf) o = nullptr;
        P.seg_buf = nullptr;
        P.seg_bytes = 0;
      }
      cudaError_t e = cudaMalloc(&P.seg_buf, need);
      if (e != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "segment scratch of %zu bytes", need);
      I.owned.push_back(P.seg_buf);
      P.seg_bytes = need;
    }
  }
  return ETD_OK;
}

etd_status build_instance_tables(etd_ctx *ctx, Instance &I) {
  cudaError_t err = cudaSuccess;
  for (int a = 0; a < I.dim; ++a) {
    etd_status st = build_axis_tables(ctx, I, a);
    if (st != ETD_OK) return st;
  }
  // manufactured-source coordinate tables
  I.has_source = (I.rkind == ETD_REACTION_ENZYME && I.rp[0] != 0.0);
  I.src_lf = 0.0;
  for (int a = 0; a < 3; ++a) I.phi[a] = nullptr;
  if (I.has_source) {
    for (int a = 0; a < I.dim; ++a) {
      const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
      std::vector<double> ph(I.n[a]);
      for (long long i = 0; i < I.n[a]; ++i) {
        const double x = (I.bc[a] == BC_DIRICHLET) ? (i + 1) * h : i * h;
        ph[i] = std::sin(M_PI * x / I.length[a]);
      }
      I.src_lf += (M_PI / I.length[a]) * (M_PI / I.length[a]);
      if (I.real_bytes == 8) {
        I.phi[a] = I.arena.put(ph.data(), ph.size() * 8, err);
      } else {
        std::vector<float> pf(ph.begin(), ph.end());
        I.phi[a] = I.arena.put(pf.data(), pf.size() * 4, err);
      }
      if (err != cudaSuccess) return cuda_fail(ctx, err, "uploading source tables");
    }
  }
  return ETD_OK;
}

// ------------------------------------------------------------ sweep args

template <typename R>
void fill_args(const Instance &I, int a, int transpose, SweepArgs<R> &A) {
  const AxisPlan &P = I.plan[a];
  memset(&A, 0, sizeof(A));
  A.N = I.N;
  A.st = P.st;
  A.nlines = P.nlines;
  A.n = (int)I.n[a];
  A.nlo_blocks = P.nlo_blocks;
  A.m = P.m;
  A.nlb = P.nlb;
  A.pitch = P.pitch;
  A.nblocks = P.nblocks;
  for (int s = 0; s < I.S; ++s)
    for (int g = 0; g < 3; ++g) {
      if constexpr (sizeof(R) == 8) A.mat[s][g] = I.tab64[transpose][a][s][g];
      else A.mat[s][g] = I.tab32[transpose][a][s][g];
    }
  A.k = I.k;
  A.kR = (R)I.k;
  A.rkind = I.rkind;
  for (int j = 0; j < 8; ++j) {
    A.rp[j] = I.rp[j];
    A.rpR[j] = (R)I.rp[j];
  }
  for (int b = 0; b < 3; ++b) A.phi[b] = (const R *)I.phi[b];
  A.nx = (int)I.n[0];
  A.ny = (int)I.n[1];
  A.src_lf = I.src_lf;
  A.src_lfR = (R)I.src_lf;
  A.axis = a;
  A.pk = P.pk;
  A.sp = P.sp;
  A.mx = P.mx;
  A.nseg = P.nseg;
  A.segphase = SEG_WHOLE;
  if (P.nseg > 1 && P.seg_buf) {
    const int nq = (P.kind == SWEEP_LAST) ? 3 * I.S : 5 * I.S;
    const size_t pairs = (size_t)2 * nq * P.nlines * P.nseg;
    A.seg_sum = (R *)P.seg_buf;
    A.seg_car = A.seg_sum + pairs;
    A.seg_sig = A.seg_car + pairs;
  }
}

// One sweep of axis a: a single launch, or for a segmented plan the summary,
// carry and solve launches (LAST: P summaries, P carries, P solve + T/S
// summaries, T/S carries, final solve).
template <typename R>
cudaError_t run_sweep(const Instance &I, int a, SweepArgs<R> &A, cudaStream_t s) {
  const AxisPlan &P = I.plan[a];
  if (P.circ) {
    CircArgs<R> C;
    if constexpr (sizeof(R) == 8) C = I.circ64[a];
    else C = I.circ32[a];
    for (int f = 0; f < 3; ++f) {
      C.in[f] = A.in[f];
      C.out[f] = A.out[f];
    }
    // strided sweeps with 32 lines per block stage their tiles by TMA
    if (a > 0 && P.nlb == 32 && !circ_encode_maps(C, I.S, P.mx * P.L)) return cudaErrorNotSupported;
    return launch_circ(C, I.S, P.L, P.kind, P.nthreads, P.smem, P.nblocks, s);
  }
  if (P.nseg <= 1) return launch_sweep(A, I.S, P.L, P.kind, P.nthreads, P.smem, s);
  if (P.cluster) {
    A.segphase = SEG_CLUSTER;
    return launch_sweep(A, I.S, P.L, P.kind, P.nthreads, P.smem, s);
  }
  const int S = I.S;
  auto sweep = [&](int phase) {
    A.segphase = phase;
    return launch_sweep(A, S, P.L, P.kind, P.nthreads, P.smem, s);
  };
  cudaError_t e = sweep(SEG_SUMMARY);
  if (e != cudaSuccess) return e;
  if (P.kind != SWEEP_LAST) {
    e = launch_seg_carry(A, S, P.kind, 0, 5 * S, s);
    if (e != cudaSuccess) return e;
    return sweep(SEG_SOLVE);
  }
  e = launch_seg_carry(A, S, P.kind, 0, S, s);
  if (e != cudaSuccess) return e;
  e = sweep(SEG_SOLVE);
  if (e != cudaSuccess) return e;
  e = launch_seg_carry(A, S, P.kind, S, 2 * S, s);
  if (e != cudaSuccess) return e;
  return sweep(SEG_FINAL);
}
template cudaError_t run_sweep<float>(const Instance &, int, SweepArgs<float> &, cudaStream_t);
template cudaError_t run_sweep<double>(const Instance &, int, SweepArgs<double> &, cudaStream_t);
template void fill_args<float>(const Instance &, int, int, SweepArgs<float> &);
template void fill_args<double>(const Instance &, int, int, SweepArgs<double> &);

// forward step of one instance on stream s: U holds U_n at t_n, gets U_{n+1}
cudaError_t prof_begin(etd_ctx *ctx, cudaStream_t s, cudaEvent_t &ev) {
  ev = nullptr;
  if (!ctx || !ctx->profiling) return cudaSuccess;
  if (ctx->prof_pool.empty()) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return e;
  } else {
    ev = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
  }
  return cudaEventRecord(ev, s);
}

cudaError_t prof_end(etd_ctx *ctx, cudaStream_t s, int kind, cudaEvent_t ev0) {
  if (!ctx || !ctx->profiling || !ev0) return cudaSuccess;
  cudaEvent_t ev1;
  cudaError_t e = prof_begin(ctx, s, ev1);
  if (e != cudaSuccess) return e;
  ctx->prof_events.push_back({kind, {ev0, ev1}});
  return cudaSuccess;
}

template <typename R>
static cudaError_t step_instance(const Instance &I, R *U, double t, cudaStream_t s, etd_ctx *prof) {
  if (misaligned_state(I, U)) return cudaErrorMisalignedAddress;
  R *cu = (R *)I.scratch[0], *cf = (R *)I.scratch[1], *w = (R *)I.scratch[2];
  for (int a = 0; a < I.dim; ++a) {
    const AxisPlan &P = I.plan[a];
    SweepArgs<R> A;
    fill_args<R>(I, a, 0, A);
    if (P.kind == SWEEP_FIRST) {
      A.in[0] = U;
      A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
      A.t_eval = t;
    } else if (P.kind == SWEEP_MIDDLE) {
      A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
      A.out[0] = cu; A.out[1] = cf; A.out[2] = w;
      A.t_eval = t;
    } else {
      A.in[0] = cu; A.in[1] = cf; A.in[2] = w;
      A.out[0] = U;
      A.t_eval = t + I.k;
    }
    A.exp_mt = std::exp(-A.t_eval);
    A.exp_mtR = (R)A.exp_mt;
    cudaEvent_t ev0;
    cudaError_t e = prof_begin(prof, s, ev0);
    if (e != cudaSuccess) return e;
    e = run_sweep<R>(I, a, A, s);
    if (e != cudaSuccess) return e;
    e = prof_end(prof, s, P.kind, ev0);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t cplx_step(const Instance &I, void *U, double t, cudaStream_t s, etd_ctx *prof);

cudaError_t forward_step(const Instance &I, void *U, double t, cudaStream_t s, etd_ctx *prof) {
  if (I.coupled) return cplx_step(I, U, t, s, prof);
  if (I.real_bytes == 8) return step_instance<double>(I, (double *)U, t, s, prof);
  return step_instance<float>(I, (float *)U, t, s, prof);
}

// ------------------------------------------------------------ instances

// ETD_CIRCULANT=0 keeps periodic axes on the table kernels unless ETD_TILES
// asks otherwise (to compare the two families)
static bool forced_only_tables() {
  const char *v = std::getenv("ETD_CIRCULANT");
  return v && v[0] == '0';
}

etd_status init_instance(etd_ctx *ctx, Instance &I, const etd_grid *grid, const double *D, const etd_reaction *rx,
                         double k, int32_t precision, bool with_scratch) {
  I.dim = grid->dim;
  I.N = 1;
  for (int a = 0; a < 3; ++a) {
    I.n[a] = a < I.dim ? grid->n[a] : 1;
    I.bc[a] = a < I.dim ? grid->bc[a] : 0;
    I.length[a] = a < I.dim ? grid->length[a] : 1.0;
    I.N *= I.n[a];
  }
  I.S = rx->nspecies;
  for (int s = 0; s < I.S; ++s) I.D[s] = D[s];
  I.k = k;
  I.rkind = rx->kind;
  for (int j = 0; j < 8; ++j) I.rp[j] = rx->params[j];
  I.real_bytes = precision == ETD_FP64 ? 8 : 4;
  // ETD_TILES="L:nlb:kernel[:pack],..." (one entry per axis; kernel 0
  // register, 1 staged, 2 tile with nlb lines per block, 3 segmented register
  // kernel with the fourth field = chunks per segment, 4 the same as one
  // cluster launch, 5 circulant kernel of a periodic axis with nlb = chunks
  // and the fourth field = lines per block on strided axes) forces tile shapes, e.g. to reproduce an autotuned
  // configuration in a profiler run
  const char *forced = std::getenv("ETD_TILES");
  for (int a = 0; a < I.dim; ++a) {
    int L = default_chunk(I, a);
    int fl = 0, fn = 0, fs = 0, fp = 1;
    if (forced) {
      const char *p = forced;
      for (int b = 0; b < a && p; ++b) {
        p = strchr(p, ',');
        if (p) ++p;
      }
      if (p && sscanf(p, "%d:%d:%d:%d", &fl, &fn, &fs, &fp) >= 3 && (fl == 4 || fl == 8 || fl == 16)) {
        const bool ok = fs == 5   ? plan_axis_circ(I, a, fl, fn > 0 ? fn : 16, fp > 1 ? fp : 32)
                        : fs == 4 ? plan_axis_seg(I, a, fl, fn, fp, true) && cluster_plan_fits(I, a)
                        : fs == 3 ? plan_axis_seg(I, a, fl, fn, fp, false)
                        : fs == 2 ? plan_axis_tile(I, a, fl, fn, fp)
                                  : plan_axis_ex(I, a, fl, ETD_MAX_BLOCK_THREADS, fn, !fs, fp == 2 && !fs ? 2 : 1);
        if (ok) continue;
      }
    }
    // periodic axes: the circulant kernels where a shape fits (fastest measured);
    // otherwise, and for other boundaries, the table kernels
    if (with_scratch && I.bc[a] == BC_PERIODIC && !forced_only_tables()) {  // (ensembles plan their own)
      const int Lc = I.real_bytes == 4 ? 16 : 8;
      bool ok = false;
      if (a == 0) ok = plan_axis_circ(I, a, Lc, 16, 32);
      else if (I.real_bytes == 4)
        ok = plan_axis_circ(I, a, Lc, 16, 32) || plan_axis_circ(I, a, Lc, 8, 32) || plan_axis_circ(I, a, Lc, 16, 16);
      else
        ok = plan_axis_circ(I, a, Lc, 8, 32) || plan_axis_circ(I, a, Lc, 16, 16);
      if (ok) continue;
    }
    // small problems (a few blocks per sweep) take the register kernel: the
    // staged kernel's prefetch pipeline only pays with many tiles per block
    // (64^2 two-species FP64: 35 against 62 us per step),
    // with few lines per block, so that the sweep spreads over the SMs
    const bool small = (long long)I.N * I.S <= (1LL << 17);
    int nlb_small = 0;
    if (small) {
      long long st = 1;
      for (int b = 0; b < a; ++b) st *= I.n[b];
      const long long avail = a == 0 ? I.N / I.n[0] : st;
      nlb_small = 1;
      while ((long long)nlb_small * 2 * 152 <= avail) nlb_small *= 2;
    }
    // short chunks on short lines (64^2 FP64: 35 us per step at L = 4, 53 at 8)
    if (small && I.n[a] >= 32 && I.n[a] <= 256) L = I.real_bytes == 4 ? 8 : 4;
    while (!plan_axis_ex(I, a, L, ETD_MAX_BLOCK_THREADS, nlb_small, small, 1) && L < 16) L *= 2;
    if (!plan_axis_ex(I, a, L, ETD_MAX_BLOCK_THREADS, nlb_small, small, 1) && !plan_axis(I, a, L, ETD_MAX_BLOCK_THREADS)) {
      // lines longer than one block: segments of 32 chunks spread over several
      // blocks, launched as one thread-block cluster where a line group's
      // segments fit one, else the multi-launch segmented sweep
      const int Ls = I.real_bytes == 4 ? 16 : 8;
      const bool seg = (plan_axis_seg(I, a, Ls, 8, 32, true) && cluster_plan_fits(I, a)) ||
                       plan_axis_seg(I, a, Ls, 8, 32, false);
      if (!seg)
        return fail(ctx, ETD_ERR_UNSUPPORTED, "axis %d with n = %lld fits neither one block nor a segmented plan", a,
                    (long long)I.n[a]);
    }
  }
  etd_status st = build_instance_tables(ctx, I);
  if (st != ETD_OK) return st;
  if (with_scratch) {
    const size_t bytes = (size_t)I.S * I.N * I.real_bytes;
    for (int f = 0; f < 3; ++f) {
      cudaError_t e = cudaMalloc(&I.scratch[f], bytes);
      if (e != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "scratch allocation of %zu bytes failed", bytes);
      I.owned.push_back(I.scratch[f]);
    }
  }
  return ETD_OK;
}

}  // namespace etd

// ================================================================= C ABI

extern "C" {

etd_status etd_create(const etd_grid *grid, const double *D, const etd_reaction *reaction, double k,
                      int32_t precision, void *stream, etd_ctx **out) {
  if (!out) return fail(nullptr, ETD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  etd_status st = validate_problem(grid, D, reaction, k, precision);
  if (st != ETD_OK) return st;
  etd_ctx *ctx = new (std::nothrow) etd_ctx();
  if (!ctx) return fail(nullptr, ETD_ERR_OOM, "host allocation failed");
  ctx->stream = (cudaStream_t)stream;
  ctx->precision = precision;
  ctx->batched = false;
  ctx->inst.resize(1);
  st = init_instance(ctx, ctx->inst[0], grid, D, reaction, k, precision, true);
  if (st != ETD_OK) {
    g_create_error = ctx->err;
    etd_destroy(ctx);
    return st;
  }
  *out = ctx;
  return ETD_OK;
}

etd_status etd_set_stream(etd_ctx *ctx, void *stream) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  ctx->stream = (cudaStream_t)stream;
  drop_graphs(ctx);
  return ETD_OK;
}

etd_status etd_step(etd_ctx *ctx, void *U, double t_n) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_step on a batched context");
  if (!U) return fail(ctx, ETD_ERR_INVALID_ARG, "U is NULL");
  if (misaligned_state(ctx->inst[0], U))
    return fail(ctx, ETD_ERR_INVALID_ARG, "U must be %zu-byte aligned for the planned kernels (tile kernels copy "
                "16 bytes, circulant sweeps store 32 bytes at a time)", state_alignment(ctx->inst[0]));
  if (!std::isfinite(t_n)) return fail(ctx, ETD_ERR_INVALID_ARG, "t_n not finite");
  cudaError_t e = forward_step(ctx->inst[0], U, t_n, ctx->stream, ctx);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "etd_step launch");
  return ETD_OK;
}

etd_status etd_run(etd_ctx *ctx, void *U, double t0, int64_t nsteps) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_run on a batched context");
  if (!U) return fail(ctx, ETD_ERR_INVALID_ARG, "U is NULL");
  if (nsteps < 0) return fail(ctx, ETD_ERR_INVALID_ARG, "nsteps < 0");
  if (!std::isfinite(t0)) return fail(ctx, ETD_ERR_INVALID_ARG, "t0 not finite");
  if (misaligned_state(ctx->inst[0], U))
    return fail(ctx, ETD_ERR_INVALID_ARG, "U must be %zu-byte aligned for the planned kernels (tile kernels copy "
                "16 bytes, circulant sweeps store 32 bytes at a time)", state_alignment(ctx->inst[0]));
  const Instance &I = ctx->inst[0];
  return run_steps(ctx, [&](cudaStream_t s, int64_t n) -> cudaError_t {
    return forward_step(I, U, t0 + (double)n * I.k, s, ctx);
  }, GraphKey{U, nullptr, t0, nsteps}, nsteps);
}

etd_status etd_run_host(etd_ctx *ctx, void *U_host, double t0, int64_t nsteps) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_run_host on a batched context");
  if (!U_host) return fail(ctx, ETD_ERR_INVALID_ARG, "U_host is NULL");
  if (nsteps < 0) return fail(ctx, ETD_ERR_INVALID_ARG, "nsteps < 0");
  if (!std::isfinite(t0)) return fail(ctx, ETD_ERR_INVALID_ARG, "t0 not finite");
  const Instance &I = ctx->inst[0];
  const size_t bytes = (size_t)I.S * I.N * I.real_bytes;
  if (!ctx->host_state) {
    cudaError_t e = cudaMalloc(&ctx->host_state, bytes);
    if (e != cudaSuccess) return fail(ctx, ETD_ERR_OOM, "device state allocation of %zu bytes failed", bytes);
  }
  cudaError_t e = cudaMemcpyAsync(ctx->host_state, U_host, bytes, cudaMemcpyHostToDevice, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "host to device copy");
  etd_status st = etd_run(ctx, ctx->host_state, t0, nsteps);
  if (st != ETD_OK) return st;
  e = cudaMemcpyAsync(U_host, ctx->host_state, bytes, cudaMemcpyDeviceToHost, ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "device to host copy");
  e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  if (circ_take_status())
    return fail(ctx, ETD_ERR_TIMEOUT, "a sweep kernel's bounded wait for its tile copies gave up");
  return ETD_OK;
}

etd_status etd_profile(etd_ctx *ctx, int32_t enable) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  ctx->profiling = enable != 0;
  return ETD_OK;
}

etd_status etd_profile_read(etd_ctx *ctx, double *ms, int64_t *launches) {
  if (!ctx || !ms || !launches) return fail(ctx, ETD_ERR_INVALID_ARG, "null argument");
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
  if (circ_take_status())
    return fail(ctx, ETD_ERR_TIMEOUT, "a sweep kernel's bounded wait for its tile copies gave up");
  for (auto &rec : ctx->prof_events) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, rec.second.first, rec.second.second);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed time");
    const int kd = rec.first < 0 ? 0 : (rec.first > 2 ? 2 : rec.first);
    ms[kd] += t;
    launches[kd] += 1;
    ctx->prof_pool.push_back(rec.second.first);
    ctx->prof_pool.push_back(rec.second.second);
  }
  ctx->prof_events.clear();
  return ETD_OK;
}

etd_status etd_get_info(const etd_ctx *ctx, etd_info *info) {
  if (!ctx || !info) return fail(nullptr, ETD_ERR_INVALID_ARG, "null ctx or info");
  memset(info, 0, sizeof(*info));
  const Instance &I = ctx->inst[0];
  info->dim = I.dim;
  info->nspecies = I.S;
  info->precision = ctx->precision;
  long long N = 0, scratch = 0;
  int launches = 0;
  for (const Instance &J : ctx->inst) {
    N += J.N;
    scratch += 3LL * J.S * J.N * J.real_bytes;
  }
  // one launch per sweep; a segmented sweep takes 3 (LAST: 5) unless it is
  // one cluster launch
  launches = 0;
  for (int a = 0; a < I.dim; ++a)
    launches += ctx->batched || I.plan[a].nseg <= 1 || I.plan[a].cluster ? 1 : (I.plan[a].kind == SWEEP_LAST ? 5 : 3);
  if (ctx->batched && ctx->ens_on) launches = 1;  // one persistent launch covers every sweep
  for (const Instance &J : ctx->inst)
    for (int a = 0; a < J.dim; ++a)
      if (J.plan[a].nseg > 1 && J.plan[a].seg_buf) scratch += (long long)J.plan[a].seg_bytes;
  info->npoints = N;
  info->state_bytes = (int64_t)I.S * N * I.real_bytes;
  info->scratch_bytes = scratch;
  // fused schedule: first sweep 1 in + 3 out, middle sweeps 3 + 3, last sweep 3 + 1
  info->algorithmic_bytes = (int64_t)(6 * I.dim - 4) * I.S * N * I.real_bytes;
  info->launches_per_step = launches;
  for (int a = 0; a < I.dim; ++a) {
    info->chunk[a] = I.plan[a].L;
    info->lines_per_block[a] = I.plan[a].nlb;
    info->staged[a] = I.plan[a].circ ? 5 : I.plan[a].nseg > 1 ? (I.plan[a].cluster ? 4 : 3) : I.plan[a].sp.staged;
    info->pack[a] = I.plan[a].nseg > 1 ? I.plan[a].mx : I.plan[a].pk;
    info->grid_blocks[a] = ctx->batched ? (ctx->ens_on ? ctx->ens_grid : ctx->batch_total_blocks[a])
                                        : I.plan[a].nblocks;
    if (I.coupled) {  // complex line kernel: one launch per axis
      info->chunk[a] = I.cax[a].chunk;
      info->lines_per_block[a] = I.cax[a].nl;
      info->staged[a] = 6;
      info->pack[a] = 1;
      info->grid_blocks[a] = I.cax[a].nblocks;
    }
  }
  return ETD_OK;
}

void etd_destroy(etd_ctx *ctx) {
  if (!ctx) return;
  drop_graphs(ctx);
  for (Instance &I : ctx->inst) {
    for (void *p : I.owned) cudaFree(p);
    I.owned.clear();
    I.arena.release();
    for (void *&p : I.axis_tables) {
      if (p) cudaFree(p);
      p = nullptr;
    }
    for (void *&p : I.circ_tables) {
      if (p) cudaFree(p);
      p = nullptr;
    }
  }
  if (ctx->host_state) cudaFree(ctx->host_state);
  if (ctx->batch_scratch) cudaFree(ctx->batch_scratch);
  for (int a = 0; a < 3; ++a) {
    if (ctx->batch_args[a]) cudaFree(ctx->batch_args[a]);
    if (ctx->batch_block_start[a]) cudaFree(ctx->batch_block_start[a]);
  }
  if (ctx->ens_items) cudaFree(ctx->ens_items);
  if (ctx->ens_queue) cudaFree(ctx->ens_queue);
  if (ctx->ens_done) cudaFree(ctx->ens_done);
  if (ctx->ens_status) cudaFree(ctx->ens_status);
  if (ctx->adj_ws) cudaFree(ctx->adj_ws);
  for (void *p : ctx->adj_ubar)
    if (p) cudaFree(p);
  if (ctx->adj_acc) cudaFree(ctx->adj_acc);
  if (ctx->adj_part) cudaFree(ctx->adj_part);
  if (ctx->ckpt) cudaFree(ctx->ckpt);
  if (ctx->seg) cudaFree(ctx->seg);
  if (ctx->seg_mid) cudaFree(ctx->seg_mid);
  for (auto &rec : ctx->prof_events) {
    cudaEventDestroy(rec.second.first);
    cudaEventDestroy(rec.second.second);
  }
  for (cudaEvent_t ev : ctx->prof_pool) cudaEventDestroy(ev);
  for (void *p : ctx->owned) cudaFree(p);
  delete ctx;
}

}  // extern "C"
