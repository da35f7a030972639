// etd_noalloc.cu -- etd_step_noalloc: one ETD-RDP-IF step that allocates no
// device memory.
//
// Some callers cannot call cudaMalloc: plugins hosted by an application that
// owns every device allocation through its own pool, or real-time loops that
// may not touch the allocator after start-up.  For them this entry point keeps
// its scratch (the three carried fields c_U, c_f, w of the step and the line
// tables) in one file-scope __device__ array of ETD_NOALLOC_BYTES.  Every GPU
// that loads the library holds that array until the process exits.  The
// caller passes the state in and gets it back; nothing is cudaMalloc'ed or
// freed here.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/etdrdpif.h"
#include "etd_context.h"
#include "etd_internal.h"
#include "etd_tables.h"

namespace etd {
etd_status validate_problem(const etd_grid *grid, const double *D, const etd_reaction *rx, double k,
                            int32_t precision);
bool plan_axis(Instance &I, int a, int L, int max_threads);
int default_chunk(const Instance &I, int a);
}  // namespace etd

using namespace etd;

// 64 MiB, 256-byte aligned; shared by every call on a device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[ETD_NOALLOC_BYTES];

namespace {

// The array's device address, looked up on every call with the caller's
// device and context current.  The host-side name g_noalloc_scratch is only
// a stand-in for the symbol: handing it to a kernel would fault (or, where
// the GPU can reach host memory, silently use the wrong memory).  The address
// is not cached: it belongs to the CUDA context that is current, and a host
// application may make another context current between calls, or
// cudaDeviceReset may recreate the primary context; the lookup is a cheap
// host-side query.
etd_status scratch_address(void **out) {
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress(g_noalloc_scratch)");
  *out = p;
  return ETD_OK;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// bump allocator over the static array (host-side bookkeeping only)
struct Carve {
  unsigned char *base;
  size_t used = 0;
  void *take(size_t bytes) {
    void *p = base + used;
    used += align256(bytes);
    return p;
  }
};

template <typename R>
void stage_tab(const HostTab &T, MatTab<R> &M, Carve &cv, std::vector<std::pair<void *, std::vector<R>>> &up) {
  up.push_back({cv.take(T.pos.size() * sizeof(R)), std::vector<R>(T.pos.begin(), T.pos.end())});
  M.pos = (const typename V4T<R>::T *)up.back().first;
  up.push_back({cv.take(T.sum.size() * sizeof(R)), std::vector<R>(T.sum.begin(), T.sum.end())});
  M.sum = (const typename V2T<R>::T *)up.back().first;
  up.push_back({cv.take(T.chunk.size() * sizeof(R)), std::vector<R>(T.chunk.begin(), T.chunk.end())});
  M.chunk = (const typename V4T<R>::T *)up.back().first;
  up.push_back({cv.take(T.e1.size() * sizeof(R)), std::vector<R>(T.e1.begin(), T.e1.end())});
  M.e1 = (const R *)up.back().first;
  up.push_back({cv.take(T.v1.size() * sizeof(R)), std::vector<R>(T.v1.begin(), T.v1.end())});
  M.v1 = (const R *)up.back().first;
  up.push_back({cv.take(T.w1.size() * sizeof(R)), std::vector<R>(T.w1.begin(), T.w1.end())});
  M.w1 = (const R *)up.back().first;
  up.push_back({cv.take(T.z1.size() * sizeof(R)), std::vector<R>(T.z1.begin(), T.z1.end())});
  M.z1 = (const R *)up.back().first;
  M.rows1 = nullptr;
  M.rows2 = nullptr;  // the no-allocation step plans one line per thread
  M.segc = nullptr;   // and whole lines per block
  if constexpr (sizeof(R) == 4) {
    const std::vector<float> r1 = fp32_rows(T);
    up.push_back({cv.take(r1.size() * sizeof(R)), std::vector<R>(r1.begin(), r1.end())});
    M.rows1 = (const float *)up.back().first;
  }
  M.r = T.r;
  M.sm_c = T.sm_c;
  M.sm_inv = T.sm_inv;
}

template <typename R>
etd_status noalloc_step(Instance &I, void *U, double t_n, cudaStream_t s, unsigned char *base) {
  Carve cv{base};
  const size_t field = (size_t)I.S * I.N * sizeof(R);
  for (int f = 0; f < 3; ++f) I.scratch[f] = cv.take(field);
  std::vector<std::pair<void *, std::vector<R>>> up;
  static const double gammas[3] = {1.0, 3.0, 4.0};
  for (int a = 0; a < I.dim; ++a) {
    const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
    for (int sp = 0; sp < I.S; ++sp)
      for (int g = 0; g < 3; ++g) {
        HostTab T;
        build_tab((int)I.n[a], I.bc[a], (I.k / gammas[g]) * I.D[sp] / (h * h), false, I.plan[a].L, T);
        if constexpr (sizeof(R) == 8) stage_tab<double>(T, I.tab64[0][a][sp][g], cv, up);
        else stage_tab<float>(T, I.tab32[0][a][sp][g], cv, up);
      }
  }
  I.has_source = (I.rkind == ETD_REACTION_ENZYME && I.rp[0] != 0.0);
  I.src_lf = 0.0;
  if (I.has_source)
    for (int a = 0; a < I.dim; ++a) {
      const double h = grid_h(I.bc[a], I.n[a], I.length[a]);
      std::vector<R> ph(I.n[a]);
      for (long long i = 0; i < I.n[a]; ++i)
        ph[i] = (R)std::sin(M_PI * ((I.bc[a] == BC_DIRICHLET) ? (i + 1) * h : i * h) / I.length[a]);
      I.src_lf += (M_PI / I.length[a]) * (M_PI / I.length[a]);
      up.push_back({cv.take(ph.size() * sizeof(R)), ph});
      I.phi[a] = up.back().first;
    }
  if (cv.used > (size_t)ETD_NOALLOC_BYTES)
    return fail(nullptr, ETD_ERR_INVALID_ARG,
                "etd_step_noalloc: problem needs %zu bytes of scratch, the static array holds %zu "
                "(3 s N element fields plus line tables)", cv.used, (size_t)ETD_NOALLOC_BYTES);
  // tables change with the problem: copy this call's tables into the array,
  // ordered on the caller's stream before the sweeps that read them
  for (auto &u : up) {
    cudaError_t e = cudaMemcpyAsync(u.first, u.second.data(), u.second.size() * sizeof(R), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "etd_step_noalloc table copy");
  }
  // the host vectors must outlive the copies (pageable source)
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "etd_step_noalloc stream synchronize");
  e = forward_step(I, U, t_n, s, nullptr);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "etd_step_noalloc launch");
  return ETD_OK;
}

}  // namespace

extern "C" etd_status etd_step_noalloc(const etd_grid *grid, const double *D, const etd_reaction *reaction,
                                       double k, int32_t precision, void *U, double t_n, void *stream) {
  etd_status st = validate_problem(grid, D, reaction, k, precision);
  if (st != ETD_OK) return st;
  if (!U) return fail(nullptr, ETD_ERR_INVALID_ARG, "etd_step_noalloc: U is NULL");
  if (!std::isfinite(t_n)) return fail(nullptr, ETD_ERR_INVALID_ARG, "etd_step_noalloc: t_n not finite");
  Instance I;
  I.dim = grid->dim;
  I.N = 1;
  for (int a = 0; a < 3; ++a) {
    I.n[a] = a < I.dim ? grid->n[a] : 1;
    I.bc[a] = a < I.dim ? grid->bc[a] : 0;
    I.length[a] = a < I.dim ? grid->length[a] : 1.0;
    I.N *= I.n[a];
  }
  I.S = reaction->nspecies;
  for (int sp = 0; sp < I.S; ++sp) I.D[sp] = D[sp];
  I.k = k;
  I.rkind = reaction->kind;
  for (int j = 0; j < 8; ++j) I.rp[j] = reaction->params[j];
  I.real_bytes = precision == ETD_FP64 ? 8 : 4;
  // reject before touching the device: the three carried fields alone
  const size_t fields = (size_t)3 * I.S * I.N * I.real_bytes;
  if (fields > (size_t)ETD_NOALLOC_BYTES)
    return fail(nullptr, ETD_ERR_INVALID_ARG,
                "etd_step_noalloc: 3 s N elements need %zu bytes, more than the %zu-byte static scratch; "
                "use etd_create/etd_step for this size", fields, (size_t)ETD_NOALLOC_BYTES);
  for (int a = 0; a < I.dim; ++a) {
    int L = default_chunk(I, a);
    while (!plan_axis(I, a, L, ETD_MAX_BLOCK_THREADS) && L < 16) L *= 2;
    if (!plan_axis(I, a, L, ETD_MAX_BLOCK_THREADS))
      return fail(nullptr, ETD_ERR_UNSUPPORTED, "axis %d with n = %lld does not fit one block", a, (long long)I.n[a]);
  }
  void *base = nullptr;
  st = scratch_address(&base);
  if (st != ETD_OK) return st;
  if (I.real_bytes == 8) return noalloc_step<double>(I, U, t_n, (cudaStream_t)stream, (unsigned char *)base);
  return noalloc_step<float>(I, U, t_n, (cudaStream_t)stream, (unsigned char *)base);
}
