// etd_finite.cu -- non-finite detection on a state (etd_check_finite).
//
// A grid-stride scan over the s N elements of U; every thread that meets a
// NaN or an infinity lowers a device word to the element's index with
// atomicMin, so the reported index is the smallest one whatever the schedule.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "../../include/etdrdpif.h"
#include "etd_context.h"

namespace {

template <typename R>
__global__ void first_nonfinite_kernel(const R *__restrict__ U, long long n, unsigned long long *first) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(U[i])) atomicMin(first, (unsigned long long)i);
}

}  // namespace

using namespace etd;

extern "C" etd_status etd_check_finite(etd_ctx *ctx, const void *U, int64_t *first_bad) {
  if (!ctx) return fail(nullptr, ETD_ERR_INVALID_ARG, "ctx is NULL");
  if (ctx->batched) return fail(ctx, ETD_ERR_INVALID_ARG, "etd_check_finite takes one problem's state");
  if (!U) return fail(ctx, ETD_ERR_INVALID_ARG, "U is NULL");
  if (first_bad) *first_bad = -1;
  const Instance &I = ctx->inst[0];
  if (!ctx->finite_word) {
    cudaError_t e = cudaMalloc(&ctx->finite_word, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "non-finite scan word");
    ctx->owned.push_back(ctx->finite_word);
  }
  unsigned long long *word = (unsigned long long *)ctx->finite_word;
  const unsigned long long none = ULLONG_MAX;
  const long long n = (long long)I.S * I.N;
  cudaStream_t s = ctx->stream;
  cudaError_t e = cudaMemcpyAsync(word, &none, sizeof(none), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "non-finite scan reset");
  const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 8);
  if (I.real_bytes == 8) first_nonfinite_kernel<double><<<blocks, 256, 0, s>>>((const double *)U, n, word);
  else first_nonfinite_kernel<float><<<blocks, 256, 0, s>>>((const float *)U, n, word);
  e = cudaGetLastError();
  unsigned long long got = none;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&got, word, sizeof(got), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "non-finite scan");
  if (got == none) return ETD_OK;
  if (first_bad) *first_bad = (int64_t)got;
  return fail(ctx, ETD_ERR_NONFINITE, "non-finite value at element %lld (species %lld, point %lld)", (long long)got,
              (long long)(got / I.N), (long long)(got % I.N));
}
