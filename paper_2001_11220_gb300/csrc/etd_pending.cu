// etd_pending.cu -- entry points whose kernels are not implemented yet; they
// validate nothing and report ETD_ERR_UNSUPPORTED.
#include "../../include/etdrdpif.h"
#include "etd_context.h"

using namespace etd;

extern "C" {


etd_status etd_batch_create(int32_t, const etd_grid *, const double *, const etd_reaction *, double, int32_t, void *,
                            etd_ctx **out) {
  if (out) *out = nullptr;
  return fail(nullptr, ETD_ERR_UNSUPPORTED, "etd_batch_create not implemented");
}

etd_status etd_batch_run(etd_ctx *ctx, void *const *, double, int64_t) {
  return fail(ctx, ETD_ERR_UNSUPPORTED, "etd_batch_run not implemented");
}


}  // extern "C"
