// weighted.cu -- weighted pair counts and the adjoint (gradient of a
// weighted-count functional with respect to the per-object weights).
#include "cute_internal.h"

namespace cute {
cute_status weighted_driver(cute_ctx *ctx, int n, const cute_pair_desc *d, uint64_t *const *counts,
                            double *const *wsum, uint64_t *oor) {
  ctx->err = "weighted counts are not built yet";
  return CUTE_E_UNSUPPORTED;
}
cute_status adjoint_driver(cute_ctx *ctx, const cute_pair_desc *d, const double *G,
                           double *grad_a, double *grad_b) {
  ctx->err = "the adjoint is not built yet";
  return CUTE_E_UNSUPPORTED;
}
}  // namespace cute
