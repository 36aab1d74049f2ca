// Entry points whose kernels are not in this build yet report EXA_ERR_ARG.
#include "ctx.cuh"

namespace exa {
exa_status loglik_mixed(exa_ctx* c, const double*, const double*, const double*, int64_t, exa_prec, exa_result*) {
  return set_err(c, EXA_ERR_ARG, "mixed precision is not available in this build");
}
void release_extra(exa_ctx*) {}
}  // namespace exa

extern "C" {
exa_status exa_loglik_grad(exa_ctx* c, const double*, const double*, const double*, int64_t, exa_prec, double*,
                           double*) {
  return exa::set_err(c, EXA_ERR_ARG, "gradient is not available in this build");
}
exa_status exa_loglik_batched(exa_ctx* c, int32_t, const int64_t*, const double* const*, const double* const*,
                              const double*, exa_prec, double*, int32_t*) {
  return exa::set_err(c, EXA_ERR_ARG, "batched form is not available in this build");
}
}
