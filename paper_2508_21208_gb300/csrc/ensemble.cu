// ensemble.cu -- batched storm ensemble (placeholder until the persistent kernel lands).
#include "api_internal.h"

struct EnsembleState {};

int ensemble_attach(dgswem_ctx *c, void *, size_t, void *) { return ctx_fail(c, DGSWEM_ESTATE, "ensemble not available"); }
void ensemble_enqueue_step(dgswem_ctx *, std::vector<const char *> *) {}
void ensemble_release(dgswem_ctx *c) { delete c->ens; c->ens = nullptr; }

extern "C" {
int dgswem_ensemble_create(int32_t, const dgswem_mesh *const *, const double *const *, const dgswem_params *,
                           const dgswem_init *, const dgswem_tuning *, dgswem_ctx **out) {
  if (out) *out = nullptr;
  return DGSWEM_EINVAL;
}
int dgswem_ensemble_get_state(dgswem_ctx *, int32_t, double *, double *, double *) { return DGSWEM_EINVAL; }
int dgswem_ensemble_info(dgswem_ctx *, int32_t, double *, double *, int64_t *) { return DGSWEM_EINVAL; }
int dgswem_ensemble_set_fault(dgswem_ctx *, int32_t) { return DGSWEM_EINVAL; }
}
