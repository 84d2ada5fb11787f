// pool.cu -- batched stepping of many domains (filled in below).
#include "internal.h"

extern "C" {
slbm_status slbm_pool_create(int32_t, int32_t, int32_t, void *, slbm_pool_t **out) {
    if (out) *out = nullptr;
    slbm::set_error(SLBM_EUNSUPPORTED, "pool not built");
    return SLBM_EUNSUPPORTED;
}
slbm_status slbm_pool_add(slbm_pool_t *, slbm_t *, int32_t *) { return SLBM_EUNSUPPORTED; }
slbm_status slbm_pool_remove(slbm_pool_t *, int32_t) { return SLBM_EUNSUPPORTED; }
slbm_status slbm_pool_step(slbm_pool_t *, int32_t, int32_t) { return SLBM_EUNSUPPORTED; }
slbm_status slbm_pool_reduce(slbm_pool_t *, double *, int32_t) { return SLBM_EUNSUPPORTED; }
slbm_status slbm_pool_set_launch(slbm_pool_t *, int32_t, int32_t) { return SLBM_EUNSUPPORTED; }
void slbm_pool_free(slbm_pool_t *) {}
}
