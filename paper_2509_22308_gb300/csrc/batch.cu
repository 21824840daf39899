// Batched design diagrams: packed multi-domain layout and persistent step kernel.
#include "../../include/lbm_em.h"
#include "runtime.h"

using namespace lbmem;

struct lbm_em_batch {
    int n;
};

extern "C" {

lbm_em_status lbm_em_batch_create(const lbm_em_instance *, int32_t, const lbm_em_batch_opts *, lbm_em_batch_t **out) {
    if (out) *out = nullptr;
    return set_error(LBM_EM_ESTATE, "batched runs are not available in this build yet");
}
lbm_em_status lbm_em_batch_run(lbm_em_batch_t *) { return set_error(LBM_EM_ESTATE, "no batch"); }
lbm_em_status lbm_em_batch_results(lbm_em_batch_t *, double *, int32_t *) { return set_error(LBM_EM_ESTATE, "no batch"); }
lbm_em_status lbm_em_batch_config(lbm_em_batch_t *, int32_t *, int32_t *, int32_t *) {
    return set_error(LBM_EM_ESTATE, "no batch");
}
lbm_em_status lbm_em_batch_destroy(lbm_em_batch_t *) { return LBM_EM_OK; }

}  // extern "C"
