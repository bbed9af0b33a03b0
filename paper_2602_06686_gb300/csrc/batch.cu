// batch.cu -- placeholder until the persistent batched driver lands.
#include "internal.h"

using namespace lbm;

extern "C" {
int lbm_batch_buffer_sizes(int, const lbm_params*, size_t*, size_t*) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_create(int, const lbm_params*, void*, lbm_batch**) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_bind(lbm_batch*, void*, void*, void*) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_lattice(lbm_batch*, int, lbm_ctx**) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_step(lbm_batch*, int, int) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_variant_count(const lbm_batch*, int*) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_variant_name(const lbm_batch*, int, char*, size_t) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_set_variant(lbm_batch*, int) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_autotune(lbm_batch*, int, int*, float*) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_set_barrier(lbm_batch*, double, int) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_launches(const lbm_batch*, long long*) { return LBM_ERR_UNSUPPORTED; }
int lbm_batch_destroy(lbm_batch*) { return LBM_OK; }
}
