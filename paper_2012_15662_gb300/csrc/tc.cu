// Split-precision tensor-core path (placeholder until the tcgen05 kernels land).
#include "common.cuh"

namespace donof {
int mixed_init(donof_ri_ctx*) { return DONOF_RI_E_UNSUPPORTED; }
void mixed_free(donof_ri_ctx*) {}
int mixed_transform(donof_ri_ctx*, int) { return DONOF_RI_E_UNSUPPORTED; }
int mixed_jk_ao(donof_ri_ctx*) { return DONOF_RI_E_UNSUPPORTED; }
int mixed_energy(donof_ri_ctx*) { return DONOF_RI_E_UNSUPPORTED; }
int mixed_fetch(donof_ri_ctx*, int, double*, size_t) { return DONOF_RI_E_UNSUPPORTED; }
int mixed_copy_ao(donof_ri_ctx*, double*, double*, bool, bool) { return DONOF_RI_E_UNSUPPORTED; }
}  // namespace donof
