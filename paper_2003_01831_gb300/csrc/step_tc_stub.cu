// Placeholder tensor-core driver (replaced by step_tc.cu).
#include "state.cuh"
namespace afqmc {
int tc_alloc(afqmc_walkers*, cudaStream_t) { return fail(AFQMC_ERR_UNSUPPORTED, "BF16X3 path not built"); }
void tc_free(afqmc_walkers*) {}
int tc_measure(afqmc_walkers*, bool, cudaStream_t) { return fail(AFQMC_ERR_UNSUPPORTED, "BF16X3 path not built"); }
int tc_propagate_and_weight(afqmc_walkers*, const double*, cudaStream_t) { return fail(AFQMC_ERR_UNSUPPORTED, "BF16X3 path not built"); }
int tc_qr(afqmc_walkers*, cudaStream_t) { return fail(AFQMC_ERR_UNSUPPORTED, "BF16X3 path not built"); }
int tc_sync_walkers_to_fp64(afqmc_walkers*, cudaStream_t) { return AFQMC_OK; }
int tc_sync_walkers_from_fp64(afqmc_walkers*, cudaStream_t) { return AFQMC_OK; }
int fp64_backward(afqmc_walkers*, const cplx*, const cplx*, cplx*, cplx*, double*, cudaStream_t) {
    return fail(AFQMC_ERR_UNSUPPORTED, "energy_backward not built");
}
}
