// wg_stubs.cu -- entry points whose kernels are not built yet return WG_ERR_UNSUPPORTED.
#include <cuda_runtime.h>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace wg {


}  // namespace wg

extern "C" {

struct wg_batch_plan {
    int unused;
};

int wigner_batch_plan_create(wg_batch_plan **plan, int, const wg_instance *, int, void *) {
    if (plan) *plan = nullptr;
    return WG_ERR_UNSUPPORTED;
}
int wigner_batch_run(wg_batch_plan *, int, void *) { return WG_ERR_UNSUPPORTED; }
void wigner_batch_plan_destroy(wg_batch_plan *) {}
int wigner_conv_sum_batched(int, const wg_instance *, void *) { return WG_ERR_UNSUPPORTED; }

}  // extern "C"
