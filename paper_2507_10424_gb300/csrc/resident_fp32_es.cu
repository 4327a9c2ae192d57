// FP32 instantiations of the resident kernel's early-stop form (see resident.cuh).
#include "resident.cuh"

namespace ldpc_impl {
namespace resident {
int dispatch_fp32_es(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    return dispatch<kModeFP32, true>(ra, p, num_sms, st);
}
}  // namespace resident
}  // namespace ldpc_impl
