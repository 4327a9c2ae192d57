// FP32 instantiations of the resident kernel (see resident.cuh), without the early-stop form.
#include "resident.cuh"

namespace ldpc_impl {
namespace resident {
int dispatch_fp32(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    return dispatch<kModeFP32, false>(ra, p, num_sms, st);
}
}  // namespace resident
}  // namespace ldpc_impl
