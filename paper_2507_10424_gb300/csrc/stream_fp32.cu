// FP32 instantiations of the streaming kernels (stream_kernels.cuh).
#include "stream_kernels.cuh"

namespace ldpc_impl {

int stream_decode_fp32(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw) {
    switch (vw) {
        case 1: return run<kModeFP32, 1>(g, a, w, st);
        case 2: return run<kModeFP32, 2>(g, a, w, st);
        case 0:
        case Tr<kModeFP32>::V: return run<kModeFP32, Tr<kModeFP32>::V>(g, a, w, st);
        default: return LDPC_ERR_INVALID_ARG;
    }
}

}  // namespace ldpc_impl
