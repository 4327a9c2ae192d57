// Fixed-point instantiations of the streaming kernels (stream_kernels.cuh).
#include "stream_kernels.cuh"

namespace ldpc_impl {

int stream_decode_fixed(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw) {
    switch (vw) {
        case 1: return run<kModeFixed, 1>(g, a, w, st);
        case 2: return run<kModeFixed, 2>(g, a, w, st);
        case 4: return run<kModeFixed, 4>(g, a, w, st);
        case 0:
        case Tr<kModeFixed>::V: return run<kModeFixed, Tr<kModeFixed>::V>(g, a, w, st);
        default: return LDPC_ERR_INVALID_ARG;
    }
}

}  // namespace ldpc_impl
