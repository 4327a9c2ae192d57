// Streaming variant, host side: workspace size and layout, and the decode entry that
// dispatches to the FP32 and fixed-point instantiations (stream_fp32.cu, stream_fixed.cu)
// of the kernels in stream_kernels.cuh.
#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace ldpc_impl {

int stream_decode_fp32(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);
int stream_decode_fixed(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);

size_t stream_bytes(int mode, int32_t N, int64_t slots, int32_t Fp, int32_t L) {
    size_t tb = mode == kModeFP32 ? 4 : 2, rb = mode == kModeFP32 ? 4 : 1;
    return (size_t)slots * Fp * tb + (size_t)N * Fp * (tb + rb) + (size_t)Fp * 13 + (size_t)(L + 2) * Fp + 256;
}

StreamWork stream_carve(int mode, void* mem, int32_t N, int64_t slots, int32_t Fp, int32_t L) {
    // Fp is a multiple of 256, so every region below starts 256-byte aligned
    const size_t tb = mode == kModeFP32 ? 4 : 2, rb = mode == kModeFP32 ? 4 : 1;
    char* p = (char*)mem;
    StreamWork w;
    w.Fp = Fp;
    w.eta = p;
    p += (size_t)slots * Fp * tb;
    w.s = p;
    p += (size_t)N * Fp * tb;
    w.r = p;
    p += (size_t)N * Fp * rb;
    w.done_iter = (int32_t*)p;
    p += (size_t)Fp * 4;
    w.pos2frame = (int32_t*)p;
    p += (size_t)Fp * 4;
    w.new_pos = (int32_t*)p;
    p += (size_t)Fp * 4;
    w.state = (uint8_t*)p;
    p += (size_t)Fp;
    w.unsat = (uint8_t*)p;
    p += (size_t)(L + 2) * Fp;
    w.n_done = (int32_t*)p;  // the last 256 bytes: counters
    w.err = w.n_done + 1;
    w.comp = w.n_done + 4;
    return w;
}

int stream_decode(int mode, const DevGraph& g, const DecodeArgs& a, const StreamWork& w,
                  cudaStream_t st, int vw) {
    // vw: frames per lane (0 = the 16-byte vector of the mode); w.Fp is a multiple of 32 vw.
    return mode == kModeFP32 ? stream_decode_fp32(g, a, w, st, vw) : stream_decode_fixed(g, a, w, st, vw);
}

}  // namespace ldpc_impl
