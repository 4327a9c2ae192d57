// Streaming variant, host side: workspace size and layout, and the decode entry that
// dispatches to the FP32 and fixed-point instantiations (stream_fp32.cu, stream_fixed.cu)
// of the kernels in stream_kernels.cuh.
#include <algorithm>

#include "../../include/ldpc.h"
#include "cmsg.cuh"
#include "ldpc_internal.h"

namespace ldpc_impl {

int stream_decode_fp32(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);
int stream_decode_fixed(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);

size_t stream_bytes(int mode, int32_t N, int64_t slots, int32_t Fp, int32_t L) {
    size_t tb = mode == kModeFP32 ? 4 : 2, rb = mode == kModeFP32 ? 4 : 1;
    return (size_t)slots * Fp * tb + (size_t)N * Fp * (tb + rb) + (size_t)N * (Fp / 4) + (size_t)Fp * 13 +
           (size_t)(L + 2) * Fp + 256;
}

StreamWork stream_carve(int mode, void* mem, int32_t N, int64_t slots, int32_t Fp, int32_t L) {
    // Fp is a multiple of 256, so every region below starts 64-byte aligned (256-byte up to hd)
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
    w.hd = (uint8_t*)p;
    p += (size_t)N * (Fp / 4);
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

// Messages of a streaming workspace, frame-major in CSR edge order: out[f E + e] = the
// message of edge e (slot: e, or i D + t on the padded row layout, for the t-th edge of row
// i) of frame f, times `scale` (1 in FP32, 1/4 in fixed point: exact). The row of an edge
// is found by binary search over the row offsets (a diagnostic path, not a hot one).
template <typename T>
__global__ void k_read_messages(const T* __restrict__ eta, int32_t Fp, const int32_t* __restrict__ row_ptr,
                                int32_t M, int32_t D, int32_t frames, int64_t E, float scale,
                                float* __restrict__ out) {
    const int64_t total = (int64_t)frames * E;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(k / E);
        const int32_t e = (int32_t)(k - (int64_t)f * E);
        int64_t slot = e;
        if (D > 0) {
            int32_t lo = 0, hi = M;  // the last row whose offset is <= e
            while (hi - lo > 1) {
                const int32_t mid = (lo + hi) >> 1;
                if (row_ptr[mid] <= e) lo = mid;
                else hi = mid;
            }
            slot = (int64_t)lo * D + (e - row_ptr[lo]);
        }
        out[k] = (float)eta[slot * Fp + f] * scale;
    }
}

// The same from compressed messages (cmsg.cuh): the message of the t-th edge of row i is
// rebuilt from the row's state, weighted by the class of the edge's bit when w_alpha is set.
__global__ void k_read_cmessages(CState cs, int32_t Fp, const int32_t* __restrict__ row_ptr,
                                 const int32_t* __restrict__ col_idx, const uint8_t* __restrict__ col_class,
                                 int32_t M, int32_t frames, int64_t E, const float* w_alpha,
                                 const float* w_beta, float* __restrict__ out) {
    const int64_t total = (int64_t)frames * E;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t f = (int32_t)(k / E);
        const int32_t e = (int32_t)(k - (int64_t)f * E);
        int32_t lo = 0, hi = M;
        while (hi - lo > 1) {
            const int32_t mid = (lo + hi) >> 1;
            if (row_ptr[mid] <= e) lo = mid;
            else hi = mid;
        }
        const int t = e - row_ptr[lo];
        const size_t o = (size_t)lo * Fp + f;
        float m = cmsg_mag(cs.m0[o], cs.m1[o], cs.w[o], t);
        if (w_alpha) {
            const int c = col_class[col_idx[e]];
            m = cmsg_weight(m, w_alpha[c], w_beta[c]);
        }
        out[k] = cmsg_signed(m, cs.w[o], t);
    }
}

int stream_read_messages(int mode, const DevGraph& g, int32_t M, int64_t E, const StreamWork& w,
                         int32_t frames, float* out, cudaStream_t st, int cmp, const float* w_alpha,
                         const float* w_beta) {
    const int64_t total = (int64_t)frames * E;
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 65535);
    if (cmp)
        k_read_cmessages<<<grid, 256, 0, st>>>(cstate_at(w.eta, M, w.Fp), w.Fp, g.row_ptr, g.col_idx,
                                               g.col_class, M, frames, E, w_alpha, w_beta, out);
    else if (mode == kModeFP32)
        k_read_messages<float><<<grid, 256, 0, st>>>((const float*)w.eta, w.Fp, g.row_ptr, M, g.ell_D,
                                                     frames, E, 1.0f, out);
    else
        k_read_messages<int16_t><<<grid, 256, 0, st>>>((const int16_t*)w.eta, w.Fp, g.row_ptr, M,
                                                       g.ell_D, frames, E, 0.25f, out);
    return cudaGetLastError() == cudaSuccess ? 1 : LDPC_ERR_CUDA;
}

int stream_decode(int mode, const DevGraph& g, const DecodeArgs& a, const StreamWork& w,
                  cudaStream_t st, int vw) {
    // vw: frames per lane (0 = the 16-byte vector of the mode); w.Fp is a multiple of 32 vw.
    return mode == kModeFP32 ? stream_decode_fp32(g, a, w, st, vw) : stream_decode_fixed(g, a, w, st, vw);
}

}  // namespace ldpc_impl
