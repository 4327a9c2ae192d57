// Dense variant: the paper's map-reduce form (Section III, Algorithm 2) on GB300, kept as
// a baseline. Every frame carries full m x n matrices, as in the paper; nothing depends
// on where H's ones are except through the mask:
//   map:    lambda(i,j) = s(j) H(i,j) - eta(i,j)                  (eq. firstIterationFanOut
//                                                                  and the later update)
//   reduce: per row, min0 / its first column / min1 over H(i,j) = 1, and the sign product
//           over the whole row with sign(0) = +1
//   map:    eta(i,j) = H(i,j) sign(lambda(i,j)) sgn(i) (min1 at min0's column, else min0)
//   reduce: s(j) = r(j) + sum over all rows i of eta(i,j)     (eq. sCalculation; eta = 0
//           off the support adds nothing)
//   then the hard decision and H b = 0 over GF(2) from the bit-packed rows.
// The paper's kernels split these steps further (its listing launches about 15 kernels per
// iteration, one frame at a time); here one CTA per (row, frame) does the first three and
// one thread per (column, frame) the column sum; frames are batched. FP32 mode.
#include <algorithm>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace ldpc_impl {
namespace {

constexpr int kRowThreads = 128;

__device__ __forceinline__ bool hbit(const uint32_t* packed, int W, int i, int j) {
    return (__ldg(packed + (size_t)i * W + (j >> 5)) >> (j & 31)) & 1u;
}

// One CTA per (row i, frame f): the row reductions and the new eta row.
__global__ void __launch_bounds__(kRowThreads) k_dense_row(const uint32_t* __restrict__ packed,
                                                           int M, int N, int W,
                                                           const float* __restrict__ s,
                                                           float* eta, int first,
                                                           const int32_t* __restrict__ done) {
    const int i = blockIdx.x, f = blockIdx.y;
    if (done[f] >= 0) return;
    const float* sf = s + (size_t)f * N;
    float* er = eta + ((size_t)f * M + i) * N;
    float min0 = __int_as_float(0x7f800000), min1 = min0;
    int loc = 0x7fffffff;
    uint32_t neg = 0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const bool h = hbit(packed, W, i, j);
        const float lam = sf[j] * (h ? 1.0f : 0.0f) - (first ? 0.0f : er[j]);
        neg ^= lam < 0.0f;  // the whole row: lambda = 0 off the support counts as +1
        if (h) {
            const float a = fabsf(lam);
            if (a < min0) {
                min1 = min0;
                min0 = a;
                loc = j;
            } else if (a < min1) {
                min1 = a;
            }
        }
    }
    // block reduction of (min0, loc, min1) and the sign parity
    __shared__ float s0[kRowThreads], s1[kRowThreads];
    __shared__ int sl[kRowThreads];
    __shared__ uint32_t sn[kRowThreads];
    s0[threadIdx.x] = min0;
    s1[threadIdx.x] = min1;
    sl[threadIdx.x] = loc;
    sn[threadIdx.x] = neg;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const int o = threadIdx.x + w;
            float a0 = s0[threadIdx.x], a1 = s1[threadIdx.x], b0 = s0[o], b1 = s1[o];
            int la = sl[threadIdx.x], lb = sl[o];
            // merge two (min0, loc, min1) summaries; ties go to the lower column
            const bool take_b = b0 < a0 || (b0 == a0 && lb < la);
            const float m0 = take_b ? b0 : a0;
            const int l0 = take_b ? lb : la;
            const float m1 = fminf(take_b ? a0 : b0, fminf(a1, b1));
            s0[threadIdx.x] = m0;
            s1[threadIdx.x] = m1;
            sl[threadIdx.x] = l0;
            sn[threadIdx.x] ^= sn[o];
        }
        __syncthreads();
    }
    const float m0 = s0[0], m1 = s1[0];
    const int l0 = sl[0];
    const uint32_t sgn = sn[0];
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const bool h = hbit(packed, W, i, j);
        float out = 0.0f;
        if (h) {
            const float lam = sf[j] - (first ? 0.0f : er[j]);
            const float m = (j == l0) ? m1 : m0;
            out = (sgn ^ (uint32_t)(lam < 0.0f)) ? -m : m;
        }
        er[j] = out;
    }
}

// One thread per (column j, frame f): s(j) = r(j) + sum over all rows of eta(i, j).
__global__ void k_dense_col(int M, int N, const float* __restrict__ r, float* s,
                            const float* __restrict__ eta, const int32_t* __restrict__ done,
                            int frames) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x, f = blockIdx.y;
    if (j >= N || done[f] >= 0) return;
    float acc = r[(size_t)f * N + j];
    const float* e = eta + (size_t)f * M * N + j;
    for (int i = 0; i < M; i++) acc = acc + e[(size_t)i * N];
    s[(size_t)f * N + j] = acc;
}

// One CTA per frame: hard decisions, H b over GF(2) (bit-packed), stop when zero.
__global__ void k_dense_syndrome(const uint32_t* __restrict__ packed, int M, int N, int W,
                                 const float* __restrict__ s, int32_t* done, int k, int test,
                                 int paper, uint32_t* bitbuf, uint8_t* unsat_final) {
    const int f = blockIdx.x;
    if (done[f] >= 0) return;
    uint32_t* bw = bitbuf + (size_t)f * W;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        uint32_t x = 0;
        for (int b = 0; b < 32 && w * 32 + b < N; b++) {
            const float v = s[(size_t)f * N + w * 32 + b];
            x |= (uint32_t)(paper ? v > 0.0f : v < 0.0f) << b;
        }
        bw[w] = x;
    }
    __syncthreads();
    __shared__ int any;
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
        uint32_t p = 0;
        for (int w = 0; w < W; w++) p ^= __popc(__ldg(packed + (size_t)i * W + w) & bw[w]) & 1u;
        if (p) any = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (unsat_final) unsat_final[f] = (uint8_t)any;
        else if (test && !any) done[f] = k;
    }
}

__global__ void k_dense_init(const float* llr, int frames, int N, float* r, float* s, int32_t* done) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (size_t)frames * N) {
        const float v = llr[t];
        r[t] = v;
        s[t] = v;
    }
    if (t < (size_t)frames) done[t] = -1;
}

__global__ void k_dense_out(const float* s, const int32_t* done, const uint8_t* unsat_final,
                            int frames, int N, int L, int paper, uint8_t* bits, int32_t* iters,
                            uint8_t* ok, float* soft) {
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < (size_t)frames * N) {
        const float v = s[t];
        bits[t] = (uint8_t)(paper ? v > 0.0f : v < 0.0f);
        if (soft) soft[t] = v;
    }
    if (t < (size_t)frames) {
        iters[t] = done[t] >= 0 ? done[t] : L;
        if (ok) ok[t] = done[t] >= 0 ? 1 : (unsat_final[t] == 0);
    }
}

}  // namespace

size_t dense_bytes(int32_t M, int32_t N, int32_t frames) {
    const int32_t W = (N + 31) / 32;
    return (size_t)frames * ((size_t)M * N * 4 + (size_t)N * 8 + (size_t)W * 4 + 8) + 1024;
}

int dense_decode(const DevGraph& g, const DecodeArgs& a, void* work, cudaStream_t st) {
    if (a.llr_is_i8) return LDPC_ERR_UNSUPPORTED;
    const int M = a.M, N = a.N, W = (N + 31) / 32, F = a.frames;
    char* p = (char*)work;
    float* eta = (float*)p;
    p += ((size_t)F * M * N * 4 + 255) & ~(size_t)255;
    float* r = (float*)p;
    p += ((size_t)F * N * 4 + 255) & ~(size_t)255;
    float* s = (float*)p;
    p += ((size_t)F * N * 4 + 255) & ~(size_t)255;
    uint32_t* bitbuf = (uint32_t*)p;
    p += ((size_t)F * W * 4 + 255) & ~(size_t)255;
    int32_t* done = (int32_t*)p;
    p += ((size_t)F * 4 + 255) & ~(size_t)255;
    uint8_t* unsat = (uint8_t*)p;
    const size_t FN = (size_t)F * N;
    int launches = 0;
    k_dense_init<<<(unsigned)((FN + 255) / 256), 256, 0, st>>>((const float*)a.llr, F, N, r, s, done);
    launches++;
    if (a.early_stop) {
        k_dense_syndrome<<<F, 128, 0, st>>>(g.packed, M, N, W, s, done, 0, 1, a.paper_slicer, bitbuf, nullptr);
        launches++;
    }
    for (int k = 1; k <= a.L; k++) {
        k_dense_row<<<dim3(M, F), kRowThreads, 0, st>>>(g.packed, M, N, W, s, eta, k == 1, done);
        k_dense_col<<<dim3((N + 127) / 128, F), 128, 0, st>>>(M, N, r, s, eta, done, F);
        launches += 2;
        if (a.early_stop && k % a.check_every == 0) {
            k_dense_syndrome<<<F, 128, 0, st>>>(g.packed, M, N, W, s, done, k, 1, a.paper_slicer, bitbuf, nullptr);
            launches++;
        }
    }
    k_dense_syndrome<<<F, 128, 0, st>>>(g.packed, M, N, W, s, done, a.L, 0, a.paper_slicer, bitbuf, unsat);
    k_dense_out<<<(unsigned)((FN + 255) / 256), 256, 0, st>>>(s, done, unsat, F, N, a.L, a.paper_slicer,
                                                              a.out_bits, a.out_iters, a.out_ok, a.out_soft);
    launches += 2;
    return cudaGetLastError() == cudaSuccess ? launches : LDPC_ERR_CUDA;
}

}  // namespace ldpc_impl
