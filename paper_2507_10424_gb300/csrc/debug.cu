// Device-side debug checks (ldpc_set_debug): before a decode, one pass over every index
// array the kernels read through and over the caller's LLRs, recording the first
// violation. The decode kernels address shared and global memory through these arrays
// (slot ids, column positions, CSR/CSC indices, the padded row layout, weight classes), so
// an entry out of range there, from a stray write into the handle's memory, would become
// an out-of-bounds access; the host refuses the decode instead. FP32 LLRs are checked for
// NaN, which the decoder does not define (its comparisons would be unordered).
//
// Report (two 64-bit words, set to all ones before the checks): [0] the smallest flat
// index of a NaN LLR (frame * N + bit), [1] the smallest (array id << 40 | entry) of a
// graph violation, array ids as in DebugArray.
#include <algorithm>
#include <cstdint>

#include "ldpc_internal.h"

namespace ldpc_impl {
namespace {

constexpr int kCheckThreads = 256;

__device__ __forceinline__ void report(unsigned long long* slot, unsigned long long v) { atomicMin(slot, v); }

__global__ void k_nan(const float* __restrict__ x, int64_t n, unsigned long long* rep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (isnan(x[i])) report(rep, (unsigned long long)i);
}

// Every entry of a in [0, bound).
template <typename T>
__global__ void k_below(const T* __restrict__ a, int64_t n, int64_t bound, int id, unsigned long long* rep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = (int64_t)a[i];
        if (v < 0 || v >= bound) report(rep, ((unsigned long long)id << 40) | (unsigned long long)i);
    }
}

// An offsets array of n + 1 entries: p[0] = 0, non-decreasing, p[n] = total.
__global__ void k_offsets(const int32_t* __restrict__ p, int64_t n, int64_t total, int id,
                          unsigned long long* rep) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i <= n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool bad = (i == 0 && p[0] != 0) || (i == n && p[n] != total) || (i < n && p[i] > p[i + 1]);
        if (bad) report(rep, ((unsigned long long)id << 40) | (unsigned long long)i);
    }
}

// Slice degrees: the d edges of lane t of slice t / 32 stay inside the slice's slots.
__global__ void k_slice_deg(const int32_t* __restrict__ base, const uint8_t* __restrict__ deg, int64_t tasks,
                            int id, unsigned long long* rep) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < tasks;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = t >> 5;
        if (base[q] + 32 * (int64_t)deg[t] > base[q + 1])
            report(rep, ((unsigned long long)id << 40) | (unsigned long long)t);
    }
}

int grid_for(int64_t n) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + kCheckThreads - 1) / kCheckThreads, 4096));
}

}  // namespace

int debug_check_launch(const DevGraph& g, int32_t M, int32_t N, int64_t E, const void* llr, int llr_is_i8,
                       int64_t frames, unsigned long long* rep, cudaStream_t st) {
    if (cudaMemsetAsync(rep, 0xff, 2 * sizeof(unsigned long long), st) != cudaSuccess) return LDPC_ERR_CUDA;
    unsigned long long* gr = rep + 1;
    auto below = [&](auto* a, int64_t n, int64_t bound, DebugArray id) {
        if (a && n > 0) k_below<<<grid_for(n), kCheckThreads, 0, st>>>(a, n, bound, (int)id, gr);
    };
    auto offsets = [&](const int32_t* p, int64_t n, int64_t total, DebugArray id) {
        if (p) k_offsets<<<grid_for(n + 1), kCheckThreads, 0, st>>>(p, n, total, (int)id, gr);
    };
    if (!llr_is_i8 && frames > 0) {
        const int64_t n = frames * (int64_t)N;
        k_nan<<<grid_for(n), kCheckThreads, 0, st>>>(static_cast<const float*>(llr), n, rep);
    }
    offsets(g.row_ptr, M, E, DebugArray::kRowPtr);
    offsets(g.col_ptr, N, E, DebugArray::kColPtr);
    below(g.col_idx, E, N, DebugArray::kColIdx);
    below(g.col_edge, E, E, DebugArray::kColEdge);
    if (g.n_classes > 0) below(g.col_class, N, g.n_classes, DebugArray::kColClass);
    if (g.sliced) {
        const int64_t rtasks = (int64_t)g.n_rslices * 32, ctasks = (int64_t)g.n_cslices * 32;
        offsets(g.r_base, g.n_rslices, g.E_pad, DebugArray::kRowBase);
        offsets(g.c_base, g.n_cslices, g.Ec_pad, DebugArray::kColBase);
        if (g.r_base && g.r_deg)
            k_slice_deg<<<grid_for(rtasks), kCheckThreads, 0, st>>>(g.r_base, g.r_deg, rtasks,
                                                                    (int)DebugArray::kRowDeg, gr);
        if (g.c_base && g.c_deg)
            k_slice_deg<<<grid_for(ctasks), kCheckThreads, 0, st>>>(g.c_base, g.c_deg, ctasks,
                                                                    (int)DebugArray::kColDeg, gr);
        below(g.r_slot_pos, g.E_pad, ctasks, DebugArray::kRowSlotPos);
        below(g.c_slot, g.Ec_pad, g.E_pad, DebugArray::kColSlot);
        below(g.col_pos, N, ctasks, DebugArray::kColPos);
        if (g.n_classes > 0) below(g.r_slot_cls, g.E_pad, g.n_classes, DebugArray::kRowSlotCls);
    }
    if (g.ell_D) {
        const int64_t slots = (int64_t)M * g.ell_D;
        below(g.ell_col, slots, N, DebugArray::kEllCol);
        below(g.ell_deg, M, g.ell_D + 1, DebugArray::kEllDeg);
        below(g.ell_cslot, E, slots, DebugArray::kEllCslot);
        if (g.n_classes > 0) below(g.ell_cls, slots, g.n_classes, DebugArray::kEllCls);
    }
    return cudaGetLastError() == cudaSuccess ? LDPC_OK : LDPC_ERR_CUDA;
}

}  // namespace ldpc_impl
