// Resident variant: one persistent kernel. Each CTA takes tiles of FT frames from an
// atomic work counter and runs every flooding iteration of Algorithm 1 for that tile with
// the edge messages eta and posteriors s of all FT frames held in shared memory; only the
// channel LLRs are read from, and the decisions written to, global memory.
//
// Shared-memory layout per frame f: eta_f[E_pad] in the sliced order (slot of the k-th
// edge of row-lane l of slice sl = slice_base[sl] + 32 k + l, so a warp's 32 lanes touch
// 32 consecutive words), then s_f[N_pad].
//
// One iteration = phase A (rows) + phase B (columns), separated by CTA barriers:
//   phase A, thread per row-lane, all FT frames: lambda = s_col - eta (eta^prev = 0 in
//     the first iteration), Observation 1 (min0, first location, min1) and Observation 2
//     (XOR of sign bits), eta = +-(min1 at the location, else min0); the same sweep XORs
//     the decisions of the gathered s, i.e. the syndrome (eq. 1-2) of the current s;
//   phase B, thread per column, all FT frames: s_j = r_j + sum of eta in ascending row
//     order (eq. lambda_j). Frames whose syndrome was zero stop before phase B.
#include <algorithm>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace ldpc_impl {
namespace {

constexpr int kMaxThreads = 1024;

template <int MODE>
struct RT;
template <>
struct RT<kModeFP32> {
    using T = float;
    using A = float;
};
template <>
struct RT<kModeFixed> {
    using T = int16_t;
    using A = int32_t;
};

__device__ __forceinline__ int32_t rsat16(int32_t v) { return max(-kSat, min(kSat, v)); }
__device__ __forceinline__ float rlam(float s, float e) { return s - e; }
__device__ __forceinline__ int32_t rlam(int32_t s, int32_t e) { return rsat16(s - e); }
__device__ __forceinline__ float rabs(float x) { return fabsf(x); }
__device__ __forceinline__ int32_t rabs(int32_t x) { return abs(x); }
__device__ __forceinline__ float rbig(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t rbig(int32_t) { return 0x7fffffff; }
template <typename A>
__device__ __forceinline__ uint32_t rslice(A s, int paper) {
    return paper ? (s > A(0)) : (s < A(0));
}
__device__ __forceinline__ int8_t rquant(float x) {
    float t = 4.0f * x;
    if (t != t) return 0;
    t = fminf(fmaxf(t, -127.0f), 127.0f);
    return (int8_t)__float2int_rn(t);
}

struct ResArgs {
    const int32_t* slice_base;
    const uint8_t* row_deg;
    const uint16_t* slot_col;
    const int32_t* col_ptr;
    const uint16_t* col_slot16;
    const int32_t* col_slot32;
    int32_t n_tasks, E_pad, N, N_pad;
    const void* llr;
    int32_t llr_i8;
    int32_t frames, n_tiles, L, early_stop, check_every, paper;
    uint8_t* out_bits;
    int32_t* out_iters;
    uint8_t* out_ok;
    float* out_soft;
    int32_t* tile_counter;
};

// Channel value of (frame, bit) in the arithmetic of the mode.
template <int MODE>
__device__ __forceinline__ typename RT<MODE>::A chan(const ResArgs& a, size_t idx) {
    if (MODE == kModeFP32) return __ldg((const float*)a.llr + idx);
    if (a.llr_i8) return (int32_t)__ldg((const int8_t*)a.llr + idx);
    return (int32_t)rquant(__ldg((const float*)a.llr + idx));
}

template <int MODE, int FT>
__global__ void __launch_bounds__(kMaxThreads, 1) k_resident(const ResArgs a) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* eta = reinterpret_cast<T*>(smem_raw);
    T* sv = eta + (size_t)FT * a.E_pad;
    __shared__ int unsat[2][FT];
    __shared__ int tile_sh;
    const int tid = threadIdx.x, nth = blockDim.x;
    const int E_pad = a.E_pad, N = a.N, N_pad = a.N_pad;

    for (;;) {
        if (tid == 0) tile_sh = atomicAdd(a.tile_counter, 1);
        if (tid < 2 * FT) unsat[tid / FT][tid % FT] = 0;
        __syncthreads();
        const int tile = tile_sh;
        if (tile >= a.n_tiles) break;
        const int fbase = tile * FT;
        const int nf = min(FT, a.frames - fbase);
        for (int f = 0; f < nf; f++)
            for (int j = tid; j < N; j += nth) sv[f * N_pad + j] = (T)chan<MODE>(a, (size_t)(fbase + f) * N + j);
        uint32_t active = (1u << nf) - 1u, okm = 0;
        int its[FT];
#pragma unroll
        for (int f = 0; f < FT; f++) its[f] = a.L;
        __syncthreads();

        for (int k = 0;; k++) {
            const int par = k & 1;
            const bool last = (k == a.L);
            const bool syn = last || (a.early_stop && (k % a.check_every == 0));
            const bool first = (k == 0);
            // ---------------- phase A: check nodes (and syndrome of the current s)
            for (int task = tid; task < a.n_tasks; task += nth) {
                const int d = a.row_deg[task];
                if (d == 0) continue;
                const int base = a.slice_base[task >> 5] + (task & 31);
                A min0[FT], min1[FT];
                int loc[FT];
                uint32_t msk[FT];
                uint32_t neg = 0, z = 0;
#pragma unroll
                for (int f = 0; f < FT; f++) {
                    min0[f] = rbig(A());
                    min1[f] = rbig(A());
                    loc[f] = 0;
                    msk[f] = 0;
                }
                const bool longrow = d > 32;
                for (int t = 0; t < d; t++) {
                    const int slot = base + 32 * t;
                    const int col = __ldg(a.slot_col + slot);
#pragma unroll
                    for (int f = 0; f < FT; f++) {
                        if (!((active >> f) & 1u)) continue;
                        const A s_ = (A)sv[f * N_pad + col];
                        if (syn) z ^= rslice(s_, a.paper) << f;
                        if (!last) {
                            const A lam = first ? s_ : rlam(s_, (A)eta[f * E_pad + slot]);
                            const A m = rabs(lam);
                            const uint32_t sg = lam < A(0);
                            if (m < min0[f]) {
                                min1[f] = min0[f];
                                min0[f] = m;
                                loc[f] = t;
                            } else if (m < min1[f]) {
                                min1[f] = m;
                            }
                            neg ^= sg << f;
                            msk[f] |= sg << (t & 31);
                            if (longrow) eta[f * E_pad + slot] = (T)lam;
                        }
                    }
                }
                if (syn && (z & active)) {
#pragma unroll
                    for (int f = 0; f < FT; f++)
                        if (((z & active) >> f) & 1u) unsat[par][f] = 1;
                }
                if (!last) {
                    for (int t = 0; t < d; t++) {
                        const int slot = base + 32 * t;
#pragma unroll
                        for (int f = 0; f < FT; f++) {
                            if (!((active >> f) & 1u)) continue;
                            const uint32_t sg = longrow ? (uint32_t)((A)eta[f * E_pad + slot] < A(0))
                                                        : ((msk[f] >> t) & 1u);
                            const A m = (t == loc[f]) ? min1[f] : min0[f];
                            eta[f * E_pad + slot] = (T)((((neg >> f) ^ sg) & 1u) ? -m : m);
                        }
                    }
                }
            }
            __syncthreads();
            if (syn) {
                uint32_t zm = 0;
#pragma unroll
                for (int f = 0; f < FT; f++) zm |= (uint32_t)(unsat[par][f] != 0) << f;
                const uint32_t conv = active & ~zm;
                okm |= conv;
                if (last) break;
#pragma unroll
                for (int f = 0; f < FT; f++)
                    if ((conv >> f) & 1u) its[f] = k;
                active &= ~conv;
                if (!active) break;
            }
            // ---------------- phase B: bit nodes
            for (int j = tid; j < N; j += nth) {
                const int t0 = __ldg(a.col_ptr + j), t1 = __ldg(a.col_ptr + j + 1);
                A acc[FT];
#pragma unroll
                for (int f = 0; f < FT; f++)
                    if ((active >> f) & 1u) acc[f] = chan<MODE>(a, (size_t)(fbase + f) * N + j);
                for (int t = t0; t < t1; t++) {
                    const int slot = a.col_slot16 ? (int)__ldg(a.col_slot16 + t) : __ldg(a.col_slot32 + t);
#pragma unroll
                    for (int f = 0; f < FT; f++)
                        if ((active >> f) & 1u) acc[f] = acc[f] + (A)eta[f * E_pad + slot];
                }
#pragma unroll
                for (int f = 0; f < FT; f++)
                    if ((active >> f) & 1u)
                        sv[f * N_pad + j] = (MODE == kModeFP32) ? (T)acc[f] : (T)rsat16((int32_t)acc[f]);
            }
            if (tid < FT) unsat[par ^ 1][tid] = 0;
            __syncthreads();
        }
        // ---------------- output of the tile
        for (int f = 0; f < nf; f++) {
            const size_t row = (size_t)(fbase + f) * N;
            for (int j = tid; j < N; j += nth) {
                const A s_ = (A)sv[f * N_pad + j];
                a.out_bits[row + j] = (uint8_t)rslice(s_, a.paper);
                if (a.out_soft) a.out_soft[row + j] = (MODE == kModeFP32) ? (float)s_ : (float)s_ * 0.25f;
            }
        }
#pragma unroll
        for (int f = 0; f < FT; f++)
            if (tid == f && f < nf) {
                a.out_iters[fbase + f] = its[f];
                if (a.out_ok) a.out_ok[fbase + f] = (okm >> f) & 1u;
            }
        __syncthreads();
    }
}

template <int MODE, int FT>
int launch(const ResArgs& ra, const ResidentPlan& p, int grid, cudaStream_t st) {
    // the opt-in shared-memory size is a per-function attribute: set it for this plan
    if (cudaFuncSetAttribute(k_resident<MODE, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)p.smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    k_resident<MODE, FT><<<grid, p.threads, p.smem, st>>>(ra);
    return cudaGetLastError() == cudaSuccess ? 1 : LDPC_ERR_CUDA;
}

template <int MODE>
int dispatch(const ResArgs& ra, const ResidentPlan& p, int grid, cudaStream_t st) {
    switch (p.FT) {
        case 1: return launch<MODE, 1>(ra, p, grid, st);
        case 2: return launch<MODE, 2>(ra, p, grid, st);
        case 3: return launch<MODE, 3>(ra, p, grid, st);
        case 4: return launch<MODE, 4>(ra, p, grid, st);
        case 6: return launch<MODE, 6>(ra, p, grid, st);
        case 8: return launch<MODE, 8>(ra, p, grid, st);
    }
    return LDPC_ERR_INVALID_ARG;
}

}  // namespace

static size_t frame_bytes(int mode, int32_t E_pad, int32_t N_pad) {
    const size_t tb = mode == kModeFP32 ? 4 : 2;
    return tb * ((size_t)E_pad + (size_t)N_pad);
}

ResidentPlan resident_plan(int mode, const DevGraph& dg, int32_t M, int32_t N, int device) {
    ResidentPlan p;
    (void)M;
    if (N > 65535 || dg.n_slices == 0) return p;
    int optin = 0, per_sm = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    const int32_t N_pad = (N + 7) & ~7;
    const size_t fb = frame_bytes(mode, dg.E_pad, N_pad);
    const size_t reserve = 1024 + 256;  // per-CTA system reserve + static shared memory
    if (fb + reserve > (size_t)optin) return p;
    static const int kFT[] = {8, 6, 4, 3, 2, 1};
    for (int ft : kFT)
        if (ft * fb + reserve <= (size_t)optin) {
            p.FT = ft;
            break;
        }
    // threads: minimise padded work of both phases; prefer more threads on ties
    const int tasks = dg.n_slices * 32;
    long best = -1;
    for (int t = 256; t <= kMaxThreads; t += 32) {
        const long cost = (long)((tasks + t - 1) / t) * t * 2 + (long)((N + t - 1) / t) * t;
        if (best < 0 || cost <= best) {  // ascending t: ties go to the larger CTA
            best = cost;
            p.threads = t;
        }
    }
    p.smem = p.FT * fb;
    p.ctas_per_sm = std::max(1, std::min((int)(per_sm / (p.smem + reserve)), 2048 / p.threads));
    p.ok = 1;
    return p;
}

int resident_decode(int mode, const DevGraph& dg, const ResidentPlan& p, const DecodeArgs& a,
                    int32_t* tile_counter, int num_sms, cudaStream_t st) {
    ResArgs ra;
    ra.slice_base = dg.s_slice_base;
    ra.row_deg = dg.s_row_deg;
    ra.slot_col = dg.s_slot_col;
    ra.col_ptr = dg.s_col_ptr;
    ra.col_slot16 = dg.s_col_slot16;
    ra.col_slot32 = dg.s_col_slot32;
    ra.n_tasks = dg.n_slices * 32;
    ra.E_pad = dg.E_pad;
    ra.N = a.N;
    ra.N_pad = (a.N + 7) & ~7;
    ra.llr = a.llr;
    ra.llr_i8 = a.llr_is_i8;
    ra.frames = a.frames;
    ra.n_tiles = (a.frames + p.FT - 1) / p.FT;
    ra.L = a.L;
    ra.early_stop = a.early_stop;
    ra.check_every = a.check_every;
    ra.paper = a.paper_slicer;
    ra.out_bits = a.out_bits;
    ra.out_iters = a.out_iters;
    ra.out_ok = a.out_ok;
    ra.out_soft = a.out_soft;
    ra.tile_counter = tile_counter;
    if (cudaMemsetAsync(tile_counter, 0, sizeof(int32_t), st) != cudaSuccess) return LDPC_ERR_CUDA;
    const int grid = std::max(1, std::min(ra.n_tiles, num_sms * p.ctas_per_sm));
    return mode == kModeFP32 ? dispatch<kModeFP32>(ra, p, grid, st) : dispatch<kModeFixed>(ra, p, grid, st);
}

}  // namespace ldpc_impl
