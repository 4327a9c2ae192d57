// Streaming variant: edge messages eta live in HBM in a frame-interleaved
// structure-of-arrays layout, element (message slot e, frame f) at e * Fp + f. The slots
// are the padded row layout's (row i owns slots i D .. i D + D - 1) when every row has at
// most 16 edges, else the CSR edge ids. A thread owns V consecutive frames (one 16-byte
// vector: 4 x fp32 or 8 x int16) of one row or column, so each warp moves 512 contiguous
// bytes per edge whatever the structure of H.
//
// Per flooding iteration k (Algorithm 1):
//   k_check: for every check i and frame: lambda_e = s_j - eta_e (eq. eta_update with
//            eta^prev), Observation 1 (min0, first location, min1) and Observation 2 (sign
//            product as XOR), then eta_e = +-(min1 at the location, min0 elsewhere).
//            The same pass XORs the hard decisions of the gathered s_j: that is the
//            syndrome of the previous iteration's decision (eq. 1-2).
//   k_var:   for every bit j and frame: s_j = r_j + sum of eta over M_j, ascending rows
//            (eq. lambda_j); frames whose previous syndrome was zero are frozen there.
// A final syndrome-only pass gives the status of frames that never stopped early. With
// early stop the running frames are compacted to the front now and then, and both passes
// then skip the frame blocks behind the positions in use (comp[1]).
#pragma once

#include "../../include/ldpc.h"
#include "cmsg.cuh"
#include "ldpc_internal.h"
#include "packed16.cuh"

#include <algorithm>
#include <type_traits>

namespace ldpc_impl {
namespace {

template <typename T, int V>
struct alignas(sizeof(T) * V) Vec {
    T x[V];
};

template <int MODE>
struct Tr;
template <>
struct Tr<kModeFP32> {
    using T = float;    // message / posterior storage
    using R = float;    // channel value storage
    using A = float;    // arithmetic
    static constexpr int V = 4;
};
template <>
struct Tr<kModeFixed> {
    using T = int16_t;
    using R = int8_t;
    using A = int32_t;
    static constexpr int V = 8;
};

__device__ __forceinline__ int32_t sat16(int32_t v) { return max(-kSat, min(kSat, v)); }
__device__ __forceinline__ float lam_of(float s, float e) { return s - e; }
__device__ __forceinline__ int32_t lam_of(int32_t s, int32_t e) { return sat16(s - e); }
__device__ __forceinline__ float absval(float x) { return fabsf(x); }
__device__ __forceinline__ int32_t absval(int32_t x) { return abs(x); }
__device__ __forceinline__ float big(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t big(int32_t) { return 0x7fffffff; }
template <typename A>
__device__ __forceinline__ uint32_t slice(A s, int paper) {
    return paper ? (s > A(0)) : (s < A(0));
}

// Quantiser of the fixed-point mode: clamp(round_half_even(4 x), -127, 127), NaN -> 0.
__device__ __forceinline__ int8_t quantize(float x) {
    float t = 4.0f * x;
    if (t != t) return 0;
    t = fminf(fmaxf(t, -127.0f), 127.0f);
    return (int8_t)__float2int_rn(t);
}

// Mark frames f0 + v (bit v of z) as having an unsatisfied check. Every check of a frame
// reports to the same byte, so the flags are read first and only the missing ones are
// written: after the first failing row, the other rows find the byte set and leave it
// (tens of thousands of stores to the same few L2 lines otherwise serialise the pass).
template <int VW>
__device__ __forceinline__ void flag_unsat(uint8_t* unsat, int f0, uint32_t z) {
    if (!z) return;
    uint32_t have = 0;
#pragma unroll
    for (int v = 0; v < VW; v++) have |= (uint32_t)(((volatile const uint8_t*)unsat)[f0 + v] != 0) << v;
    const uint32_t need = z & ~have;
    if (need) {
#pragma unroll
        for (int v = 0; v < VW; v++)
            if ((need >> v) & 1) unsat[f0 + v] = 1;
    }
}

// ------------------------------------------------------------------------------------
// Per-frame state
// ------------------------------------------------------------------------------------
__global__ void k_init_state(uint8_t* state, int32_t* done_iter, int32_t* pos2frame, int32_t* comp,
                             int Fp, int frames) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < Fp) {
        state[f] = f < frames;
        done_iter[f] = -1;
        pos2frame[f] = f < frames ? f : -1;
    }
    if (f == 0) {
        comp[0] = 0;       // no compaction pending
        comp[1] = frames;  // positions in use
        comp[2] = frames;
    }
}

// ------------------------------------------------------------------------------------
// Frame compaction (early stop). Stopped frames leave holes in the frame-interleaved
// arrays, and a frame block is skipped only when none of its frames runs. When at most half
// of the positions in use still run, the running frames move to the front, in order, and
// the blocks behind them go idle (a compaction moves about half an iteration's bytes, so it
// pays when it halves the work of the iterations left):
//   k_cmp_scan:  new position of every running frame (a prefix count), and the decision;
//   k_cmp_emit:  decisions, soft values and status of the stopped frames that are still
//                in place (their posteriors are about to be overwritten);
//   k_cmp_rows:  every row of r, s, eta and the position -> frame map compacted in place
//                (destinations never exceed sources, so a row is compacted chunk by chunk
//                after reading each chunk whole);
//   k_cmp_tail:  the frame states of the new layout, and the positions in use.
// Every kernel returns at once when no compaction is pending.
// ------------------------------------------------------------------------------------
constexpr int kCmpThreads = 1024;

__global__ void __launch_bounds__(kCmpThreads) k_cmp_scan(const uint8_t* __restrict__ state,
                                                          int32_t* __restrict__ new_pos,
                                                          int32_t* comp) {
    __shared__ int part[kCmpThreads];
    const int cur = comp[1];
    const int per = (cur + kCmpThreads - 1) / kCmpThreads;
    const int p0 = threadIdx.x * per, p1 = min(cur, p0 + per);
    int n = 0;
    for (int p = p0; p < p1; p++) n += state[p] != 0;
    part[threadIdx.x] = n;
    __syncthreads();
    for (int o = 1; o < kCmpThreads; o <<= 1) {  // inclusive scan of the per-thread counts
        const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    const int total = part[kCmpThreads - 1];
    const bool go = 2 * total <= cur && cur - total >= 64;
    if (go) {
        int q = part[threadIdx.x] - n;  // exclusive prefix
        for (int p = p0; p < p1; p++) new_pos[p] = state[p] != 0 ? q++ : -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        comp[0] = go;
        comp[2] = total;
    }
}

template <int MODE>
__global__ void k_cmp_emit(const typename Tr<MODE>::T* s, int Fp, int N, const uint8_t* state,
                           const int32_t* pos2frame, const int32_t* done_iter, const int32_t* comp,
                           uint8_t* bits, float* soft, int32_t* out_iters, uint8_t* out_ok, int paper) {
    using A = typename Tr<MODE>::A;
    if (!comp[0]) return;
    __shared__ float tile[32][33];
    __shared__ int32_t fr[32];
    __shared__ int any;
    const int cur = comp[1];
    const int tj = (N + 31) / 32, tp = (cur + 31) / 32;
    for (long long tt = blockIdx.x; tt < (long long)tj * tp; tt += gridDim.x) {  // 32 x 32 tiles
        const int j0 = (int)(tt % tj) * 32, p0 = (int)(tt / tj) * 32;
        __syncthreads();  // the previous tile is written out
        if (threadIdx.x == 0 && threadIdx.y == 0) any = 0;
        __syncthreads();
        if (threadIdx.y == 0) {
            const int p = p0 + threadIdx.x;
            const int f = p < cur && state[p] == 0 ? pos2frame[p] : -1;  // stopped, in place
            fr[threadIdx.x] = f;
            if (f >= 0) {
                any = 1;
                if (j0 == 0) {
                    out_iters[f] = done_iter[f];
                    if (out_ok) out_ok[f] = 1;
                }
            }
        }
        __syncthreads();
        if (!any) continue;
        for (int y = threadIdx.y; y < 32; y += blockDim.y) {
            const int j = j0 + y, p = p0 + threadIdx.x;
            tile[y][threadIdx.x] = (j < N && p < cur) ? (float)s[(size_t)j * Fp + p] : 0.0f;
        }
        __syncthreads();
        for (int y = threadIdx.y; y < 32; y += blockDim.y) {
            const int f = fr[y], j = j0 + threadIdx.x;
            if (f >= 0 && j < N) {
                const float v = tile[threadIdx.x][y];  // exact for fp32 and int16 values
                const size_t idx = (size_t)f * N + j;
                bits[idx] = (uint8_t)slice((A)v, paper);
                if (soft) soft[idx] = (MODE == kModeFP32) ? v : v * 0.25f;
            }
        }
    }
}

// rows_deg / D (nullable): rows are padded-row slots, and slot i D + t with t >= deg(i)
// holds nothing (skipped).
template <typename E>
__global__ void __launch_bounds__(256) k_cmp_rows(E* arr, long long n_rows, int Fp,
                                                  const int32_t* __restrict__ new_pos,
                                                  const int32_t* comp, const uint8_t* rows_deg = nullptr,
                                                  int D = 1) {
    if (!comp[0]) return;
    constexpr int K = 8, CH = 256 * K;  // positions per chunk
    const int cur = comp[1];
    for (long long row = blockIdx.x; row < n_rows; row += gridDim.x) {
        if (rows_deg && (int)(row % D) >= __ldg(rows_deg + row / D)) continue;
        E* a = arr + row * Fp;
        for (int c0 = 0; c0 < cur; c0 += CH) {
            E v[K];
            int d[K];
#pragma unroll
            for (int q = 0; q < K; q++) {
                const int p = c0 + q * 256 + (int)threadIdx.x;
                d[q] = p < cur ? new_pos[p] : -1;
                if (d[q] >= 0) v[q] = a[p];
            }
            __syncthreads();  // the whole chunk is read before any of it is overwritten
#pragma unroll
            for (int q = 0; q < K; q++)
                if (d[q] >= 0) a[d[q]] = v[q];
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(kCmpThreads) k_cmp_tail(uint8_t* state, int32_t* pos2frame,
                                                          int32_t* comp) {
    if (!comp[0]) return;
    const int cur = comp[1], kept = comp[2];
    for (int p = threadIdx.x; p < cur; p += blockDim.x) {
        state[p] = p < kept;  // every frame moved to the front is running
        if (p >= kept) pos2frame[p] = -1;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        comp[0] = 0;
        comp[1] = kept;
    }
}

// llr [frames][N] (frame-major) -> r, s [N][Fp] (frame-interleaved). A block of 8 warps
// moves a tile of 32 frames x 128 bits: each warp reads frame rows (four coalesced 128-byte
// loads per row, sixteen per thread in flight), then writes bit rows of 32 frames; the
// shared tile is padded so that neither phase has bank conflicts.
constexpr int kLoadTJ = 128, kLoadTF = 32;
template <int MODE>
__global__ void __launch_bounds__(256) k_load(const void* llr, int llr_i8, int frames, int N,
                                              typename Tr<MODE>::R* r, typename Tr<MODE>::T* s, int Fp) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    __shared__ float tile[kLoadTF][kLoadTJ + 1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kLoadTJ, f0 = blockIdx.y * kLoadTF;
#pragma unroll
    for (int y = warp; y < kLoadTF; y += 8) {
        const int f = f0 + y;
#pragma unroll
        for (int q = 0; q < kLoadTJ / 32; q++) {
            const int j = j0 + q * 32 + lane;
            float v = 0.0f;
            if (f < frames && j < N) {
                const size_t idx = (size_t)f * N + j;
                v = llr_i8 ? (float)((const int8_t*)llr)[idx] : ((const float*)llr)[idx];
            }
            tile[y][q * 32 + lane] = v;
        }
    }
    __syncthreads();
#pragma unroll 4
    for (int c = warp; c < kLoadTJ; c += 8) {
        const int j = j0 + c, f = f0 + lane;
        if (j < N && f < Fp) {
            const float v = tile[lane][c];
            const size_t idx = (size_t)j * Fp + f;
            if (MODE == kModeFP32) {  // "+ 0.0f" turns -0.0 into +0.0, no other value
                r[idx] = (R)(v + 0.0f);
                s[idx] = (T)(v + 0.0f);
            } else {
                const int8_t q8 = llr_i8 ? (int8_t)v : quantize(v);
                r[idx] = (R)q8;
                s[idx] = (T)q8;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Check-node pass. Block = 4 warps = 4 rows; lane = one frame vector (V frames).
// MODE_SYN: syndrome only (final status pass), no message update.
// ------------------------------------------------------------------------------------
// Learned weights of one iteration: magnitude m of an edge whose bit has class c becomes
// max(fma(alpha[c], m, -beta[c]), 0).
struct IterWeights {
    const uint8_t* col_class;
    const float* alpha;
    const float* beta;
};

template <int MODE, bool FIRST, bool SYN_ONLY, bool W = false, int VW = Tr<MODE>::V>
__global__ void __launch_bounds__(128) k_check(const int32_t* __restrict__ row_ptr,
                                               const int32_t* __restrict__ col_idx, int M,
                                               const typename Tr<MODE>::T* __restrict__ s,
                                               typename Tr<MODE>::T* eta, int Fp,
                                               const uint8_t* __restrict__ state, uint8_t* unsat,
                                               int do_syn, const int* n_done, int frames,
                                               int paper, IterWeights wt = IterWeights()) {
    using T = typename Tr<MODE>::T;
    using A = typename Tr<MODE>::A;
    constexpr int V = VW;
    using VT = Vec<T, V>;
    using VS = Vec<uint8_t, V>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 4 + warp;
    const int f0 = (blockIdx.y * 32 + lane) * V;
    if (i >= M) return;
    if (*(volatile const int*)n_done >= frames) return;
    const VS st = *reinterpret_cast<const VS*>(state + f0);
    uint32_t act = 0;
#pragma unroll
    for (int v = 0; v < V; v++) act |= (uint32_t)(st.x[v] != 0) << v;
    if (!act) return;

    const int e0 = __ldg(row_ptr + i), d = __ldg(row_ptr + i + 1) - e0;
    A min0[V], min1[V];
    int loc[V];
    uint32_t msk[V];
    uint32_t neg = 0, z = 0;
#pragma unroll
    for (int v = 0; v < V; v++) {
        min0[v] = big(A());
        min1[v] = big(A());
        loc[v] = 0;
        msk[v] = 0;
    }
    const bool longrow = d > 32;
    for (int t = 0; t < d; t++) {
        const int c = __ldg(col_idx + e0 + t);
        const VT sv = *reinterpret_cast<const VT*>(s + (size_t)c * Fp + f0);
        VT ev;
        T* ep = eta + (size_t)(e0 + t) * Fp + f0;
        if (!FIRST && !SYN_ONLY) ev = *reinterpret_cast<const VT*>(ep);
        VT lv;
#pragma unroll
        for (int v = 0; v < V; v++) {
            const A sa = (A)sv.x[v];
            z ^= slice(sa, paper) << v;
            if (!SYN_ONLY) {
                const A lam = FIRST ? sa : lam_of(sa, (A)ev.x[v]);
                const A a = absval(lam);
                const uint32_t sg = lam < A(0);
                // Observation 1 without branches: a new minimum demotes min0 to min1 and
                // records its location (the first one: ties do not move it)
                const bool lt0 = a < min0[v];
                min1[v] = lt0 ? min0[v] : min(min1[v], a);
                min0[v] = lt0 ? a : min0[v];
                loc[v] = lt0 ? t : loc[v];
                neg ^= sg << v;
                msk[v] |= (sg << (t & 31));
                lv.x[v] = (T)lam;
            }
        }
        if (!SYN_ONLY && longrow) *reinterpret_cast<VT*>(ep) = lv;  // stash lambda in place
    }
    if (do_syn) flag_unsat<V>(unsat, f0, z & act);
    if constexpr (!SYN_ONLY) {
    for (int t = 0; t < d; t++) {
        T* ep = eta + (size_t)(e0 + t) * Fp + f0;
        VT lv;
        if (longrow) lv = *reinterpret_cast<const VT*>(ep);
        float wa = 1.0f, wb = 0.0f;
        if constexpr (W) {
            const int c = __ldg(wt.col_class + __ldg(col_idx + e0 + t));
            wa = __ldg(wt.alpha + c);
            wb = __ldg(wt.beta + c);
        }
        VT out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            const uint32_t sg = longrow ? (uint32_t)((A)lv.x[v] < A(0)) : ((msk[v] >> t) & 1u);
            A m = (t == loc[v]) ? min1[v] : min0[v];
            if constexpr (W) {
                const float x = __fmaf_rn(wa, (float)m, -wb);
                m = (A)(x > 0.0f ? x : 0.0f);
            }
            out.x[v] = (T)((((neg >> v) ^ sg) & 1u) ? -m : m);
        }
        *reinterpret_cast<VT*>(ep) = out;
    }
    }
}

// ------------------------------------------------------------------------------------
// Check-node pass on the padded row layout (rows of at most D edges; same block and lane
// mapping as k_check). Row i's columns and messages sit at slots i D .. i D + D - 1, so
// every load but the gather of s is issued at entry: the frame state, the degree and the
// columns together, then the old messages and the gathered s of the whole row, and only
// then the arithmetic. lambda stays in registers between the two sweeps; the new magnitude
// is min1 where |lambda| = min0 (Observation 1: on a tie min1 = min0, so the first
// location needs no tracking) and the sign is the XOR of the row's sign bits with the
// edge's own (Observation 2).
// Sign bits are read directly: FP32 s never holds -0.0 (k_load adds +0.0, and round-to-
// nearest sums and differences of values other than -0.0 are never -0.0), so the sign bit
// of lambda and of s is [v < 0]; the same holds for int32. Fixed point with an even
// number of frames per lane works on packed int16 pairs, exactly as per frame.
// ------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sbits(float x) { return __float_as_uint(x); }
__device__ __forceinline__ uint32_t sbits(int32_t x) { return (uint32_t)x; }
__device__ __forceinline__ float signed_mag(float m, uint32_t sgn) {  // m >= 0
    return __uint_as_float(__float_as_uint(m) | (sgn & 0x80000000u));
}
__device__ __forceinline__ int32_t signed_mag(int32_t m, uint32_t sgn) { return (int32_t)sgn < 0 ? -m : m; }

// Read-only (non-coherent) load of a 2-, 4-, 8- or 16-byte vector.
template <typename VT>
__device__ __forceinline__ VT ld_nc(const VT* p) {
    VT v;
    if constexpr (sizeof(VT) == 16) {
        const uint4 x = __ldg(reinterpret_cast<const uint4*>(p));
        memcpy(&v, &x, 16);
    } else if constexpr (sizeof(VT) == 8) {
        const uint2 x = __ldg(reinterpret_cast<const uint2*>(p));
        memcpy(&v, &x, 8);
    } else if constexpr (sizeof(VT) == 4) {
        const unsigned int x = __ldg(reinterpret_cast<const unsigned int*>(p));
        memcpy(&v, &x, 4);
    } else {
        static_assert(sizeof(VT) == 2, "2-, 4-, 8- or 16-byte vectors");
        const unsigned short x = __ldg(reinterpret_cast<const unsigned short*>(p));
        memcpy(&v, &x, 2);
    }
    return v;
}

template <int MODE, int VW>
struct RowVec {  // per-frame values
    using VT = Vec<typename Tr<MODE>::T, VW>;
    static constexpr bool kPacked = false;
};
template <int VW>
struct RowVec<kModeFixed, VW> {
    static constexpr bool kPacked = VW % 2 == 0;  // int16 pairs in 32-bit words
    using VT = typename std::conditional<kPacked, Words<(VW + 1) / 2>, Vec<int16_t, VW>>::type;
};

// Operands of a row update held in registers: sv[t], ev[t] = the gathered s and the old
// message of edge t; lambda replaces s in sv.
template <typename VT, int D>
struct RegRow {
    VT sv[D], ev[D];
    const int* cols;
    __device__ __forceinline__ VT s(int t) const { return sv[t]; }
    __device__ __forceinline__ VT e(int t) const { return ev[t]; }
    __device__ __forceinline__ void keep(int t, const VT& l) { sv[t] = l; }
    __device__ __forceinline__ VT lam(int t) const { return sv[t]; }
    // learned weights of edge t: through the class of its column
    __device__ __forceinline__ void weights(int t, const IterWeights& wt, float& wa, float& wb) const {
        const int cls = __ldg(wt.col_class + cols[t]);
        wa = __ldg(wt.alpha + cls);
        wb = __ldg(wt.beta + cls);
    }
};
// Operands in a shared-memory stage: chunk t holds s of edge t (lambda replaces it),
// chunk D + t the old message; this lane's vector sits at byte lane sizeof(VT).
template <typename VT, int D>
struct SmemRow {
    unsigned char* st;
    int chunk, lane;
    const int* cls;       // learned-weight class of each edge (shared memory)
    const float* walpha;  // weight tables of the iteration (shared memory)
    const float* wbeta;
    __device__ __forceinline__ VT* at(int c) const {
        return reinterpret_cast<VT*>(st + (size_t)c * chunk + (size_t)lane * sizeof(VT));
    }
    __device__ __forceinline__ VT s(int t) const { return *at(t); }
    __device__ __forceinline__ VT e(int t) const { return *at(D + t); }
    __device__ __forceinline__ void keep(int t, const VT& l) { *at(t) = l; }
    __device__ __forceinline__ VT lam(int t) const { return *at(t); }
    __device__ __forceinline__ void weights(int t, const IterWeights&, float& wa, float& wb) const {
        const int c = cls[t];
        wa = walpha[c];
        wb = wbeta[c];
    }
};

// The row update of one lane's VW frames over the d <= D edges of a row (Observation 1:
// min0, min1; Observation 2: XOR of sign bits): writes the new messages to erow + t Fp
// and returns the syndrome bits of the gathered s (bit v for frame v) when SYN.
template <int MODE, bool FIRST, bool SYN, bool PAPER, bool W, int VW, int D, class Row>
__device__ __forceinline__ uint32_t row_update(Row& row, int d, typename Tr<MODE>::T* erow, int Fp,
                                               const IterWeights& wt) {
    using T = typename Tr<MODE>::T;
    using A = typename Tr<MODE>::A;
    using RV = RowVec<MODE, VW>;
    using VT = typename RV::VT;
    uint32_t z = 0;
    if constexpr (!RV::kPacked) {
        A min0[VW], min1[VW];
        uint32_t sx[VW], zx[VW];
#pragma unroll
        for (int v = 0; v < VW; v++) {
            min0[v] = big(A());
            min1[v] = big(A());
            sx[v] = 0;
            zx[v] = 0;
        }
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (t >= d) break;  // d is the same for the whole warp: a branch, no idle slots
                const VT sv = row.s(t);
                VT ev;
                if (!FIRST) ev = row.e(t);
                VT lv;
#pragma unroll
                for (int v = 0; v < VW; v++) {
                    const A sa = (A)sv.x[v];
                    if (SYN) zx[v] ^= PAPER ? sbits(A(0) - sa) : sbits(sa);
                    const A l = FIRST ? sa : lam_of(sa, (A)ev.x[v]);
                    const A m = absval(l);
                    min1[v] = min(min1[v], max(min0[v], m));
                    min0[v] = min(min0[v], m);
                    sx[v] ^= sbits(l);
                    lv.x[v] = (T)l;  // exact: lambda is saturated to the storage range
                }
                row.keep(t, lv);
            }
        if (SYN) {
#pragma unroll
            for (int v = 0; v < VW; v++) z |= (zx[v] >> 31) << v;
        }
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (t >= d) break;  // d is the same for the whole warp: a branch, no idle slots
                float wa = 1.0f, wb = 0.0f;
                if constexpr (W) row.weights(t, wt, wa, wb);
                const VT lv = row.lam(t);
                VT out;
#pragma unroll
                for (int v = 0; v < VW; v++) {
                    const A l = (A)lv.x[v];
                    A m = absval(l) == min0[v] ? min1[v] : min0[v];
                    if constexpr (W) {  // max(fma(alpha, m, -beta), 0)
                        const float x = __fmaf_rn(wa, (float)m, -wb);
                        m = (A)(x > 0.0f ? x : 0.0f);
                    }
                    out.x[v] = (T)signed_mag(m, sbits(l) ^ sx[v]);
                }
                *reinterpret_cast<VT*>(erow + (size_t)t * Fp) = out;
            }
    } else {
        constexpr int P = VW / 2;
        uint32_t min0[P], min1[P], sx[P], zx[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            min0[p] = 0x7fff7fffu;
            min1[p] = 0x7fff7fffu;
            sx[p] = 0;
            zx[p] = 0;
        }
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (t >= d) break;  // d is the same for the whole warp: a branch, no idle slots
                const VT sv = row.s(t);
                VT ev;
                if (!FIRST) ev = row.e(t);
                VT lv;
#pragma unroll
                for (int p = 0; p < P; p++) {
                    const uint32_t sw = sv.w[p];
                    if (SYN) zx[p] ^= PAPER ? p_neg(sw) : sw;
                    const uint32_t l =
                        FIRST ? sw : p_pack_sat(p_sub_lo(p_acc_lo(0, sw), ev.w[p]), p_sub_hi(p_acc_hi(0, sw), ev.w[p]));
                    const uint32_t m = p_max(l, p_neg(l));
                    min1[p] = p_min(min1[p], p_max(min0[p], m));
                    min0[p] = p_min(min0[p], m);
                    sx[p] ^= l;
                    lv.w[p] = l;
                }
                row.keep(t, lv);
            }
        if (SYN) {
#pragma unroll
            for (int p = 0; p < P; p++) z |= (((zx[p] >> 15) & 1u) | ((zx[p] >> 30) & 2u)) << (2 * p);
        }
        PackedPick pk[P];
#pragma unroll
        for (int p = 0; p < P; p++) pk[p].set(min0[p], min1[p], sx[p]);
#pragma unroll
        for (int t = 0; t < D; t++) {
            if (t >= d) break;  // d is the same for the whole warp: a branch, no idle slots
                const VT lv = row.lam(t);
                VT out;
#pragma unroll
                for (int p = 0; p < P; p++) out.w[p] = pk[p](lv.w[p]);
                *reinterpret_cast<VT*>(erow + (size_t)t * Fp) = out;
            }
    }
    return z;
}

template <int MODE, bool FIRST, bool W, int VW, int D>
__global__ void __launch_bounds__(128, D <= 8 ? 4 : 2)
    k_check_ell(const int32_t* __restrict__ ell_col, const uint8_t* __restrict__ ell_deg, int M,
                const typename Tr<MODE>::T* __restrict__ s, typename Tr<MODE>::T* __restrict__ eta,
                int Fp, const uint8_t* __restrict__ state, uint8_t* __restrict__ unsat, int do_syn,
                int paper, IterWeights wt = IterWeights()) {
    using T = typename Tr<MODE>::T;
    using VT = typename RowVec<MODE, VW>::VT;
    using VS = Vec<uint8_t, VW>;
    static_assert(sizeof(VT) == sizeof(T) * VW, "one vector = VW frames");
    static_assert(D % 4 == 0, "columns load as 16-byte vectors");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 4 + warp;
    const int f0 = (blockIdx.y * 32 + lane) * VW;
    if (i >= M) return;
    const VS st = *reinterpret_cast<const VS*>(state + f0);
    const int d = __ldg(ell_deg + i);
    int c[D];
#pragma unroll
    for (int q = 0; q < D / 4; q++) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(ell_col + (size_t)i * D) + q);
        c[4 * q] = v.x;
        c[4 * q + 1] = v.y;
        c[4 * q + 2] = v.z;
        c[4 * q + 3] = v.w;
    }
    uint32_t act = 0;
#pragma unroll
    for (int v = 0; v < VW; v++) act |= (uint32_t)(st.x[v] != 0) << v;
    if (!act) return;

    T* const erow = eta + (size_t)i * D * Fp + f0;
    RegRow<VT, D> row;
    row.cols = c;
#pragma unroll
    for (int t = 0; t < D; t++)
        if (t < d) {
            row.sv[t] = ld_nc(reinterpret_cast<const VT*>(s + (size_t)c[t] * Fp + f0));
            if (!FIRST) row.ev[t] = *reinterpret_cast<const VT*>(erow + (size_t)t * Fp);
        }
    uint32_t z = 0;
    if (!do_syn) z = row_update<MODE, FIRST, false, false, W, VW, D>(row, d, erow, Fp, wt);
    else if (!paper) z = row_update<MODE, FIRST, true, false, W, VW, D>(row, d, erow, Fp, wt);
    else z = row_update<MODE, FIRST, true, true, W, VW, D>(row, d, erow, Fp, wt);
    if (do_syn) flag_unsat<VW>(unsat, f0, z & act);
}

// ------------------------------------------------------------------------------------
// Final syndrome pass on the padded row layout (status of frames that never stopped): the
// XOR of the decisions of a row's bits (eq. 1-2), every load of the row issued at once.
// ------------------------------------------------------------------------------------
template <int MODE, int VW, int D>
__global__ void __launch_bounds__(128) k_syn_ell(const int32_t* __restrict__ ell_col,
                                                 const uint8_t* __restrict__ ell_deg, int M,
                                                 const typename Tr<MODE>::T* __restrict__ s, int Fp,
                                                 const uint8_t* __restrict__ state,
                                                 uint8_t* __restrict__ unsat, int paper) {
    using A = typename Tr<MODE>::A;
    using VT = Vec<typename Tr<MODE>::T, VW>;
    using VS = Vec<uint8_t, VW>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int i = blockIdx.x * 4 + warp;
    const int f0 = (blockIdx.y * 32 + lane) * VW;
    if (i >= M) return;
    const VS st = *reinterpret_cast<const VS*>(state + f0);
    const int d = __ldg(ell_deg + i);
    int c[D];
#pragma unroll
    for (int q = 0; q < D / 4; q++) {
        const int4 v = __ldg(reinterpret_cast<const int4*>(ell_col + (size_t)i * D) + q);
        c[4 * q] = v.x;
        c[4 * q + 1] = v.y;
        c[4 * q + 2] = v.z;
        c[4 * q + 3] = v.w;
    }
    uint32_t act = 0;
#pragma unroll
    for (int v = 0; v < VW; v++) act |= (uint32_t)(st.x[v] != 0) << v;
    if (!act) return;
    VT sv[D];
#pragma unroll
    for (int t = 0; t < D; t++)
        if (t < d) sv[t] = ld_nc(reinterpret_cast<const VT*>(s + (size_t)c[t] * Fp + f0));
    uint32_t z = 0;
#pragma unroll
    for (int t = 0; t < D; t++)
        if (t < d) {
#pragma unroll
            for (int v = 0; v < VW; v++) z ^= slice((A)sv[t].x[v], paper) << v;
        }
    flag_unsat<VW>(unsat, f0, z & act);
}

// ------------------------------------------------------------------------------------
// Staged check pass (padded row layout): a persistent kernel in which every warp runs its
// own pipeline of S shared-memory stages. A task is one row of one frame block (32 lanes x
// VW frames); the warp's tasks are warp_id, warp_id + W_total, ... (rows fastest, so all
// warps work on the same frame block at a time and its s stays in L2). For the task of
// step k + S - 1 the warp's lanes issue bulk asynchronous copies (cp.async.bulk, the TMA
// engine's untiled form) of the row's gathered s chunks and old message chunks into stage
// (k + S - 1) mod S, completing on that stage's mbarrier, while it computes the task of
// step k from stage k mod S; the row data (degree, columns, frame state) of the task after
// that is loaded one step ahead. Shared memory, not registers, holds the bytes in flight.
// Every wait is bounded: on timeout the kernel records kErrTimeout in *err, waits (again
// bounded) for its own copies still in flight, and returns.
// ------------------------------------------------------------------------------------
// The row update on compressed messages (cmsg.cuh; FP32): the lane's VW frames of a row of
// d <= D edges, operands in a shared-memory stage (chunk t: s of edge t; chunks D, D + 1,
// D + 2: the row's old m0, m1, w). The old message of edge t is rebuilt from the old state
// (weighted with the previous iteration's weights, cls / walpha / wbeta), lambda = s - eta,
// and the new state (min0, min1, first location of min0, message signs) is written to
// cs at offset off; returns the syndrome bits of the gathered s when SYN.
template <bool FIRST, bool SYN, bool PAPER, bool W, int VW, int D>
__device__ __forceinline__ uint32_t row_update_cmp(const unsigned char* st, int chunk, int lane, int d,
                                                   const int* cls, const float* walpha,
                                                   const float* wbeta, const CState& cs, size_t off) {
    static_assert(D <= 16, "signs and locations of at most 16 edges fit the word");
    using VF = Vec<float, VW>;
    using VU = Vec<uint32_t, VW>;
    auto at = [&](int c) { return st + (size_t)c * chunk + (size_t)lane * sizeof(VF); };
    VF om0, om1;
    VU ow;
    if (!FIRST) {
        om0 = *reinterpret_cast<const VF*>(at(D));
        om1 = *reinterpret_cast<const VF*>(at(D + 1));
        ow = *reinterpret_cast<const VU*>(at(D + 2));
    }
    float min0[VW], min1[VW];
    uint32_t oh[VW], sg[VW], zx[VW];  // sg: lambda's sign bits, the first edge's highest
#pragma unroll
    for (int v = 0; v < VW; v++) {
        min0[v] = big(0.0f);
        min1[v] = big(0.0f);
        oh[v] = 0;
        sg[v] = 0;
        zx[v] = 0;
    }
#pragma unroll
    for (int t = 0; t < D; t++) {
        if (t >= d) break;  // d is the same for the whole warp: a branch, no idle slots
            const VF sv = *reinterpret_cast<const VF*>(at(t));
            float wa = 1.0f, wb = 0.0f;
            if constexpr (W && !FIRST) {
                const int c = cls[t];
                wa = walpha[c];
                wb = wbeta[c];
            }
#pragma unroll
            for (int v = 0; v < VW; v++) {
                const float sa = sv.x[v];
                if (SYN) zx[v] ^= PAPER ? sbits(0.0f - sa) : sbits(sa);
                float l = sa;
                if constexpr (!FIRST) {
                    float m = cmsg_mag(om0.x[v], om1.x[v], ow.x[v], t);
                    if constexpr (W) m = cmsg_weight(m, wa, wb);
                    l = sa - cmsg_signed(m, ow.x[v], t);
                }
                const float a = fabsf(l);
                const bool lt = a < min0[v];  // strict: the first location of min0 stays
                min1[v] = lt ? min0[v] : fminf(min1[v], a);
                min0[v] = lt ? a : min0[v];
                oh[v] = lt ? (1u << t) : oh[v];
                sg[v] = __funnelshift_l(sbits(l), sg[v], 1);  // (sg << 1) | sign of l
            }
        }
    uint32_t z = 0;
    if (SYN) {
#pragma unroll
        for (int v = 0; v < VW; v++) z |= (zx[v] >> 31) << v;
    }
    const uint32_t dmask = (1u << d) - 1u;  // d <= 16
    VF n0, n1;
    VU nw;
#pragma unroll
    for (int v = 0; v < VW; v++) {
        n0.x[v] = min0[v];
        n1.x[v] = min1[v];
        // message signs: the row's sign parity XOR each edge's own sign; edge t's sign sits
        // at bit d - 1 - t of sg, at bit 16 + t of the word (bit reversal, shift)
        const uint32_t sgt = __brev(sg[v]) >> (16 - d);
        nw.x[v] = oh[v] | ((sgt ^ ((__popc(sg[v]) & 1u) ? dmask << 16 : 0u)));
    }
    *reinterpret_cast<VF*>(cs.m0 + off) = n0;
    *reinterpret_cast<VF*>(cs.m1 + off) = n1;
    *reinterpret_cast<VU*>(cs.w + off) = nw;
    return z;
}

constexpr int kErrTimeout = 1;
constexpr uint32_t kDrainTries = 1u << 16;  // about 1.3 s at most

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// One try of at most about 20 us (the suspend-time hint) for the phase of the parity.
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase of the given parity; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t limit) {
    for (uint32_t n = 0; n < limit; n++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// L2 eviction policies: the gathered posteriors are read by about d_v rows of the frame
// block being swept (keep them), the messages are read once per pass (let them go first).
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
// Global -> shared bulk copy of `bytes` (a multiple of 16; both addresses 16-byte
// aligned) under an L2 cache policy, completing `bytes` transactions on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t policy) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}

struct StagedArgs {
    const int32_t* ell_col;
    const uint8_t* ell_deg;
    const uint8_t* ell_cls;  // learned-weight class of each slot
    int M, Fp, n_fblocks, stages, paper, n_classes;
    uint32_t wait_limit;
    const uint8_t* state;
    uint8_t* unsat;
    int32_t* err;
    const int32_t* comp;  // [1]: positions in use (frame blocks behind them get no task)
};

// Shared memory of one warp: S stages of [D s chunks][D message chunks], each chunk
// 32 VW sizeof(T) bytes; then per stage one 32-bit word per lane (degree << 8 | frame
// mask) and D learned-weight classes; then S mbarriers. With learned weights the CTA's
// copy of the iteration's alpha and beta tables (256 entries each) follows.
template <int MODE, int VW, int D, bool CMP = false>
struct StagedLayout {
    static constexpr int kChunk = 32 * VW * (int)sizeof(typename Tr<MODE>::T);
    // per-edge messages: D s chunks and D message chunks; compressed: D s chunks and the
    // row's three state chunks
    static constexpr int kStage = (CMP ? D + 3 : 2 * D) * kChunk;
    static constexpr int kMeta = 32 * 4 + D * 4;
    __host__ __device__ static constexpr size_t warp_bytes(int S) {
        return (size_t)S * (kStage + kMeta + 8);
    }
    static constexpr int kWeightBytes = 2 * 256 * 4;
};

constexpr int kStagedMaxThreads = 384;

// SYN: test the syndrome of the gathered s (the decision of the previous iteration).
// SYN_ONLY: the final syndrome pass (with FIRST: s copies only, no message update).
// CMP (FP32 only): the messages are compressed (cmsg.cuh): eta points at the row states,
// each task copies the row's old state (three chunks) instead of its old messages, and
// writes the new state; the weights given are the previous iteration's (they rebuild the
// old messages; the new state holds unweighted minima).
template <int MODE, bool FIRST, bool SYN, bool W, int VW, int D, bool SYN_ONLY = false, bool CMP = false>
__global__ void __launch_bounds__(kStagedMaxThreads) k_check_staged(const StagedArgs a,
                                                      const typename Tr<MODE>::T* __restrict__ s,
                                                      typename Tr<MODE>::T* __restrict__ eta,
                                                      IterWeights wt) {
    using T = typename Tr<MODE>::T;
    using VT = typename RowVec<MODE, VW>::VT;
    using VS = Vec<uint8_t, VW>;
    using LY = StagedLayout<MODE, VW, D, CMP>;
    static_assert(LY::kChunk % 16 == 0, "bulk copies move multiples of 16 bytes");
    extern __shared__ __align__(128) unsigned char smem_st[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int S = a.stages, M = a.M;
    // the frame blocks in use: after a frame compaction the running frames sit at the front
    const int NB = min(a.n_fblocks, (__ldcg(a.comp + 1) + 32 * VW - 1) / (32 * VW));
    unsigned char* const buf = smem_st + (size_t)warp * S * LY::kStage;
    unsigned char* const meta = smem_st + (size_t)nw * S * LY::kStage + (size_t)warp * S * LY::kMeta;
    uint64_t* const bar = reinterpret_cast<uint64_t*>(smem_st + (size_t)nw * S * (LY::kStage + LY::kMeta)) +
                          (size_t)warp * S;
    float* const walpha = reinterpret_cast<float*>(smem_st + (size_t)nw * LY::warp_bytes(S));
    float* const wbeta = walpha + 256;
    if constexpr (W) {  // the iteration's weight tables, shared by the CTA
        for (int c = threadIdx.x; c < a.n_classes; c += blockDim.x) {
            walpha[c] = __ldg(wt.alpha + c);
            wbeta[c] = __ldg(wt.beta + c);
        }
        __syncthreads();
    }
    if (lane == 0)
        for (int q = 0; q < S; q++) mbar_init(&bar[q], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    __syncwarp();

    // tasks first, first + stride, ... with task = y M + i (row i of frame block y); the
    // host guarantees M NB + stride < 2^31. (i, y) advance without a division per task.
    const int first = blockIdx.x * nw + warp, stride = gridDim.x * nw;
    const int di = stride % M, dy = stride / M;
    const int FB = 32 * VW;  // frames per block
    static_assert(!CMP || MODE == kModeFP32, "compressed messages are FP32");
    const uint32_t tx = (FIRST || CMP ? 1u : 2u) * (uint32_t)LY::kChunk;  // per edge
    const uint32_t tx_row = (CMP && !FIRST) ? 3u * (uint32_t)LY::kChunk : 0u;  // per row
    const CState cs = CMP ? cstate_at(eta, M, a.Fp) : CState{};
    int ci = first % M, cy = first / M;  // the task being computed
    int ni = ci, ny = cy;                // the next task to issue
    int nx_d = 0, nx_c = 0, nx_cls = 0;  // its row data, loaded one step ahead
    uint32_t nx_act = 0;
    uint32_t pend = 0, phase = 0;        // per stage: copies in flight / parity awaited
    uint32_t zacc = 0;                   // syndrome bits of this lane's frames, this frame block
    const uint64_t keep_s = policy_evict_last(), drop_eta = policy_evict_first();

    auto load_row = [&]() {
        if (ny >= NB) return;
        nx_d = __ldg(a.ell_deg + ni);
        nx_c = lane < D ? __ldg(a.ell_col + (size_t)ni * D + lane) : 0;
        if (W) nx_cls = lane < D ? __ldg(a.ell_cls + (size_t)ni * D + lane) : 0;
        const VS st = *reinterpret_cast<const VS*>(a.state + (size_t)ny * FB + lane * VW);
        uint32_t m = 0;
#pragma unroll
        for (int v = 0; v < VW; v++) m |= (uint32_t)(st.x[v] != 0) << v;
        nx_act = m;
    };
    // issue the copies of the next task into stage q and move on to the task after it; a
    // frame block with no active frame gets no copies (its phase completes at once)
    auto issue = [&](int q) {
        if (ny >= NB) return;
        const int d = nx_d;
        const bool any = __ballot_sync(0xffffffffu, nx_act != 0) != 0;
        reinterpret_cast<uint32_t*>(meta + (size_t)q * LY::kMeta)[lane] =
            ((uint32_t)d << 8) | (any ? nx_act : 0u);
        if (W && lane < D) reinterpret_cast<int*>(meta + (size_t)q * LY::kMeta + 128)[lane] = nx_cls;
        // the generic-proxy reads of this stage (its previous task) precede the copies
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive_expect_tx(&bar[q], any ? tx * (uint32_t)d + tx_row : 0u);
        __syncwarp();
        if (any && lane < d) {
            unsigned char* st = buf + (size_t)q * LY::kStage;
            const size_t fo = (size_t)ny * FB;
            bulk_g2s(st + (size_t)lane * LY::kChunk, s + (size_t)nx_c * a.Fp + fo, LY::kChunk, &bar[q],
                     keep_s);
            if (!FIRST && !CMP)
                bulk_g2s(st + (size_t)(D + lane) * LY::kChunk, eta + ((size_t)ni * D + lane) * a.Fp + fo,
                         LY::kChunk, &bar[q], drop_eta);
        }
        if (CMP && !FIRST && any && lane >= D && lane < D + 3) {  // the row's old state
            unsigned char* st = buf + (size_t)q * LY::kStage;
            const int c = lane - D;
            const float* src = c == 0 ? cs.m0 : c == 1 ? cs.m1 : reinterpret_cast<const float*>(cs.w);
            bulk_g2s(st + (size_t)lane * LY::kChunk, src + (size_t)ni * a.Fp + (size_t)ny * FB, LY::kChunk,
                     &bar[q], drop_eta);
        }
        pend |= 1u << q;
        ni += di;
        ny += dy;
        if (ni >= M) {
            ni -= M;
            ny++;
        }
        load_row();
    };

    load_row();
    for (int q = 0; q < S; q++) issue(q);
    for (int q = 0; cy < NB; q = (q + 1 == S) ? 0 : q + 1) {
        const uint32_t par = (phase >> q) & 1u;
        // the warp agrees on the outcome, so that it leaves or stays together
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[q], par, a.wait_limit))) {
            if (lane == 0) atomicExch(a.err, kErrTimeout);
            for (int j = 0; j < S; j++)  // let the copies in flight land (bounded)
                if ((pend >> j) & 1u) mbar_wait(&bar[j], (phase >> j) & 1u, kDrainTries);
            return;
        }
        phase ^= 1u << q;
        pend &= ~(1u << q);
        const uint32_t mw = reinterpret_cast<const uint32_t*>(meta + (size_t)q * LY::kMeta)[lane];
        const uint32_t act = mw & 0xffu;
        const int d = (int)(mw >> 8);
        unsigned char* const st = buf + (size_t)q * LY::kStage;
        if (SYN_ONLY && act) {  // XOR of the decisions of the row's bits
            using A = typename Tr<MODE>::A;
            using VP = Vec<T, VW>;
            uint32_t z = 0;
#pragma unroll
            for (int t = 0; t < D; t++)
                if (t < d) {
                    const VP sv = *reinterpret_cast<const VP*>(st + (size_t)t * LY::kChunk + lane * sizeof(VP));
#pragma unroll
                    for (int v = 0; v < VW; v++) z ^= slice((A)sv.x[v], a.paper) << v;
                }
            zacc |= z & act;
        } else if (act) {
            if constexpr (CMP) {
                const int* cls = reinterpret_cast<const int*>(meta + (size_t)q * LY::kMeta + 128);
                const size_t off = (size_t)ci * a.Fp + (size_t)cy * FB + lane * VW;
                if constexpr (SYN) {
                    const uint32_t z =
                        a.paper ? row_update_cmp<FIRST, true, true, W, VW, D>(st, LY::kChunk, lane, d, cls, walpha, wbeta, cs, off)
                                : row_update_cmp<FIRST, true, false, W, VW, D>(st, LY::kChunk, lane, d, cls, walpha, wbeta, cs, off);
                    zacc |= z & act;
                } else {
                    row_update_cmp<FIRST, false, false, W, VW, D>(st, LY::kChunk, lane, d, cls, walpha, wbeta, cs, off);
                }
            } else {
                const int f0 = cy * FB + lane * VW;
                SmemRow<VT, D> row{st, LY::kChunk, lane,
                                   reinterpret_cast<const int*>(meta + (size_t)q * LY::kMeta + 128), walpha,
                                   wbeta};
                T* const erow = eta + (size_t)ci * D * a.Fp + f0;
                if constexpr (SYN) {
                    const uint32_t z = a.paper ? row_update<MODE, FIRST, true, true, W, VW, D>(row, d, erow, a.Fp, wt)
                                               : row_update<MODE, FIRST, true, false, W, VW, D>(row, d, erow, a.Fp, wt);
                    zacc |= z & act;
                } else {
                    row_update<MODE, FIRST, false, false, W, VW, D>(row, d, erow, a.Fp, wt);
                }
            }
        }
        __syncwarp();
        issue(q);  // the task S steps ahead into the stage just read
        const int py = cy;
        ci += di;
        cy += dy;
        if (ci >= M) {
            ci -= M;
            cy++;
        }
        if ((SYN || SYN_ONLY) && cy != py) {  // the warp's rows of this frame block are done
            flag_unsat<VW>(a.unsat, py * FB + lane * VW, zacc);
            zacc = 0;
        }
    }
}

// ------------------------------------------------------------------------------------
// Variable-node pass. Block = 4 warps = 4 columns; lane = one frame vector.
// test_prev: the previous decision's syndrome (in unsat) decides whether a frame stops.
// CMP (FP32): the messages are compressed (cmsg.cuh): col_edge holds padded-row slots
// i 2^dshift + t, and the message of each edge is rebuilt from row i's state cs, weighted
// (W) with this iteration's weights of the column's class.
// HD (the last iteration, 4 or 8 frames per lane): each lane also writes the decisions of
// its frames as one byte, bit v = frame f0 + v, to hd[j][Fp / VW] (byte f0 / VW), for the
// final syndrome and the output bits (k_syn_hd, k_store_hd). Only lanes that update
// their frames write: the other bytes belong to frames whose status is already known.
// ------------------------------------------------------------------------------------
// The pass is bound by the latency of its gathers (index, then message or row state), not
// by bandwidth: it runs at 16 blocks of 128 threads per SM (all 64 warps, at most 32
// registers), which measured faster than fewer, larger-register warps (N=64800 FP32 with
// compressed messages: 102 -> 96.5 ms per 4096-frame, 50-iteration decode).
// One task: column j for the V frames at positions f0 .. f0 + V - 1.
template <int MODE, int VW, bool CMP, bool W, bool HD>
__device__ __forceinline__ void var_task(int j, int f0, const int32_t* __restrict__ col_ptr,
                                         const int32_t* __restrict__ col_edge,
                                         const typename Tr<MODE>::R* __restrict__ r,
                                         typename Tr<MODE>::T* s,
                                         const typename Tr<MODE>::T* __restrict__ eta, int Fp,
                                         uint8_t* state, int32_t* done_iter,
                                         const int32_t* __restrict__ pos2frame,
                                         const uint8_t* __restrict__ unsat, int test_prev, int k,
                                         int* n_done, const CState& cs, int dshift,
                                         const IterWeights& wt, uint8_t* hd, int paper) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    using A = typename Tr<MODE>::A;
    constexpr int V = VW;
    using VT = Vec<T, V>;
    using VR = Vec<R, V>;
    using VS = Vec<uint8_t, V>;
    const VS st = *reinterpret_cast<const VS*>(state + f0);
    uint32_t act = 0;
#pragma unroll
    for (int v = 0; v < V; v++) act |= (uint32_t)(st.x[v] != 0) << v;
    if (!act) return;
    uint32_t upd = act;
    if (test_prev) {
        const VS un = *reinterpret_cast<const VS*>(unsat + f0);
        uint32_t conv = 0;
#pragma unroll
        for (int v = 0; v < V; v++) conv |= (uint32_t)(un.x[v] == 0) << v;
        conv &= act;
        upd = act & ~conv;
        if (j == 0 && conv) {  // one designated thread per frame records the stop
#pragma unroll
            for (int v = 0; v < V; v++)
                if ((conv >> v) & 1) {
                    done_iter[pos2frame[f0 + v]] = k - 1;
                    state[f0 + v] = 0;
                    atomicAdd(n_done, 1);
                }
        }
    }
    if (!upd) return;
    const int t0 = __ldg(col_ptr + j), t1 = __ldg(col_ptr + j + 1);
    const VR rv = *reinterpret_cast<const VR*>(r + (size_t)j * Fp + f0);
    A acc[V];
#pragma unroll
    for (int v = 0; v < V; v++) acc[v] = (A)rv.x[v];
    if constexpr (CMP) {
        static_assert(MODE == kModeFP32, "compressed messages are FP32");
        using VF = Vec<float, V>;
        using VU = Vec<uint32_t, V>;
        float wa = 1.0f, wb = 0.0f;
        if constexpr (W) {
            const int c = __ldg(wt.col_class + j);
            wa = __ldg(wt.alpha + c);
            wb = __ldg(wt.beta + c);
        }
        const int tmask = (1 << dshift) - 1;
        // Not unrolled: at the 32-register bound each further edge in flight (three 16-byte
        // row-state loads) spilled, and the spills cost 4 % of the whole decode.
#pragma unroll 1
        for (int t = t0; t < t1; t++) {
            const int slot = __ldg(col_edge + t);
            const size_t o = (size_t)(slot >> dshift) * Fp + f0;
            const int tp = slot & tmask;
            const VF m0 = ld_nc(reinterpret_cast<const VF*>(cs.m0 + o));
            const VF m1 = ld_nc(reinterpret_cast<const VF*>(cs.m1 + o));
            const VU w = ld_nc(reinterpret_cast<const VU*>(cs.w + o));
#pragma unroll
            for (int v = 0; v < V; v++) {
                float m = cmsg_mag(m0.x[v], m1.x[v], w.x[v], tp);
                if constexpr (W) m = cmsg_weight(m, wa, wb);
                acc[v] = acc[v] + (A)cmsg_signed(m, w.x[v], tp);
            }
        }
    } else if constexpr (MODE == kModeFixed && V % 2 == 0) {
        // int16 pairs: each lane of a word added by one two-way dot product (dp2a)
        using VW32 = Words<V / 2>;
        for (int t = t0; t < t1; t++) {
            const int e = __ldg(col_edge + t);
            const VW32 ev = *reinterpret_cast<const VW32*>(eta + (size_t)e * Fp + f0);
#pragma unroll
            for (int p = 0; p < V / 2; p++) {
                acc[2 * p] = p_acc_lo(acc[2 * p], ev.w[p]);
                acc[2 * p + 1] = p_acc_hi(acc[2 * p + 1], ev.w[p]);
            }
        }
    } else {
        for (int t = t0; t < t1; t++) {
            const int e = __ldg(col_edge + t);
            const VT ev = *reinterpret_cast<const VT*>(eta + (size_t)e * Fp + f0);
#pragma unroll
            for (int v = 0; v < V; v++) acc[v] = acc[v] + (A)ev.x[v];
        }
    }
    if constexpr (HD) {
        static_assert(V == 4 || V == 8, "one byte of decisions per lane");
        uint32_t b = 0;
#pragma unroll
        for (int v = 0; v < V; v++) b |= slice(acc[v], paper) << v;  // the sign survives sat16
        hd[(size_t)j * (Fp / V) + f0 / V] = (uint8_t)b;
    }
    T* sp = s + (size_t)j * Fp + f0;
    if (upd == (1u << V) - 1u) {
        if constexpr (MODE == kModeFixed && V % 2 == 0) {  // saturated and packed in pairs
            Words<V / 2> out;
#pragma unroll
            for (int p = 0; p < V / 2; p++) out.w[p] = p_pack_sat((int32_t)acc[2 * p], (int32_t)acc[2 * p + 1]);
            *reinterpret_cast<Words<V / 2>*>(sp) = out;
        } else {
            VT out;
#pragma unroll
            for (int v = 0; v < V; v++) {
                if (MODE == kModeFP32) out.x[v] = (T)acc[v];
                else out.x[v] = (T)sat16((int32_t)acc[v]);
            }
            *reinterpret_cast<VT*>(sp) = out;
        }
    } else {
#pragma unroll
        for (int v = 0; v < V; v++)
            if ((upd >> v) & 1) sp[v] = (MODE == kModeFP32) ? (T)acc[v] : (T)sat16((int32_t)acc[v]);
    }
}

// The bit pass over the positions in use (comp[1]: after a frame compaction the running
// frames sit at the front): tasks t = y G + c, column group c (4 columns, one per warp) of
// frame block y (32 lanes x V frames).
// Fixed point: a grid of at most as many CTAs as fit the GPU at once takes the tasks in
// steps of the grid size, so frame blocks behind the positions in use get no CTA at all
// (and no CTA is retired and started per task: 7 % faster on the N=64800 code).
// FP32: one CTA per task (grid G x frame blocks), which the hardware starts in task order,
// and a CTA behind the positions in use returns at once. With compressed messages the
// gathered row states of a frame block are then reused in L2 by the CTAs running together
// (CTAs that loop over strided tasks drift apart: 20 % slower on the N=64800 code); with
// per-edge messages the looping form measured 1.7 % slower on the QC N=2304 code.
template <int MODE, int VW = Tr<MODE>::V, bool CMP = false, bool W = false, bool HD = false>
__global__ void __launch_bounds__(128, 16) k_var(const int32_t* __restrict__ col_ptr,
                                             const int32_t* __restrict__ col_edge, int N,
                                             const typename Tr<MODE>::R* __restrict__ r,
                                             typename Tr<MODE>::T* s,
                                             const typename Tr<MODE>::T* __restrict__ eta, int Fp,
                                             uint8_t* state, int32_t* done_iter,
                                             const int32_t* __restrict__ pos2frame,
                                             const uint8_t* __restrict__ unsat, int test_prev,
                                             int k, int* n_done, int frames, const int32_t* comp,
                                             CState cs = CState{}, int dshift = 0,
                                             IterWeights wt = IterWeights(), uint8_t* hd = nullptr,
                                             int paper = 0) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int FB = 32 * VW;
    if constexpr (MODE == kModeFP32) {
        const int j = blockIdx.x * 4 + warp, y = blockIdx.y;
        const int cur = __ldcg(comp + 1), done = *(volatile const int*)n_done;  // one round trip
        if (j >= N || y * FB >= cur || done >= frames) return;
        var_task<MODE, VW, CMP, W, HD>(j, (y * 32 + lane) * VW, col_ptr, col_edge, r, s, eta, Fp, state,
                                       done_iter, pos2frame, unsat, test_prev, k, n_done, cs, dshift, wt,
                                       hd, paper);
        return;
    }
    if (*(volatile const int*)n_done >= frames) return;
    const int nb = min(Fp / FB, (__ldcg(comp + 1) + FB - 1) / FB);
    const int G = (N + 3) / 4;
    const int step_y = (int)(gridDim.x / G), step_c = (int)(gridDim.x % G);
    int y = (int)(blockIdx.x / G), c = (int)(blockIdx.x % G);
    for (; y < nb;) {
        const int j = c * 4 + warp;
        if (j < N)
            var_task<MODE, VW, CMP, W, HD>(j, (y * 32 + lane) * VW, col_ptr, col_edge, r, s, eta, Fp, state,
                                           done_iter, pos2frame, unsat, test_prev, k, n_done, cs, dshift,
                                           wt, hd, paper);
        y += step_y;
        c += step_c;
        if (c >= G) {
            c -= G;
            y++;
        }
    }
}

// s [N][Fp] (by position) -> bits (and soft) [frames][N] (by frame). A block of 8 warps
// moves a tile of 128 bits x 32 positions: each warp reads bit rows (32 positions, one
// coalesced load), then writes frame rows of 128 decisions (four 32-byte stores per row).
constexpr int kStoreTJ = 128, kStoreTF = 32;
template <int MODE>
__global__ void __launch_bounds__(256) k_store(const typename Tr<MODE>::T* s, int Fp, int N,
                                               const int32_t* pos2frame, const int32_t* comp,
                                               uint8_t* bits, float* soft, int paper) {
    using A = typename Tr<MODE>::A;
    __shared__ float tile[kStoreTJ][kStoreTF + 1];
    __shared__ int32_t fr[kStoreTF];
    const int cur = comp[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j0 = blockIdx.x * kStoreTJ, p0 = blockIdx.y * kStoreTF;
    if (p0 >= cur) return;
    if (warp == 0) {
        const int p = p0 + lane;
        fr[lane] = p < cur ? pos2frame[p] : -1;
    }
#pragma unroll 4
    for (int c = warp; c < kStoreTJ; c += 8) {
        const int j = j0 + c, p = p0 + lane;
        tile[c][lane] = (j < N && p < cur) ? (float)s[(size_t)j * Fp + p] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int y = warp; y < kStoreTF; y += 8) {
        const int f = fr[y];
        if (f < 0) continue;
#pragma unroll
        for (int q = 0; q < kStoreTJ / 32; q++) {
            const int j = j0 + q * 32 + lane;
            if (j < N) {
                const float v = tile[q * 32 + lane][y];  // exact for fp32 and int16 values
                const size_t idx = (size_t)f * N + j;
                bits[idx] = (uint8_t)slice((A)v, paper);
                if (soft) soft[idx] = (MODE == kModeFP32) ? v : v * 0.25f;
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Decisions of the last bit pass, packed (HD variant of k_var): hd[j][Fp / VW] bytes, bit v
// of byte g = the decision at position g VW + v. A 32-bit word u of a row of hd holds
// positions 4 u VW + q, q = k VW + v at bit 8 k + v (the upper nibbles stay 0 when VW = 4).
// ------------------------------------------------------------------------------------
// Final syndrome (eq. 1-2) from the packed decisions: a thread XORs the words of a row's
// bits for kSynRows rows in a row. The 8 warps of a block take 8 runs of rows over the same
// 32 words of hd (blockIdx.y), OR their failure words in shared memory, and one warp sets
// the failing positions in the bit array ubits (bit p of word p / 32 = position p fails;
// cleared beforehand), reading each word first so that the atomic is skipped once its bits
// are set: every block reports to the same few words. A warp reads 32 consecutive words of
// one row of hd: 128 bytes, mostly from L2 (the decisions of 4096 frames of N=64800 bits
// take 33 MB).
constexpr int kSynRows = 8;
template <int VW, int D>
__global__ void __launch_bounds__(256) k_syn_hd(const int32_t* __restrict__ ell_col,
                                                const uint8_t* __restrict__ ell_deg, int M,
                                                const uint8_t* __restrict__ hd, int Fp,
                                                uint32_t* __restrict__ ubits) {
    __shared__ uint32_t red[8][32];
    const int nw = Fp / (4 * VW);  // words per row of hd
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int run = blockIdx.x * 8 + warp, u = blockIdx.y * 32 + lane;
    const int i0 = run * kSynRows;
    uint32_t fail = 0;
    if (i0 < M && u < nw) {
        const uint32_t* hw = reinterpret_cast<const uint32_t*>(hd) + u;
        const int i1 = min(M, i0 + kSynRows);
        for (int i = i0; i < i1; i++) {
            const int d = __ldg(ell_deg + i);
            int c[D];
#pragma unroll
            for (int q = 0; q < D / 4; q++) {
                const int4 v = __ldg(reinterpret_cast<const int4*>(ell_col + (size_t)i * D) + q);
                c[4 * q] = v.x;
                c[4 * q + 1] = v.y;
                c[4 * q + 2] = v.z;
                c[4 * q + 3] = v.w;
            }
            uint32_t z = 0;
#pragma unroll
            for (int t = 0; t < D; t++) {
                if (t >= d) break;
                z ^= __ldg(hw + (size_t)c[t] * nw);
            }
            fail |= z;
        }
    }
    red[warp][lane] = fail;
    __syncthreads();
    if (warp != 0 || u >= nw) return;
    uint32_t f = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) f |= red[k][lane];
    // word u covers positions 4 u VW + 8 k + v (bit 8 k + v, v < VW): to position bits
    uint32_t bits = f;
    int word = u, shift = 0;
    if constexpr (VW == 4) {
        bits = 0;
#pragma unroll
        for (int k = 0; k < 4; k++) bits |= ((f >> (8 * k)) & 15u) << (4 * k);
        word = u >> 1;
        shift = 16 * (u & 1);
    }
    bits <<= shift;
    if (bits && (((volatile const uint32_t*)ubits)[word] & bits) != bits) atomicOr(ubits + word, bits);
}

// Output bits from the packed decisions (no soft output, and every position in use was
// updated by the last bit pass: no early stop). A warp takes 32 bits j (lane = bit) and
// four words of hd: each lane loads 16 bytes of its bit's row, and one ballot per position
// gives the decisions of the 32 bits at that position (a 32 x 32 bit transpose); the lane
// of that position then writes them as 32 bytes of its frame's row of `bits`.
template <int VW>
__global__ void __launch_bounds__(256) k_store_hd(const uint8_t* __restrict__ hd, int Fp, int N,
                                                  const int32_t* __restrict__ pos2frame,
                                                  const int32_t* __restrict__ comp, uint8_t* __restrict__ bits) {
    constexpr int PW = 4 * VW;    // positions per word
    constexpr int WPB = 32 / PW;  // words per 32 positions
    const int nw = Fp / PW;
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * 8 + (threadIdx.x >> 5);
    const int nq = nw / 4;  // groups of 4 words
    const int jt = gw / nq, u0 = (gw - jt * nq) * 4;
    const int j0 = jt * 32;
    if (j0 >= N) return;  // warp-uniform
    const int cur = comp[1];
    if (u0 * PW >= cur) return;  // warp-uniform: no position in use
    const int j = j0 + lane;
    uint4 w4 = make_uint4(0u, 0u, 0u, 0u);
    if (j < N) w4 = __ldg(reinterpret_cast<const uint4*>(hd + (size_t)j * (Fp / VW)) + u0 / 4);
    const uint32_t words[4] = {w4.x, w4.y, w4.z, w4.w};
    const bool vec = (N & 15) == 0 && j0 + 32 <= N && ((uintptr_t)bits & 15) == 0;
#pragma unroll
    for (int bt = 0; bt < 4 / WPB; bt++) {  // 32 positions at a time
        uint32_t mine = 0;
#pragma unroll
        for (int x = 0; x < WPB; x++) {
#pragma unroll
            for (int q = 0; q < PW; q++) {
                const uint32_t m = __ballot_sync(0xffffffffu, (words[bt * WPB + x] >> ((q / VW) * 8 + q % VW)) & 1u);
                if (lane == x * PW + q) mine = m;
            }
        }
        const int p = (u0 + bt * WPB) * PW + lane;
        if (p >= cur) continue;
        const int f = pos2frame[p];
        if (f < 0) continue;
        uint8_t* dst = bits + (size_t)f * N + j0;
        if (vec) {  // 16-byte aligned: bits, N and j0 are
            uint32_t o[8];
#pragma unroll
            for (int k = 0; k < 8; k++) o[k] = (((mine >> (4 * k)) & 15u) * 0x00204081u) & 0x01010101u;
            reinterpret_cast<uint4*>(dst)[0] = make_uint4(o[0], o[1], o[2], o[3]);
            reinterpret_cast<uint4*>(dst)[1] = make_uint4(o[4], o[5], o[6], o[7]);
        } else {
            for (int k = 0; k < 32 && j0 + k < N; k++) dst[k] = (uint8_t)((mine >> k) & 1u);
        }
    }
}

// Status of the frames in the final layout (positions in use).
// ubits (nullable): the final syndrome as a bit array (k_syn_hd) instead of unsat_final.
__global__ void k_finish(const int32_t* done_iter, const int32_t* pos2frame, const int32_t* comp,
                         const uint8_t* unsat_final, int Fp, int L, int32_t* out_iters,
                         uint8_t* out_ok, const uint32_t* ubits = nullptr) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= Fp || p >= comp[1]) return;
    const int f = pos2frame[p];
    if (f < 0) return;
    const int d = done_iter[f];
    out_iters[f] = d >= 0 ? d : L;
    const int fails = ubits ? (int)((ubits[p >> 5] >> (p & 31)) & 1u) : (unsat_final[p] != 0);
    if (out_ok) out_ok[f] = d >= 0 ? 1 : !fails;
}

// Launch of the staged check pass; false when the shape does not fit the device or the
// task count does not fit 32 bits (the caller then runs the unstaged kernel).
template <int MODE, int V, bool FIRST, bool W, int D, bool SYN_ONLY = false, bool CMP = false>
bool launch_staged(const DevGraph& g, const DecodeArgs& a, const StreamWork& w,
                   const typename Tr<MODE>::T* s, typename Tr<MODE>::T* eta, uint8_t* un,
                   int test_prev, const IterWeights& wt, cudaStream_t st) {
    if (w.stages <= 0 || w.stage_warps <= 0 || w.num_sms <= 0 || !w.err) return false;
    using LY = StagedLayout<MODE, V, D, CMP>;
    const int threads = 32 * w.stage_warps;
    if (threads > kStagedMaxThreads) return false;
    const size_t smem = staged_smem_bytes(MODE, V, D, CMP, w.stage_warps, w.stages, W);
    static_assert(LY::kStage + LY::kMeta + 8 == (CMP ? D + 3 : 2 * D) * LY::kChunk + 32 * 4 + D * 4 + 8,
                  "the kernel's layout is the one staged_smem_bytes sizes");
    if (W && a.n_classes > 256) return false;
    auto kern = SYN_ONLY ? k_check_staged<MODE, true, false, false, V, D, true>
                : test_prev ? k_check_staged<MODE, FIRST, true, W, V, D, false, CMP>
                            : k_check_staged<MODE, FIRST, false, W, V, D, false, CMP>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return false;
    }
    const int nb = w.Fp / (32 * V);
    const long long tasks = (long long)a.M * nb;
    const long long ctas = std::max<long long>(1, std::min<long long>((long long)w.num_sms * per_sm,
                                               (tasks + w.stage_warps - 1) / w.stage_warps));
    if (tasks + ctas * w.stage_warps >= (1ll << 31)) return false;
    StagedArgs sa;
    sa.ell_col = g.ell_col;
    sa.ell_deg = g.ell_deg;
    sa.ell_cls = g.ell_cls;
    sa.n_classes = a.n_classes;
    sa.M = a.M;
    sa.Fp = w.Fp;
    sa.n_fblocks = nb;
    sa.stages = w.stages;
    sa.paper = a.paper_slicer;
    sa.wait_limit = w.wait_limit;
    sa.state = w.state;
    sa.unsat = un;
    sa.err = w.err;
    sa.comp = w.comp;
    kern<<<(int)ctas, threads, smem, st>>>(sa, s, eta, wt);
    return true;
}

// The staged launch with w.stage_vw frames per lane (0: the run's V); any width up to V
// works on the same frame stride.
template <int MODE, int V, bool FIRST, bool W, int D, bool CMP = false>
bool staged(const DevGraph& g, const DecodeArgs& a, const StreamWork& w,
            const typename Tr<MODE>::T* s, typename Tr<MODE>::T* eta, uint8_t* un, int test_prev,
            const IterWeights& wt, cudaStream_t st) {
    switch (w.stage_vw) {
        case 0: return launch_staged<MODE, V, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
        case 1: return launch_staged<MODE, 1, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
        case 2:
            if constexpr (V >= 2)
                return launch_staged<MODE, 2, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
            break;
        case 4:
            if constexpr (V >= 4)
                return launch_staged<MODE, 4, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
            break;
        case 8:
            if constexpr (V >= 8)
                return launch_staged<MODE, 8, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
            break;
    }
    return launch_staged<MODE, V, FIRST, W, D, false, CMP>(g, a, w, s, eta, un, test_prev, wt, st);
}

// One check pass on compressed messages (FP32, padded row layout, staged kernel only);
// false when the staged kernel cannot run (the caller then keeps per-edge messages; this
// can only happen on the first iteration, before any state exists).
template <int V, bool FIRST, bool W>
bool check_pass_cmp(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, const float* s,
                    float* state, uint8_t* un, int test_prev, const IterWeights& wt_prev, cudaStream_t st) {
    if (g.ell_D == 8) return staged<kModeFP32, V, FIRST, W, 8, true>(g, a, w, s, state, un, test_prev, wt_prev, st);
    if (g.ell_D == 16) return staged<kModeFP32, V, FIRST, W, 16, true>(g, a, w, s, state, un, test_prev, wt_prev, st);
    return false;
}

// One check pass of iteration k: with the padded row layout, the staged kernel (when
// staging is on) or the register kernel; else the general kernel on the CSR order.
template <int MODE, int V, bool FIRST, bool W>
void check_pass_t(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, dim3 gc,
                  const typename Tr<MODE>::T* s, typename Tr<MODE>::T* eta, uint8_t* un,
                  int test_prev, const IterWeights& wt, cudaStream_t st) {
    const int Fp = w.Fp;
    if (g.ell_D == 8) {
        if (staged<MODE, V, FIRST, W, 8>(g, a, w, s, eta, un, test_prev, wt, st)) return;
        k_check_ell<MODE, FIRST, W, V, 8><<<gc, 128, 0, st>>>(g.ell_col, g.ell_deg, a.M, s, eta, Fp,
                                                              w.state, un, test_prev, a.paper_slicer, wt);
        return;
    }
    if (g.ell_D == 16) {
        if (staged<MODE, V, FIRST, W, 16>(g, a, w, s, eta, un, test_prev, wt, st)) return;
        k_check_ell<MODE, FIRST, W, V, 16><<<gc, 128, 0, st>>>(g.ell_col, g.ell_deg, a.M, s, eta, Fp,
                                                               w.state, un, test_prev, a.paper_slicer, wt);
        return;
    }
    k_check<MODE, FIRST, false, W, V><<<gc, 128, 0, st>>>(g.row_ptr, g.col_idx, a.M, s, eta, Fp,
                                                          w.state, un, test_prev, w.n_done, a.frames,
                                                          a.paper_slicer, wt);
}

template <int MODE, int V>
void check_pass(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, dim3 gc,
                const typename Tr<MODE>::T* s, typename Tr<MODE>::T* eta, uint8_t* un,
                int test_prev, bool first, const IterWeights& wt, cudaStream_t st) {
    if constexpr (MODE == kModeFP32) {  // learned weights exist in FP32 mode only
        if (wt.alpha != nullptr) {
            if (first) check_pass_t<MODE, V, true, true>(g, a, w, gc, s, eta, un, test_prev, wt, st);
            else check_pass_t<MODE, V, false, true>(g, a, w, gc, s, eta, un, test_prev, wt, st);
            return;
        }
    }
    if (first) check_pass_t<MODE, V, true, false>(g, a, w, gc, s, eta, un, test_prev, wt, st);
    else check_pass_t<MODE, V, false, false>(g, a, w, gc, s, eta, un, test_prev, wt, st);
}

// Frame compaction after an iteration (taking effect only when the scan decides so).
constexpr int kCompactEvery = 4;  // iterations between compaction checks

template <int MODE>
int compact(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, bool cmp) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    const int Fp = w.Fp;
    k_cmp_scan<<<1, kCmpThreads, 0, st>>>(w.state, w.new_pos, w.comp);
    const int blocks = std::max(1, std::min(65535, w.num_sms > 0 ? 8 * w.num_sms : 1024));
    k_cmp_emit<MODE><<<blocks, dim3(32, 8), 0, st>>>(
        (const T*)w.s, Fp, a.N, w.state, w.pos2frame, w.done_iter, w.comp, a.out_bits, a.out_soft,
        a.out_iters, a.out_ok, a.paper_slicer);
    if (cmp) {  // the rows' compressed messages: m0 and m1 (binary32), then the words
        const CState cs = cstate_at(w.eta, a.M, Fp);
        k_cmp_rows<float><<<blocks, 256, 0, st>>>(cs.m0, 2ll * a.M, Fp, w.new_pos, w.comp);
        k_cmp_rows<uint32_t><<<blocks, 256, 0, st>>>(cs.w, (long long)a.M, Fp, w.new_pos, w.comp);
    } else {
        k_cmp_rows<T><<<blocks, 256, 0, st>>>((T*)w.eta, (long long)g.eta_slots, Fp, w.new_pos, w.comp,
                                              g.ell_D ? g.ell_deg : nullptr, g.ell_D ? g.ell_D : 1);
    }
    k_cmp_rows<T><<<blocks, 256, 0, st>>>((T*)w.s, (long long)a.N, Fp, w.new_pos, w.comp);
    k_cmp_rows<R><<<blocks, 256, 0, st>>>((R*)w.r, (long long)a.N, Fp, w.new_pos, w.comp);
    k_cmp_rows<int32_t><<<1, 256, 0, st>>>(w.pos2frame, 1, Fp, w.new_pos, w.comp);
    k_cmp_tail<<<1, kCmpThreads, 0, st>>>(w.state, w.pos2frame, w.comp);
    return cmp ? 8 : 7;
}

// One bit pass of iteration k; hd: the HD variant (the last iteration, decisions packed).
template <int MODE, int V, bool CMP, bool W>
void var_pass(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, dim3 gv, const int32_t* cslot,
              uint8_t* un, int test_prev, int k, bool hd, const CState& cs, int dshift,
              const IterWeights& wt, cudaStream_t st) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    const R* r = (const R*)w.r;
    T* s = (T*)w.s;
    const T* eta = (const T*)w.eta;
    if constexpr (V == 4 || V == 8) {
        if (hd) {
            k_var<MODE, V, CMP, W, true><<<gv, 128, 0, st>>>(g.col_ptr, cslot, a.N, r, s, eta, w.Fp, w.state,
                                                             w.done_iter, w.pos2frame, un, test_prev, k,
                                                             w.n_done, a.frames, w.comp, cs, dshift, wt,
                                                             w.hd, a.paper_slicer);
            return;
        }
    }
    k_var<MODE, V, CMP, W><<<gv, 128, 0, st>>>(g.col_ptr, cslot, a.N, r, s, eta, w.Fp, w.state, w.done_iter,
                                               w.pos2frame, un, test_prev, k, w.n_done, a.frames, w.comp, cs,
                                               dshift, wt);
}

template <int MODE, int V>
int run(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    const int Fp = w.Fp;
    T* s = (T*)w.s;
    T* eta = (T*)w.eta;
    R* r = (R*)w.r;
    int launches = 0;
    if (cudaMemsetAsync(w.n_done, 0, sizeof(int32_t), st) != cudaSuccess) return LDPC_ERR_CUDA;
    if (cudaMemsetAsync(w.unsat, 0, (size_t)(a.L + 2) * Fp, st) != cudaSuccess) return LDPC_ERR_CUDA;
    uint8_t* state = w.state;
    k_init_state<<<(Fp + 255) / 256, 256, 0, st>>>(state, w.done_iter, w.pos2frame, w.comp, Fp,
                                                    a.frames);
    launches++;
    k_load<MODE><<<dim3((a.N + kLoadTJ - 1) / kLoadTJ, Fp / kLoadTF), 256, 0, st>>>(a.llr, a.llr_is_i8,
                                                                                      a.frames, a.N, r, s, Fp);
    launches++;
    const dim3 gc((a.M + 3) / 4, Fp / (32 * V));
    // the bit pass (k_var): in fixed point at most as many CTAs as are resident (16 per SM)
    // loop over the tasks of the frame blocks in use; in FP32 one CTA per task (column group
    // x frame block)
    const long long var_tasks = (long long)((a.N + 3) / 4) * (Fp / (32 * V));
    const dim3 gv = MODE == kModeFP32
                        ? dim3((a.N + 3) / 4, Fp / (32 * V))
                        : dim3((unsigned)std::max(1ll, std::min(var_tasks, 16ll * (w.num_sms > 0 ? w.num_sms : 148))));
    // message slot of each edge in column order: padded-row slots or CSR edge ids
    const int32_t* cslot = g.ell_D ? g.ell_cslot : g.col_edge;
    // compressed messages (cmsg.cuh) where the mode, the layout and the staging allow
    // (the staged kernel holds at most 256 classes of learned weights)
    bool cmp = MODE == kModeFP32 && w.msg_compressed && g.ell_D > 0 && w.stages > 0 &&
               (a.w_rows == 0 || a.n_classes <= 256);
    const int dshift = g.ell_D == 16 ? 4 : 3;
    // decisions of the last bit pass packed into w.hd (4 or 8 frames per lane): for the final
    // syndrome on the padded row layout, and for the output bits when no frame stops early
    // and no soft output is asked for (every position in use is then updated by that pass)
    const bool hd_store = !a.early_stop && !a.out_soft;
    const bool hd = (V == 4 || V == 8) && w.hd && a.L >= 1 && (g.ell_D > 0 || hd_store);
    auto weights_of = [&](int k) {  // learned weights of iteration k (none for k < 1)
        IterWeights wt{};
        if (MODE == kModeFP32 && a.w_rows > 0 && k >= 1) {
            const int row = (k < a.w_rows ? k : a.w_rows) - 1;
            wt = IterWeights{g.col_class, a.w_alpha + (size_t)row * a.n_classes,
                             a.w_beta + (size_t)row * a.n_classes};
        }
        return wt;
    };
    for (int k = 1; k <= a.L; k++) {
        const int test_prev = a.early_stop && ((k - 1) % a.check_every == 0);
        uint8_t* un = w.unsat + (size_t)k * Fp;
        const IterWeights wt = weights_of(k);
        if constexpr (MODE == kModeFP32) {
            if (cmp) {
                // the first pass has no old messages to rebuild, so no weights (there are
                // none for iteration 0); later passes rebuild with the previous iteration's
                const IterWeights wp = weights_of(k - 1);
                const bool W = a.w_rows > 0;
                const bool ok = k == 1 ? check_pass_cmp<V, true, false>(g, a, w, s, (float*)eta, un, test_prev, wp, st)
                                       : (W ? check_pass_cmp<V, false, true>(g, a, w, s, (float*)eta, un, test_prev, wp, st)
                                            : check_pass_cmp<V, false, false>(g, a, w, s, (float*)eta, un, test_prev, wp, st));
                if (ok) {
                    const CState cs = cstate_at(eta, a.M, Fp);
                    if (W)
                        var_pass<MODE, V, true, true>(g, a, w, gv, g.ell_cslot, un, test_prev, k, hd && k == a.L,
                                                      cs, dshift, wt, st);
                    else
                        var_pass<MODE, V, true, false>(g, a, w, gv, g.ell_cslot, un, test_prev, k, hd && k == a.L,
                                                       cs, dshift, wt, st);
                    launches += 2;
                    if (a.early_stop && k < a.L && k % kCompactEvery == 0 && w.comp)
                        launches += compact<MODE>(g, a, w, st, true);
                    continue;
                }
                if (k > 1) return LDPC_ERR_CUDA;  // cannot happen: the first launch decided
                cmp = false;                       // per-edge messages from here on
            }
        }
        check_pass<MODE, V>(g, a, w, gc, s, eta, un, test_prev, k == 1, wt, st);
        var_pass<MODE, V, false, false>(g, a, w, gv, cslot, un, test_prev, k, hd && k == a.L, CState{}, 0,
                                        IterWeights(), st);
        launches += 2;
        if (a.early_stop && k < a.L && k % kCompactEvery == 0 && w.comp)
            launches += compact<MODE>(g, a, w, st, false);
    }
    if (w.used_compressed) *w.used_compressed = cmp ? 1 : 0;
    uint8_t* unf = w.unsat + (size_t)(a.L + 1) * Fp;
    bool syn_done = false;
    uint32_t* ubits = nullptr;  // the final syndrome as bits, in the (cleared) unf region
    if constexpr (V == 4 || V == 8) {
        if (hd && (g.ell_D == 8 || g.ell_D == 16)) {
            const int runs = (a.M + kSynRows - 1) / kSynRows;
            const dim3 gs((unsigned)((runs + 7) / 8), (unsigned)((Fp / (4 * V) + 31) / 32));
            ubits = reinterpret_cast<uint32_t*>(unf);  // Fp / 8 of its Fp bytes, 256-byte aligned
            if (g.ell_D == 8)
                k_syn_hd<V, 8><<<gs, 256, 0, st>>>(g.ell_col, g.ell_deg, a.M, w.hd, Fp, ubits);
            else
                k_syn_hd<V, 16><<<gs, 256, 0, st>>>(g.ell_col, g.ell_deg, a.M, w.hd, Fp, ubits);
            syn_done = true;
        }
    }
    if (!syn_done) {
        if (g.ell_D == 8) {
            if (!launch_staged<MODE, V, true, false, 8, true>(g, a, w, s, eta, unf, 1, IterWeights(), st))
                k_syn_ell<MODE, V, 8><<<gc, 128, 0, st>>>(g.ell_col, g.ell_deg, a.M, s, Fp, state, unf,
                                                          a.paper_slicer);
        } else if (g.ell_D == 16) {
            if (!launch_staged<MODE, V, true, false, 16, true>(g, a, w, s, eta, unf, 1, IterWeights(), st))
                k_syn_ell<MODE, V, 16><<<gc, 128, 0, st>>>(g.ell_col, g.ell_deg, a.M, s, Fp, state, unf,
                                                           a.paper_slicer);
        } else
            k_check<MODE, false, true, false, V><<<gc, 128, 0, st>>>(g.row_ptr, g.col_idx, a.M, s, eta, Fp,
                                                                     state, unf, 1, w.n_done, a.frames,
                                                                     a.paper_slicer);
    }
    // (frames that stopped early are skipped there: their status is known)
    bool stored = false;
    if constexpr (V == 4 || V == 8) {
        if (hd && hd_store) {
            const int64_t warps = (int64_t)((a.N + 31) / 32) * (Fp / (16 * V));
            k_store_hd<V><<<(unsigned)((warps + 7) / 8), 256, 0, st>>>(w.hd, Fp, a.N, w.pos2frame, w.comp,
                                                                     a.out_bits);
            stored = true;
        }
    }
    if (!stored)
        k_store<MODE><<<dim3((a.N + kStoreTJ - 1) / kStoreTJ, Fp / kStoreTF), 256, 0, st>>>(
            s, Fp, a.N, w.pos2frame, w.comp, a.out_bits, a.out_soft, a.paper_slicer);
    k_finish<<<(Fp + 255) / 256, 256, 0, st>>>(w.done_iter, w.pos2frame, w.comp, unf, Fp, a.L,
                                               a.out_iters, a.out_ok, ubits);
    launches += 3;
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return launches;
}

}  // namespace

// The streaming decode in one arithmetic mode (stream_fp32.cu, stream_fixed.cu); vw as for
// stream_decode.
int stream_decode_fp32(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);
int stream_decode_fixed(const DevGraph& g, const DecodeArgs& a, const StreamWork& w, cudaStream_t st, int vw);

}  // namespace ldpc_impl
