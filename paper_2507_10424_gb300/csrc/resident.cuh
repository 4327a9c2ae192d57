// Resident variant: one persistent kernel per decode. Each CTA takes tiles of FT frames
// from an atomic work counter and runs every flooding iteration of Algorithm 1 for its
// tile with the edge messages eta, the posteriors s and the channel values r of all FT
// frames held in shared memory; global memory sees only the channel LLRs once and the
// decisions once per frame.
//
// Shared-memory layout: the FT frames of a tile are interleaved, so that one vector load
// (FT x 4 bytes in FP32, FT x 2 bytes in fixed point) serves every frame of an edge:
//   eta[row slot][FT]      row slots in the row-sliced order (slot of the k-th edge of
//                          lane l of slice q = r_base[q] + 32 k + l),
//   s[position][FT], r[position][FT]   by degree-sorted column position,
//   the index arrays of both sliced layouts (when they fit).
//
// One iteration = phase A (rows) then phase B (columns), separated by CTA barriers:
//   phase A, one thread per row lane: lambda = s - eta (eta^prev = 0 in the first
//     iteration; eq. eta_update), Observation 1 (min0, first location, min1) and
//     Observation 2 (XOR of sign bits), then eta = +-(min1 at the location, else min0).
//     The same sweep XORs the decisions of the gathered s: the syndrome of the current s
//     (eq. 1-2);
//   phase B, one thread per column lane: s = r + the column's eta in ascending row order
//     (eq. lambda_j).
// A frame whose syndrome is zero is written out at once (iterations = k); it keeps being
// computed with its tile (no per-frame branches in the inner loops) but is never written
// again. The tile ends when all its frames are out or after max_iter iterations.
#pragma once

#include <algorithm>
#include <type_traits>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"
#include "packed16.cuh"

namespace ldpc_impl {
namespace resident {

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

template <typename T, int V>
struct alignas(sizeof(T) * V) VecR {
    T x[V];
};

__device__ __forceinline__ int32_t rsat16(int32_t v) { return max(-kSat, min(kSat, v)); }
__device__ __forceinline__ float rabs(float x) { return fabsf(x); }
__device__ __forceinline__ int32_t rabs(int32_t x) { return abs(x); }
__device__ __forceinline__ float rbig(float) { return __int_as_float(0x7f800000); }
__device__ __forceinline__ int32_t rbig(int32_t) { return 0x7fffffff; }
__device__ __forceinline__ float rsat_out(float v) { return v; }
__device__ __forceinline__ int32_t rsat_out(int32_t v) { return rsat16(v); }
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

// Byte offsets of the shared-memory regions (host and device agree on them).
struct ResLayout {
    uint32_t eta, s, r, rpos, cslot, cpos, rdeg, cdeg, rbase, cbase, wcls, wtab, total;
};
__host__ __device__ inline uint32_t al16(uint32_t x) { return (x + 15u) & ~15u; }
__host__ __device__ inline ResLayout res_layout(int tb, int FT, int E_pad, int Ec_pad, int n_rsl,
                                                int n_csl, int N, bool idx, int w_entries = 0) {
    ResLayout L{};
    uint32_t o = 0;
    L.eta = o;
    o = al16(o + (uint32_t)E_pad * FT * tb);
    L.s = o;
    o = al16(o + (uint32_t)n_csl * 32 * FT * tb);
    L.r = o;
    o = al16(o + (uint32_t)n_csl * 32 * FT * tb);
    if (idx) {
        L.rpos = o;
        o = al16(o + (uint32_t)E_pad * 2);
        L.cslot = o;
        o = al16(o + (uint32_t)Ec_pad * 2);
        L.cpos = o;
        o = al16(o + (uint32_t)N * 2);
        L.rdeg = o;
        o = al16(o + (uint32_t)n_rsl * 32);
        L.cdeg = o;
        o = al16(o + (uint32_t)n_csl * 32);
        L.rbase = o;
        o = al16(o + (uint32_t)(n_rsl + 1) * 4);
        L.cbase = o;
        o = al16(o + (uint32_t)(n_csl + 1) * 4);
        if (w_entries > 0) {  // learned weights: class of each row slot, alpha and beta tables
            L.wcls = o;
            o = al16(o + (uint32_t)E_pad);
            L.wtab = o;
            o = al16(o + (uint32_t)w_entries * 2 * 4);
        }
    }
    L.total = o;
    return L;
}

struct ResArgs {
    const int32_t* r_base;
    const uint8_t* r_deg;
    const uint16_t* r_slot_pos;
    const int32_t* c_base;
    const uint8_t* c_deg;
    const uint16_t* c_slot;
    const uint16_t* col_pos;
    const uint8_t* r_slot_cls;
    int32_t n_rsl, n_csl, E_pad, Ec_pad, N;
    int32_t w_rows, n_classes;  // learned weights (FP32), w_rows = 0: plain Min-Sum
    const float* w_alpha;       // [w_rows][n_classes]
    const float* w_beta;
    const void* llr;
    int32_t llr_i8;
    int32_t frames, n_tiles, L, early_stop, check_every, paper;
    uint8_t* out_bits;
    int32_t* out_iters;
    uint8_t* out_ok;
    float* out_soft;
    int32_t* tile_counter;
};

struct Idx {
    const int32_t* r_base;
    const uint8_t* r_deg;
    const uint16_t* r_slot_pos;
    const int32_t* c_base;
    const uint8_t* c_deg;
    const uint16_t* c_slot;
    const uint16_t* col_pos;
    const uint8_t* wcls;   // class of each row slot (learned weights)
    const float* walpha;   // alpha row of the current iteration
    const float* wbeta;    // beta row of the current iteration
};

// Channel value of (frame, bit) in the arithmetic of the mode.
template <int MODE>
__device__ __forceinline__ typename RT<MODE>::A chan(const ResArgs& a, size_t idx) {
    if (MODE == kModeFP32) return __ldg((const float*)a.llr + idx);
    if (a.llr_i8) return (int32_t)__ldg((const int8_t*)a.llr + idx);
    return (int32_t)rquant(__ldg((const float*)a.llr + idx));
}

// Raw bits of a value whose sign bit is the decision "negative" (the values never hold
// -0.0: channel values are canonicalised at load, and round-to-nearest sums and
// differences of non-(-0) values are never -0.0).
__device__ __forceinline__ uint32_t bits_of(float x) { return __float_as_uint(x); }
__device__ __forceinline__ uint32_t bits_of(int32_t x) { return (uint32_t)x; }
// Sign-bit word of the hard decision: standard [s < 0], or the paper's [s > 0] = [0 - s < 0].
template <bool PAPER, typename A>
__device__ __forceinline__ uint32_t dec_bits(A s) { return PAPER ? bits_of(A(0) - s) : bits_of(s); }
// m with the sign bit of `sgn` (m >= 0).
__device__ __forceinline__ float with_sign(float m, uint32_t sgn) {
    return __uint_as_float(__float_as_uint(m) | (sgn & 0x80000000u));
}
__device__ __forceinline__ int32_t with_sign(int32_t m, uint32_t sgn) { return (int32_t)sgn < 0 ? -m : m; }
// lambda = s - eta, saturated in fixed point.
__device__ __forceinline__ float lam_sat(float s, float e) { return s - e; }
__device__ __forceinline__ int32_t lam_sat(int32_t s, int32_t e) { return rsat16(s - e); }

// min(a, b, c) in one three-input instruction (binary32; no NaN reaches it).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
// Observation 1 over two more magnitudes a0, a1: the smallest of the pair may become min0,
// and the second smallest of {min0, min1, a0, a1} is min(max(min0, lo), min1, hi) for the
// sorted pair lo <= hi (the second smallest of two sorted pairs).
__device__ __forceinline__ void two_min_pair(float& min0, float& min1, float a0, float a1) {
    const float lo = fminf(a0, a1), hi = fmaxf(a0, a1);
    min1 = fmin3(min1, fmaxf(min0, lo), hi);
    min0 = fminf(min0, lo);
}
// Second sweep of a row (FP32, plain Min-Sum), with the row's total sign folded into the
// two candidate magnitudes once: the message to an edge is p1 where |lambda| = min0, else
// p0, with lambda's own sign bit XORed in (Observation 2).
__device__ __forceinline__ float signed_pick(float lam, float min0, float p0, float p1) {
    const float v = (fabsf(lam) == min0) ? p1 : p0;
    return __uint_as_float(__float_as_uint(v) ^ (__float_as_uint(lam) & 0x80000000u));
}

// Task of round k for this thread: rounds alternate direction so that the work of a
// thread's tasks (sorted by decreasing degree) evens out. Strictly increasing in k.
__device__ __forceinline__ int snake(int k, int nth) {
    return k * nth + ((k & 1) ? (nth - 1 - (int)threadIdx.x) : (int)threadIdx.x);
}

// Largest row / column degree whose fully unrolled body keeps its operands in registers:
// about 32 (FP32 rows), 24 (fixed-point rows: the packed sweeps need more temporaries) or
// 30 (columns: slot ids too) registers of operands, at FT x sizeof(T) / 4 registers per
// edge vector. (Within the 64 registers of a 1024-thread CTA.) Fixed-point rows that also
// gather the syndrome (SYN) take 32 registers of operands: measured on the QC N=2304 batch
// with early stop, 4-frame tiles, rows of 13-16 edges unrolled instead of read twice by the
// loop form: 7.82 -> 7.53 ms, although the kernel then spills a few words; without the
// syndrome the same bodies were slower (6.59 -> 6.68 ms).
template <int MODE, int FT>
__host__ __device__ constexpr int vec_regs() {
    return (FT * (MODE == kModeFP32 ? 4 : 2) + 3) / 4;
}
template <int MODE, int FT, bool SYN = true>
__host__ __device__ constexpr int row_body_max() {
    return (MODE == kModeFP32 || SYN ? 32 : 24) / vec_regs<MODE, FT>() < 16
               ? (MODE == kModeFP32 || SYN ? 32 : 24) / vec_regs<MODE, FT>()
               : 16;
}
template <int MODE, int FT>
__host__ __device__ constexpr int col_body_max() {
    return 30 / (1 + vec_regs<MODE, FT>()) < 10 ? 30 / (1 + vec_regs<MODE, FT>()) : 10;
}

// ---------------------------------------------------------------------------------------
// The edge-slot array holds lambda after the column pass and the new message after the row
// pass (each edge belongs to one row and one column, so the passes never touch a slot
// twice at once):
//   init       lambda = r of the edge's bit (eta^prev = 0 in the first iteration);
//   rows       Observation 1 (min0, min1: on a tie min1 = min0, so the first location needs
//              no tracking) and Observation 2 (XOR of the sign bits) over the row's lambdas,
//              then eta = +-(min1 where |lambda| = min0, else min0), sign = total x own
//              (eq. eta_update);
//   columns    s = r + the column's eta in ascending row order (eq. lambda_j), then
//              lambda = s - eta (saturated in fixed point) into each of the column's slots;
//   syndrome   the XOR of the decisions of the row's bits, gathered from s (eq. 1-2), on the
//              iterations that test it.
// The row pass reads its slots contiguously: no gather of s and no index read per edge.
// ---------------------------------------------------------------------------------------

// Decision byte of a posterior vector (standard slicer): bit f = [s_f < 0], the sign bit
// (s never holds -0.0, and the fixed-point sums are saturated integers).
template <typename T, int FT>
__device__ __forceinline__ uint32_t dec_byte(const VecR<T, FT>& v) {
    uint32_t b = 0;
#pragma unroll
    for (int f = 0; f < FT; f++) b |= (bits_of((typename std::conditional<sizeof(T) == 4, float, int32_t>::type)v.x[f]) >> 31) << f;
    return b;
}
// The same for packed pairs: frame 2p in bit 15 of word p, frame 2p + 1 in bit 31.
template <int P>
__device__ __forceinline__ uint32_t dec_byte_packed(const Words<P>& w) {
    uint32_t b = 0;
#pragma unroll
    for (int p = 0; p < P; p++) b |= (((w.w[p] >> 15) & 1u) << (2 * p)) | ((w.w[p] >> 31) << (2 * p + 1));
    return b;
}

// The syndrome of s gathered by the row pass itself (early-stop kernels, on the iterations
// that test it): per row, bit 31 of zx[f] is the XOR of frame f's decisions over the row's
// bits (read from s through the slot's column position); the failing frames of the
// thread's rows collect in z, and a warp-wide OR reaches the CTA's word once per pass.
// With ON false every member is empty and the row pass is the plain one.
// DEC: the decisions come from the slots' decision bytes instead (bit f = frame f's
// decision on the slot's bit, written by the column pass): one contiguous byte per edge
// instead of a position index and a gathered posterior vector.
template <int MODE, int FT, bool PAPER, bool ON, bool DEC = false>
struct RowSyn {
    static constexpr bool kOn = ON;
    const VecR<typename RT<MODE>::T, FT>* s;
    uint32_t* unsat_w;
    const uint8_t* dec;
    uint32_t zx[FT];
    uint32_t z;
    __device__ __forceinline__ RowSyn(const VecR<typename RT<MODE>::T, FT>* s_, uint32_t* u,
                                      const uint8_t* d = nullptr)
        : s(s_), unsat_w(u), dec(d), z(0) {}
    __device__ __forceinline__ void row_begin() {
        if constexpr (ON) {
#pragma unroll
            for (int f = 0; f < FT; f++) zx[f] = 0;
        }
    }
    __device__ __forceinline__ void add(const Idx& ix, int slot) {
        if constexpr (ON && DEC) {
            zx[0] ^= dec[slot];
        } else if constexpr (ON) {
            using A = typename RT<MODE>::A;
            const auto sv = s[ix.r_slot_pos[slot]];
#pragma unroll
            for (int f = 0; f < FT; f++) zx[f] ^= dec_bits<PAPER>((A)sv.x[f]);
        }
    }
    __device__ __forceinline__ void row_end() {
        if constexpr (ON && DEC) {
            z |= zx[0];
        } else if constexpr (ON) {
#pragma unroll
            for (int f = 0; f < FT; f++) z |= (zx[f] >> 31) << f;
        }
    }
    // every thread of the CTA calls this once, after its last row
    __device__ __forceinline__ void flush() {
        if constexpr (ON) {
            const uint32_t zw = __reduce_or_sync(0xffffffffu, z);
            if (zw && (threadIdx.x & 31) == 0) atomicOr(unsat_w, zw);
        }
    }
};

// One row of exactly DC edges, per frame: the row's lambdas are read once into registers
// (fully unrolled), then the new messages are written.
// W: the learned decoder with a single weight class (alpha = wa, beta = wb for every edge).
template <int MODE, int FT, bool W, int DC, typename SY>
__device__ __forceinline__ void row_fixed(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots,
                                          int base, SY& sy, float wa = 1.0f, float wb = 0.0f) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    A min0[FT], min1[FT];
    uint32_t sx[FT];
#pragma unroll
    for (int f = 0; f < FT; f++) {
        min0[f] = rbig(A());
        min1[f] = rbig(A());
        sx[f] = 0;
    }
    VT lv[DC];
    sy.row_begin();
#pragma unroll
    for (int t = 0; t < DC; t++) {
        lv[t] = slots[base + 32 * t];
        sy.add(ix, base + 32 * t);
    }
    if constexpr (MODE == kModeFP32) {  // the magnitudes two at a time
#pragma unroll
        for (int t = 0; t + 1 < DC; t += 2) {
#pragma unroll
            for (int f = 0; f < FT; f++) {
                two_min_pair(min0[f], min1[f], fabsf(lv[t].x[f]), fabsf(lv[t + 1].x[f]));
                sx[f] ^= bits_of((A)lv[t].x[f]) ^ bits_of((A)lv[t + 1].x[f]);
            }
        }
    }
#pragma unroll
    for (int t = MODE == kModeFP32 ? DC - DC % 2 : 0; t < DC; t++) {
#pragma unroll
        for (int f = 0; f < FT; f++) {
            const A lam = (A)lv[t].x[f];
            const A m = rabs(lam);
            min1[f] = min(min1[f], max(min0[f], m));
            min0[f] = min(min0[f], m);
            sx[f] ^= bits_of(lam);
        }
    }
    if constexpr (MODE == kModeFP32) {
        // the two candidate magnitudes, weighted once per row when W: max(fma(alpha, m,
        // -beta), 0) of min0 and of min1 is what each edge would get from its own pick
        float p0[FT], p1[FT];
#pragma unroll
        for (int f = 0; f < FT; f++) {
            float c0 = (float)min0[f], c1 = (float)min1[f];
            if constexpr (W) {
                const float x0 = __fmaf_rn(wa, c0, -wb), x1 = __fmaf_rn(wa, c1, -wb);
                c0 = x0 > 0.0f ? x0 : 0.0f;
                c1 = x1 > 0.0f ? x1 : 0.0f;
            }
            p0[f] = with_sign(c0, sx[f]);
            p1[f] = with_sign(c1, sx[f]);
        }
#pragma unroll
        for (int t = 0; t < DC; t++) {
            VT out;
#pragma unroll
            for (int f = 0; f < FT; f++) out.x[f] = (T)signed_pick((float)lv[t].x[f], (float)min0[f], p0[f], p1[f]);
            slots[base + 32 * t] = out;
        }
    } else {
        static_assert(!W, "learned weights are FP32");
#pragma unroll
        for (int t = 0; t < DC; t++) {
            const int slot = base + 32 * t;
            VT out;
#pragma unroll
            for (int f = 0; f < FT; f++) {
                const A lam = (A)lv[t].x[f];
                const A m = (rabs(lam) == min0[f]) ? min1[f] : min0[f];
                out.x[f] = (T)with_sign(m, bits_of(lam) ^ sx[f]);
            }
            slots[slot] = out;
        }
    }
    sy.row_end();
}

template <int FT, int DC, typename SY>
__device__ __forceinline__ void row_fixed_packed(const Idx& ix, Words<FT / 2>* slots, int base,
                                                 SY& sy) {
    constexpr int P = FT / 2;
    using WT = Words<P>;
    uint32_t min0[P], min1[P], sx[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        min0[p] = 0x7fff7fffu;
        min1[p] = 0x7fff7fffu;
        sx[p] = 0;
    }
    WT lv[DC];
    sy.row_begin();
#pragma unroll
    for (int t = 0; t < DC; t++) {
        lv[t] = slots[base + 32 * t];
        sy.add(ix, base + 32 * t);
#pragma unroll
        for (int p = 0; p < P; p++) {
            const uint32_t lam = lv[t].w[p];
            const uint32_t m = p_max(lam, p_neg(lam));
            min1[p] = p_min(min1[p], p_max(min0[p], m));
            min0[p] = p_min(min0[p], m);
            sx[p] ^= lam;
        }
    }
    PackedPick pk[P];  // the slots take -eta (the column pass's sums and lambda use it so)
#pragma unroll
    for (int p = 0; p < P; p++) pk[p].set_neg(min0[p], min1[p], sx[p]);
#pragma unroll
    for (int t = 0; t < DC; t++) {
        WT out;
#pragma unroll
        for (int p = 0; p < P; p++) out.w[p] = pk[p](lv[t].w[p]);
        slots[base + 32 * t] = out;
    }
    sy.row_end();
}

// Exact-degree dispatch: rows of 2 .. MAXD edges take the fully unrolled body of their
// degree (the degree-sorted slices keep a warp's rows on the same case); returns false for
// longer rows.
template <int MAXD, typename Body>
__device__ __forceinline__ bool by_degree(int d, Body&& body) {
    bool done = true;
    switch (d) {
#define LDPC_CASE(DC) \
    case DC:          \
        if constexpr (DC <= MAXD) body(std::integral_constant<int, DC>()); \
        else done = false; \
        break;
        LDPC_CASE(1) LDPC_CASE(2) LDPC_CASE(3) LDPC_CASE(4) LDPC_CASE(5) LDPC_CASE(6) LDPC_CASE(7)
        LDPC_CASE(8) LDPC_CASE(9) LDPC_CASE(10) LDPC_CASE(11) LDPC_CASE(12) LDPC_CASE(13)
        LDPC_CASE(14) LDPC_CASE(15) LDPC_CASE(16)
#undef LDPC_CASE
        default: done = false;
    }
    return done;
}

// Row pass, per frame. Rows too long for an unrolled body read lambda twice (two sweeps);
// every row's slots end up holding the new messages. sy: the syndrome gather riding along.
// W1 (with W): the code has a single weight class, so the weights apply to the row's two
// candidate magnitudes once and the rows take the unrolled bodies; with several classes the
// weights are looked up per edge in the loop form.
template <int MODE, int FT, bool W, bool UNROLL = true, typename SY>
__device__ __forceinline__ void rows_pass(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots,
                                          int n_rtasks, SY&& sy, bool w1 = false) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    constexpr int UNR = FT >= 4 ? 2 : 4;
    const int nth = blockDim.x;
    float wa1 = 1.0f, wb1 = 0.0f;
    if constexpr (W) {
        if (w1) {
            wa1 = ix.walpha[0];
            wb1 = ix.wbeta[0];
        }
    }
    for (int k = 0;; k++) {
        const int task = snake(k, nth);  // strictly increasing in k
        if (task >= n_rtasks) break;
        const int d = ix.r_deg[task];
        if (d == 0) continue;
        const int base = ix.r_base[task >> 5] + (task & 31);
        if constexpr (UNROLL) {
            if ((!W || w1) && by_degree<row_body_max<MODE, FT>()>(d, [&](auto dc) {
                    row_fixed<MODE, FT, W, decltype(dc)::value>(ix, slots, base, sy, wa1, wb1);
                }))
                continue;
        }
        A min0[FT], min1[FT];
        uint32_t sx[FT];
#pragma unroll
        for (int f = 0; f < FT; f++) {
            min0[f] = rbig(A());
            min1[f] = rbig(A());
            sx[f] = 0;
        }
        sy.row_begin();
#pragma unroll UNR
        for (int t = 0; t < d; t++) {
            const VT lv = slots[base + 32 * t];
            sy.add(ix, base + 32 * t);
#pragma unroll
            for (int f = 0; f < FT; f++) {
                const A lam = (A)lv.x[f];
                const A m = rabs(lam);
                min1[f] = min(min1[f], max(min0[f], m));
                min0[f] = min(min0[f], m);
                sx[f] ^= bits_of(lam);
            }
        }
        if constexpr (MODE == kModeFP32 && !W) {
            float p0[FT], p1[FT];
#pragma unroll
            for (int f = 0; f < FT; f++) {
                p0[f] = with_sign((float)min0[f], sx[f]);
                p1[f] = with_sign((float)min1[f], sx[f]);
            }
#pragma unroll UNR
            for (int t = 0; t < d; t++) {
                const int slot = base + 32 * t;
                const VT lv = slots[slot];
                VT out;
#pragma unroll
                for (int f = 0; f < FT; f++) out.x[f] = (T)signed_pick((float)lv.x[f], (float)min0[f], p0[f], p1[f]);
                slots[slot] = out;
            }
        } else {
#pragma unroll UNR
            for (int t = 0; t < d; t++) {
                const int slot = base + 32 * t;
                const VT lv = slots[slot];
                float wa = 1.0f, wb = 0.0f;
                if constexpr (W) {
                    const int c = ix.wcls[slot];
                    wa = ix.walpha[c];
                    wb = ix.wbeta[c];
                }
                VT out;
#pragma unroll
                for (int f = 0; f < FT; f++) {
                    const A lam = (A)lv.x[f];
                    A m = (rabs(lam) == min0[f]) ? min1[f] : min0[f];
                    if constexpr (W) {  // max(fma(alpha, m, -beta), 0)
                        const float x = __fmaf_rn(wa, (float)m, -wb);
                        m = (A)(x > 0.0f ? x : 0.0f);
                    }
                    out.x[f] = (T)with_sign(m, bits_of(lam) ^ sx[f]);
                }
                slots[slot] = out;
            }
        }
        sy.row_end();
    }
    sy.flush();
}

// ---------------------------------------------------------------------------------------
// Fixed point with an even number of interleaved frames: the int16 values of two frames
// share a 32-bit word (frame 2p in the low half, 2p + 1 in the high half) and the passes
// work on the pair at once with the packed 16-bit min / max / add instructions. Every
// step is exact, so the results are those of the per-frame code. The row pass reads
// lambda = sat(s - eta) from the slots (formed by the column pass, PackedLam) and writes
// the negated new messages -eta back:
//   |lambda| = max(lambda, -lambda), -x = ~x + 1 lane by lane;
//   min0, min1, the XOR of the words (the sign bits of both lanes), as before;
//   sweep 2: magnitude min1 where |lambda| = min0 (|lambda| - min0 - 1 < 0), the row's
//            sign parity and the negation folded into the two candidates once per row,
//            and lambda's own sign applied by (m ^ mask) + (mask & 1) (PackedPick).
// ---------------------------------------------------------------------------------------
template <int FT, bool UNROLL = true, typename SY>
__device__ __forceinline__ void rows_pass_packed(const Idx& ix, VecR<int16_t, FT>* slots_v,
                                                 int n_rtasks, SY&& sy) {
    constexpr int P = FT / 2;
    using WT = Words<P>;
    constexpr int UNR = FT >= 4 ? 2 : 4;
    WT* slots = reinterpret_cast<WT*>(slots_v);
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int task = snake(k, nth);
        if (task >= n_rtasks) break;
        const int d = ix.r_deg[task];
        if (d == 0) continue;
        const int base = ix.r_base[task >> 5] + (task & 31);
        if constexpr (UNROLL) {
            if (by_degree<row_body_max<kModeFixed, FT, std::decay_t<SY>::kOn>()>(d, [&](auto dc) {
                    row_fixed_packed<FT, decltype(dc)::value>(ix, slots, base, sy);
                }))
                continue;
        }
        uint32_t min0[P], min1[P], sx[P];
#pragma unroll
        for (int p = 0; p < P; p++) {
            min0[p] = 0x7fff7fffu;
            min1[p] = 0x7fff7fffu;
            sx[p] = 0;
        }
        sy.row_begin();
#pragma unroll UNR
        for (int t = 0; t < d; t++) {
            const WT lv = slots[base + 32 * t];
            sy.add(ix, base + 32 * t);
#pragma unroll
            for (int p = 0; p < P; p++) {
                const uint32_t lam = lv.w[p];
                const uint32_t m = p_max(lam, p_neg(lam));
                min1[p] = p_min(min1[p], p_max(min0[p], m));
                min0[p] = p_min(min0[p], m);
                sx[p] ^= lam;
            }
        }
        PackedPick pk[P];  // the slots take -eta
#pragma unroll
        for (int p = 0; p < P; p++) pk[p].set_neg(min0[p], min1[p], sx[p]);
#pragma unroll UNR
        for (int t = 0; t < d; t++) {
            const int slot = base + 32 * t;
            const WT lv = slots[slot];
            WT out;
#pragma unroll
            for (int p = 0; p < P; p++) out.w[p] = pk[p](lv.w[p]);
            slots[slot] = out;
        }
        sy.row_end();
    }
    sy.flush();
}

// Syndrome of the current s for every row: bit f of the row's result is set when frame f
// fails the check; the CTA's word collects them.
template <int MODE, int FT, bool PAPER, bool DEC = false>
__device__ __forceinline__ void syn_pass(const Idx& ix, const VecR<typename RT<MODE>::T, FT>* s,
                                         int n_rtasks, uint32_t* unsat_w,
                                         const uint8_t* dec = nullptr) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int task = snake(k, nth);
        if (task >= n_rtasks) break;
        const int d = ix.r_deg[task];
        if (d == 0) continue;
        const int base = ix.r_base[task >> 5] + (task & 31);
        uint32_t z = 0;
        if constexpr (DEC) {  // the slots' decision bytes (written by the last column pass)
#pragma unroll 4
            for (int t = 0; t < d; t++) z ^= dec[base + 32 * t];
        } else {
            uint32_t zx[FT];
#pragma unroll
            for (int f = 0; f < FT; f++) zx[f] = 0;
#pragma unroll 4
            for (int t = 0; t < d; t++) {
                const VT sv = s[ix.r_slot_pos[base + 32 * t]];
#pragma unroll
                for (int f = 0; f < FT; f++) zx[f] ^= dec_bits<PAPER>((A)sv.x[f]);
            }
#pragma unroll
            for (int f = 0; f < FT; f++) z |= (zx[f] >> 31) << f;
        }
        if (z) atomicOr(unsat_w, z);
    }
}

// First lambda of every edge: the channel value of its bit (DEC: and the decision byte of
// the channel values, for the syndrome before the first iteration).
template <int MODE, int FT, bool DEC = false>
__device__ __forceinline__ void init_pass(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots,
                                          const VecR<typename RT<MODE>::T, FT>* r, int N,
                                          uint8_t* dec = nullptr) {
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int p = snake(k, nth);
        if (p >= N) break;
        const int d = ix.c_deg[p];
        const int base = ix.c_base[p >> 5] + (p & 31);
        const auto rv = r[p];
        const uint32_t db = DEC ? dec_byte(rv) : 0u;
        for (int t = 0; t < d; t++) {
            const int slot = ix.c_slot[base + 32 * t];
            slots[slot] = rv;
            if constexpr (DEC) dec[slot] = (uint8_t)db;
        }
    }
}

// One column of exactly DC edges, per frame: s = r + sum of eta (ascending rows), then
// lambda = s - eta into each of its slots. Fully unrolled: slots and messages stay in
// registers between the two loops, and no predicated-off iteration is issued.
template <int MODE, int FT, int DC, bool DEC = false>
__device__ __forceinline__ void col_fixed(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots,
                                          VecR<typename RT<MODE>::T, FT>* s,
                                          const VecR<typename RT<MODE>::T, FT>& rv, int p, int base,
                                          uint8_t* dec = nullptr) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    A acc[FT];
#pragma unroll
    for (int f = 0; f < FT; f++) acc[f] = (A)rv.x[f];
    int sl[DC];
    VT ev[DC];
#pragma unroll
    for (int t = 0; t < DC; t++) {
        sl[t] = ix.c_slot[base + 32 * t];
        ev[t] = slots[sl[t]];
#pragma unroll
        for (int f = 0; f < FT; f++) acc[f] = acc[f] + (A)ev[t].x[f];
    }
    VT out;
#pragma unroll
    for (int f = 0; f < FT; f++) out.x[f] = (T)rsat_out(acc[f]);
    s[p] = out;
#pragma unroll
    for (int t = 0; t < DC; t++) {
        VT lv;
#pragma unroll
        for (int f = 0; f < FT; f++) lv.x[f] = (T)lam_sat((A)out.x[f], (A)ev[t].x[f]);
        slots[sl[t]] = lv;
    }
    if constexpr (DEC) {
        if (dec) {
            const uint8_t db = (uint8_t)dec_byte(out);
#pragma unroll
            for (int t = 0; t < DC; t++) dec[sl[t]] = db;
        }
    }
}

// A column of any degree: the second loop reads its slots and messages again.
template <int MODE, int FT, bool DEC = false>
__device__ __forceinline__ void col_any(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots,
                                        VecR<typename RT<MODE>::T, FT>* s,
                                        const VecR<typename RT<MODE>::T, FT>& rv, int p, int base,
                                        int d, uint8_t* dec = nullptr) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    A acc[FT];
#pragma unroll
    for (int f = 0; f < FT; f++) acc[f] = (A)rv.x[f];
    for (int t = 0; t < d; t++) {
        const VT ev = slots[ix.c_slot[base + 32 * t]];
#pragma unroll
        for (int f = 0; f < FT; f++) acc[f] = acc[f] + (A)ev.x[f];
    }
    VT out;
#pragma unroll
    for (int f = 0; f < FT; f++) out.x[f] = (T)rsat_out(acc[f]);
    s[p] = out;
    const uint32_t db = DEC ? dec_byte(out) : 0u;
    for (int t = 0; t < d; t++) {
        const int slot = ix.c_slot[base + 32 * t];
        const VT ev = slots[slot];
        VT lv;
#pragma unroll
        for (int f = 0; f < FT; f++) lv.x[f] = (T)lam_sat((A)out.x[f], (A)ev.x[f]);
        slots[slot] = lv;
        if constexpr (DEC) {
            if (dec) dec[slot] = (uint8_t)db;
        }
    }
}

// Packed fixed point: the slots hold the negated messages ne = -eta between the row and
// the column pass (the row pass negates its two candidate magnitudes once per row). The
// column pass sums s = r - sum(ne) in 32 bits (one dp2a per lane and edge), saturates and
// packs, then forms lambda = sat(s - eta) = sat(s + ne) lane by lane without leaving the
// packed form. With s, ne in [-32767, 32767], clamping ne to
// [-32767 - min(s, 0), 32767 - max(s, 0)] (both bounds representable) makes s + ne' equal to
// sat(s + ne) exactly: ne is raised only when s < 0 and s + ne < -32767, lowered only when
// s > 0 and s + ne > 32767, and otherwise the sum is already within the limits; the wrapping
// packed add is exact because the result is in range. Per column: the two bounds; per edge:
// max, min, add.
struct PackedLam {
    uint32_t lo = 0, hi = 0, sw = 0;
    __device__ __forceinline__ void set(uint32_t s) {
        sw = s;
        lo = p_add(~p_min(s, 0u), 0x80028002u);  // -32767 - min(s, 0) = ~min(s, 0) - 32766
        hi = p_add(~p_max(s, 0u), 0x80008000u);  // 32767 - max(s, 0) = ~max(s, 0) + 32768 (mod 2^16)
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t ne) const {
        return p_add(sw, p_min(p_max(ne, lo), hi));
    }
};

template <int FT, int DC, bool DEC = false>
__device__ __forceinline__ void col_fixed_packed(const Idx& ix, Words<FT / 2>* slots, Words<FT / 2>* s,
                                                 const Words<FT / 2>& rv, int p0, int base,
                                                 uint8_t* dec = nullptr) {
    constexpr int P = FT / 2;
    using WT = Words<P>;
    int32_t lo[P], hi[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        lo[p] = p_lo(rv.w[p]);
        hi[p] = p_hi(rv.w[p]);
    }
    int sl[DC];
    WT ev[DC];
#pragma unroll
    for (int t = 0; t < DC; t++) {
        sl[t] = ix.c_slot[base + 32 * t];
        ev[t] = slots[sl[t]];
#pragma unroll
        for (int p = 0; p < P; p++) {
            lo[p] = p_sub_lo(lo[p], ev[t].w[p]);  // the slots hold -eta
            hi[p] = p_sub_hi(hi[p], ev[t].w[p]);
        }
    }
    WT out;
#pragma unroll
    for (int p = 0; p < P; p++) out.w[p] = p_pack_sat(lo[p], hi[p]);
    s[p0] = out;
    PackedLam lam[P];
#pragma unroll
    for (int p = 0; p < P; p++) lam[p].set(out.w[p]);
#pragma unroll
    for (int t = 0; t < DC; t++) {
        WT lv;
#pragma unroll
        for (int p = 0; p < P; p++) lv.w[p] = lam[p](ev[t].w[p]);
        slots[sl[t]] = lv;
    }
    if constexpr (DEC) {
        if (dec) {
            const uint8_t db = (uint8_t)dec_byte_packed(out);
#pragma unroll
            for (int t = 0; t < DC; t++) dec[sl[t]] = db;
        }
    }
}

template <int FT, bool DEC = false>
__device__ __forceinline__ void col_any_packed(const Idx& ix, Words<FT / 2>* slots, Words<FT / 2>* s,
                                               const Words<FT / 2>& rv, int p0, int base, int d,
                                               uint8_t* dec = nullptr) {
    constexpr int P = FT / 2;
    using WT = Words<P>;
    int32_t lo[P], hi[P];
#pragma unroll
    for (int p = 0; p < P; p++) {
        lo[p] = p_lo(rv.w[p]);
        hi[p] = p_hi(rv.w[p]);
    }
    for (int t = 0; t < d; t++) {
        const WT ev = slots[ix.c_slot[base + 32 * t]];
#pragma unroll
        for (int p = 0; p < P; p++) {
            lo[p] = p_sub_lo(lo[p], ev.w[p]);  // the slots hold -eta
            hi[p] = p_sub_hi(hi[p], ev.w[p]);
        }
    }
    WT out;
#pragma unroll
    for (int p = 0; p < P; p++) out.w[p] = p_pack_sat(lo[p], hi[p]);
    s[p0] = out;
    PackedLam lam[P];
#pragma unroll
    for (int p = 0; p < P; p++) lam[p].set(out.w[p]);
    const uint32_t db = DEC ? dec_byte_packed(out) : 0u;
    for (int t = 0; t < d; t++) {
        const int slot = ix.c_slot[base + 32 * t];
        const WT ev = slots[slot];
        WT lv;
#pragma unroll
        for (int p = 0; p < P; p++) lv.w[p] = lam[p](ev.w[p]);
        slots[slot] = lv;
        if constexpr (DEC) {
            if (dec) dec[slot] = (uint8_t)db;
        }
    }
}

// Column pass over every column position of the tile; columns up to col_body_max edges take
// the fully unrolled body of their degree (the degree-sorted slices keep a warp's columns
// on the same case).
// DEC: also the decision byte of each column into its slots of `dec` (when not null).
template <int MODE, int FT, bool UNROLL = true, bool DEC = false>
__device__ __forceinline__ void cols_pass(const Idx& ix, VecR<typename RT<MODE>::T, FT>* slots_v,
                                          VecR<typename RT<MODE>::T, FT>* s_v,
                                          const VecR<typename RT<MODE>::T, FT>* r_v, int N,
                                          uint8_t* dec = nullptr) {
    constexpr bool kPacked = MODE == kModeFixed && FT % 2 == 0;
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int p = snake(k, nth);
        if (p >= N) break;
        const int d = ix.c_deg[p];
        const int base = ix.c_base[p >> 5] + (p & 31);
        if constexpr (kPacked) {
            using WT = Words<FT / 2>;
            WT* slots = reinterpret_cast<WT*>(slots_v);
            WT* s = reinterpret_cast<WT*>(s_v);
            const WT rv = reinterpret_cast<const WT*>(r_v)[p];
            if (!UNROLL || !by_degree<col_body_max<MODE, FT>()>(d, [&](auto dc) {
                    col_fixed_packed<FT, decltype(dc)::value, DEC>(ix, slots, s, rv, p, base, dec);
                }))
                col_any_packed<FT, DEC>(ix, slots, s, rv, p, base, d, dec);
        } else {
            const auto rv = r_v[p];
            if (!UNROLL || !by_degree<col_body_max<MODE, FT>()>(d, [&](auto dc) {
                    col_fixed<MODE, FT, decltype(dc)::value, DEC>(ix, slots_v, s_v, rv, p, base, dec);
                }))
                col_any<MODE, FT, DEC>(ix, slots_v, s_v, rv, p, base, d, dec);
        }
    }
}

// Write the decisions (and posteriors) of the frames in `mask`.
template <int MODE, int FT>
__device__ __forceinline__ void emit(const ResArgs& a, const Idx& ix,
                                     const VecR<typename RT<MODE>::T, FT>* s, int fbase,
                                     uint32_t mask, int iters, uint32_t okm) {
    using A = typename RT<MODE>::A;
    const int N = a.N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const auto v = s[ix.col_pos[j]];
#pragma unroll
        for (int f = 0; f < FT; f++) {
            if (!((mask >> f) & 1u)) continue;
            const size_t o = (size_t)(fbase + f) * N + j;
            const A x = (A)v.x[f];
            a.out_bits[o] = (uint8_t)rslice(x, a.paper);
            if (a.out_soft) a.out_soft[o] = (MODE == kModeFP32) ? (float)x : (float)x * 0.25f;
        }
    }
#pragma unroll
    for (int f = 0; f < FT; f++)
        if (threadIdx.x == f && ((mask >> f) & 1u)) {
            a.out_iters[fbase + f] = iters;
            if (a.out_ok) a.out_ok[fbase + f] = (okm >> f) & 1u;
        }
}

template <typename T>
__device__ __forceinline__ void copy_to_smem(T* dst, const T* src, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Every iteration of one tile of nf frames (frames fbase .. fbase + nf - 1 of a.llr) with
// eta, s and r at the given addresses (shared memory, or a CTA's slot of global scratch),
// ending with the decisions of every frame written out. unsat_w: two words reset to 0.
// UNROLL: the fully unrolled row and column bodies (false in kernels that inline several
// tile shapes and would exceed their register budget). Weighted rows take the unrolled
// bodies only when the code has one weight class (the weights then act on the row's two
// candidate magnitudes); with several classes they take the loop form: unrolled, their
// per-edge class and weight loads raised the early-stop kernels to the 64-register bound,
// which costs small tiles resident CTAs per SM.
// ES (early-stop kernels): the row pass of iteration k + 1 also gathers the syndrome of s
// after iteration k, which s still holds until the column pass, so a tested iteration
// costs no pass of its own; the frames that are codewords are written out between the
// two passes. Without ES the syndrome is a pass of its own before the row pass (one
// barrier more per tested iteration).
// DEC (early-stop kernels with the index arrays in shared memory): every syndrome reads
// the slots' decision bytes `dec` [E_pad], which the init pass and the column passes before
// a tested iteration write, instead of gathering s through the slots' column positions.
template <int MODE, int FT, bool PAPER, bool W, typename VT, bool UNROLL = true, bool ES = false,
          bool DEC = false>
__device__ __forceinline__ void decode_tile(const ResArgs& a, Idx ix, VT* eta, VT* s, VT* r,
                                            uint32_t* unsat_w, int fbase, int nf,
                                            const float* walpha0, const float* wbeta0,
                                            int n_rtasks, uint8_t* dec = nullptr) {
    static_assert(!DEC || (ES && !PAPER), "decision bytes are the standard slicer's");
    using T = typename RT<MODE>::T;
    constexpr bool kPacked = MODE == kModeFixed && FT % 2 == 0;
    const int N = a.N;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        VT v;
#pragma unroll
        for (int f = 0; f < FT; f++)  // "+ 0" turns -0.0 into +0.0 and changes no other value
            v.x[f] = f < nf ? (T)(chan<MODE>(a, (size_t)(fbase + f) * N + j) + 0) : T(0);
        const int p = ix.col_pos[j];
        s[p] = v;
        r[p] = v;
    }
    uint32_t active = (1u << nf) - 1u;
    __syncthreads();
    init_pass<MODE, FT, DEC>(ix, eta, r, N, dec);  // the edge slots hold lambda from here on
    __syncthreads();

    for (int k = 0;; k++) {
        const int par = k & 1;
        const bool last = (k == a.L);
        const bool syn = last || (a.early_stop && (k % a.check_every == 0));
        if (syn && (!ES || last)) {  // the decisions of the current s: stop the codewords
            syn_pass<MODE, FT, PAPER, DEC>(ix, s, n_rtasks, &unsat_w[par], dec);
            __syncthreads();
            const uint32_t conv = active & ~unsat_w[par];
            if (last) {
                emit<MODE, FT>(a, ix, s, fbase, active, a.L, conv);
                break;
            }
            if (conv) {
                emit<MODE, FT>(a, ix, s, fbase, conv, k, conv);
                active &= ~conv;
                if (!active) break;
            }
        }
        if (W) {  // weights of iteration k + 1 (the last row serves the later iterations)
            const int row = min(k + 1, a.w_rows) - 1;
            ix.walpha = walpha0 + row * a.n_classes;
            ix.wbeta = wbeta0 + row * a.n_classes;
        }
        if (ES && syn) {
            if constexpr (kPacked)
                rows_pass_packed<FT, UNROLL>(ix, eta, n_rtasks,
                                             RowSyn<MODE, FT, PAPER, true, DEC>(s, &unsat_w[par], dec));
            else
                rows_pass<MODE, FT, W, UNROLL>(ix, eta, n_rtasks,
                                               RowSyn<MODE, FT, PAPER, true, DEC>(s, &unsat_w[par], dec),
                                               W && a.n_classes == 1);
            __syncthreads();
            const uint32_t conv = active & ~unsat_w[par];
            if (conv) {  // s still holds the decisions of iteration k
                emit<MODE, FT>(a, ix, s, fbase, conv, k, conv);
                active &= ~conv;
                if (!active) break;
                __syncthreads();  // emit's reads of s before the column pass rewrites s
            }
        } else {
            if constexpr (kPacked)
                rows_pass_packed<FT, UNROLL>(ix, eta, n_rtasks,
                                             RowSyn<MODE, FT, PAPER, false>(s, nullptr));
            else
                rows_pass<MODE, FT, W, UNROLL>(ix, eta, n_rtasks,
                                               RowSyn<MODE, FT, PAPER, false>(s, nullptr),
                                               W && a.n_classes == 1);
            __syncthreads();  // (also orders emit's reads of s before the column pass rewrites s)
        }
        if constexpr (DEC) {  // decision bytes only before an iteration that tests the syndrome
            const int k1 = k + 1;
            const bool tested = k1 == a.L || (a.early_stop && k1 % a.check_every == 0);
            cols_pass<MODE, FT, UNROLL, true>(ix, eta, s, r, N, tested ? dec : nullptr);
        } else {
            cols_pass<MODE, FT, UNROLL>(ix, eta, s, r, N);
        }
        if (threadIdx.x == 0) unsat_w[par ^ 1] = 0;
        __syncthreads();
    }
}

template <int MODE, int FT, bool IDX_SMEM, bool PAPER, bool W, bool ES>
__global__ void __launch_bounds__(kMaxThreads, 1) k_resident(const ResArgs a) {
    using T = typename RT<MODE>::T;
    using VT = VecR<T, FT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t unsat_w[2];
    __shared__ int tile_sh;
    const int w_entries = W ? a.w_rows * a.n_classes : 0;
    const ResLayout lay = res_layout((int)sizeof(T), FT, a.E_pad, a.Ec_pad, a.n_rsl, a.n_csl, a.N,
                                     IDX_SMEM, w_entries);
    // early stop with the index arrays in shared memory: the slots' decision bytes take the
    // place of the slot position array (E_pad bytes of its 2 E_pad). Taken where the gather
    // of s it replaces is dear: fixed point (the gather's per-frame sign extraction costs
    // ALU, the bound there, and registers) and FP32 tiles of 4 frames (16-byte vectors
    // gathered). FP32 tiles of 2 frames keep the gather: measured on the QC N=2304 batch
    // with early stop, decision bytes took 10.26 -> 10.91 ms (fixed point 9.09 -> 8.08 ms,
    // FP32 4-frame tiles on N=576 0.0759 -> 0.0704 ms).
    constexpr bool kDec = ES && IDX_SMEM && !PAPER && (MODE == kModeFixed || FT >= 4);
    uint8_t* dec = nullptr;
    VT* eta = reinterpret_cast<VT*>(smem_raw + lay.eta);
    VT* s = reinterpret_cast<VT*>(smem_raw + lay.s);
    VT* r = reinterpret_cast<VT*>(smem_raw + lay.r);
    Idx ix;
    if (IDX_SMEM) {
        uint16_t* rpos = reinterpret_cast<uint16_t*>(smem_raw + lay.rpos);
        uint16_t* cslot = reinterpret_cast<uint16_t*>(smem_raw + lay.cslot);
        uint16_t* cpos = reinterpret_cast<uint16_t*>(smem_raw + lay.cpos);
        uint8_t* rdeg = smem_raw + lay.rdeg;
        uint8_t* cdeg = smem_raw + lay.cdeg;
        int32_t* rbase = reinterpret_cast<int32_t*>(smem_raw + lay.rbase);
        int32_t* cbase = reinterpret_cast<int32_t*>(smem_raw + lay.cbase);
        if (!kDec) copy_to_smem(rpos, a.r_slot_pos, a.E_pad);  // (kDec: the decision bytes' region)
        copy_to_smem(cslot, a.c_slot, a.Ec_pad);
        copy_to_smem(cpos, a.col_pos, a.N);
        copy_to_smem(rdeg, a.r_deg, a.n_rsl * 32);
        copy_to_smem(cdeg, a.c_deg, a.n_csl * 32);
        copy_to_smem(rbase, a.r_base, a.n_rsl + 1);
        copy_to_smem(cbase, a.c_base, a.n_csl + 1);
        ix = Idx{rbase, rdeg, kDec ? a.r_slot_pos : rpos, cbase, cdeg, cslot, cpos, nullptr, nullptr, nullptr};
        dec = reinterpret_cast<uint8_t*>(rpos);
        if (W) {
            uint8_t* wcls = smem_raw + lay.wcls;
            float* wtab = reinterpret_cast<float*>(smem_raw + lay.wtab);
            copy_to_smem(wcls, a.r_slot_cls, a.E_pad);
            copy_to_smem(wtab, a.w_alpha, w_entries);
            copy_to_smem(wtab + w_entries, a.w_beta, w_entries);
            ix.wcls = wcls;
            ix.walpha = wtab;
            ix.wbeta = wtab + w_entries;
        }
    } else {
        ix = Idx{a.r_base, a.r_deg, a.r_slot_pos, a.c_base, a.c_deg, a.c_slot, a.col_pos,
                 a.r_slot_cls, a.w_alpha, a.w_beta};
    }
    const float* walpha0 = ix.walpha;
    const float* wbeta0 = ix.wbeta;
    const int n_rtasks = a.n_rsl * 32;

    for (;;) {
        if (threadIdx.x == 0) {
            tile_sh = atomicAdd(a.tile_counter, 1);
            unsat_w[0] = 0;
            unsat_w[1] = 0;
        }
        __syncthreads();
        const int tile = tile_sh;
        if (tile >= a.n_tiles) break;
        const int fbase = tile * FT;
        decode_tile<MODE, FT, PAPER, W, VT, true, ES, kDec>(a, ix, eta, s, r, unsat_w, fbase,
                                                            min(FT, a.frames - fbase), walpha0, wbeta0,
                                                            n_rtasks, dec);
        __syncthreads();
    }
}

template <int MODE, int FT, bool IDX, bool PAPER, bool W, bool ES>
int launch(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    auto kern = k_resident<MODE, FT, IDX, PAPER, W, ES>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, p.threads, p.smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    if (per_sm < 1) return LDPC_ERR_UNSUPPORTED;
    const int grid = std::max(1, std::min(ra.n_tiles, num_sms * per_sm));
    kern<<<grid, p.threads, p.smem, st>>>(ra);
    return cudaGetLastError() == cudaSuccess ? 1 : LDPC_ERR_CUDA;
}

// Instantiations: index arrays in shared memory with FT in {1, 2, 4}; in global memory
// with FT in {1, 2}; each with the standard and the paper's slicer, and, for the standard
// slicer, the early-stop form (ES) too.
template <int MODE, bool IDX, bool PAPER, bool W, bool ES>
int launch_ft(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    switch (p.FT) {
        case 1: return launch<MODE, 1, IDX, PAPER, W, ES>(ra, p, num_sms, st);
        case 2: return launch<MODE, 2, IDX, PAPER, W, ES>(ra, p, num_sms, st);
        case 4:
            if constexpr (IDX) return launch<MODE, 4, IDX, PAPER, W, ES>(ra, p, num_sms, st);
            break;
    }
    return LDPC_ERR_INVALID_ARG;
}

// ES = true: decodes that test the syndrome during the iterations, standard slicer.
template <int MODE, bool W, bool ES>
int dispatch_w(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    if constexpr (ES) {
        return p.idx_smem ? launch_ft<MODE, true, false, W, true>(ra, p, num_sms, st)
                          : launch_ft<MODE, false, false, W, true>(ra, p, num_sms, st);
    } else {
        if (p.idx_smem)
            return ra.paper ? launch_ft<MODE, true, true, W, false>(ra, p, num_sms, st)
                            : launch_ft<MODE, true, false, W, false>(ra, p, num_sms, st);
        return ra.paper ? launch_ft<MODE, false, true, W, false>(ra, p, num_sms, st)
                        : launch_ft<MODE, false, false, W, false>(ra, p, num_sms, st);
    }
}

// Whether a decode takes the early-stop kernels.
inline bool use_es(const ResArgs& ra) { return ra.early_stop && !ra.paper && ra.L > 0; }

// Learned weights exist in FP32 mode only.
template <int MODE, bool ES>
int dispatch(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st) {
    if constexpr (MODE == kModeFP32)
        if (ra.w_rows > 0) return dispatch_w<MODE, true, ES>(ra, p, num_sms, st);
    return dispatch_w<MODE, false, ES>(ra, p, num_sms, st);
}

// resident_fp32.cu / resident_fixed.cu hold the kernels without ES, resident_fp32_es.cu /
// resident_fixed_es.cu those with it (translation units of their own: the build runs them
// in parallel).
int dispatch_fp32(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st);
int dispatch_fixed(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st);
int dispatch_fp32_es(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st);
int dispatch_fixed_es(const ResArgs& ra, const ResidentPlan& p, int num_sms, cudaStream_t st);

}  // namespace resident
}  // namespace ldpc_impl
