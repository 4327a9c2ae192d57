// Packed 16-bit integer helpers of the fixed-point mode: the int16 values of two frames
// share a 32-bit word (the even frame in the low half, the odd frame in the high half) and
// one instruction treats both. Every helper is exact on values in [-32767, 32767].
#pragma once

#include <stdint.h>

namespace ldpc_impl {

template <int P>
struct alignas(4 * P) Words {
    uint32_t w[P];
};
__device__ __forceinline__ uint32_t p_min(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("min.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t p_max(uint32_t a, uint32_t b) {
    uint32_t d;
    asm("max.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t p_add(uint32_t a, uint32_t b) {  // lane-wise, wrapping
    uint32_t d;
    asm("add.s16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t p_neg(uint32_t a) { return p_add(~a, 0x00010001u); }
__device__ __forceinline__ int32_t p_lo(uint32_t w) { return (int32_t)(int16_t)(w & 0xffffu); }
__device__ __forceinline__ int32_t p_hi(uint32_t w) { return (int32_t)w >> 16; }
// acc + the low (p_acc_lo) or high (p_acc_hi) lane of w, or minus it (p_sub_lo, p_sub_hi):
// one two-way 16 x 8-bit dot product (dp2a) with the byte weights (1, 0), (0, 1), (-1, 0)
// or (0, -1); it extracts, sign-extends and adds in one instruction. Exact in int32.
template <int B>
__device__ __forceinline__ int32_t p_dot(int32_t acc, uint32_t w) {
    int32_t d;
    asm("dp2a.lo.s32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(w), "r"(B), "r"(acc));
    return d;
}
__device__ __forceinline__ int32_t p_acc_lo(int32_t acc, uint32_t w) { return p_dot<0x0001>(acc, w); }
__device__ __forceinline__ int32_t p_acc_hi(int32_t acc, uint32_t w) { return p_dot<0x0100>(acc, w); }
__device__ __forceinline__ int32_t p_sub_lo(int32_t acc, uint32_t w) { return p_dot<0x00ff>(acc, w); }
__device__ __forceinline__ int32_t p_sub_hi(int32_t acc, uint32_t w) { return p_dot<0xff00>(acc, w); }
// Both lanes saturated to [-32767, 32767] and packed (lo in the low half).
__device__ __forceinline__ uint32_t p_pack_sat(int32_t lo, int32_t hi) {
    uint32_t d;
    asm("cvt.pack.sat.s16.s32 %0, %1, %2;" : "=r"(d) : "r"(hi), "r"(lo));
    return p_max(d, 0x80018001u);
}
// Lanes of all ones where bit 0 / bit 16 of b01 is set (b01 has no other bits).
__device__ __forceinline__ uint32_t p_spread(uint32_t b01) { return b01 * 0xffffu; }
// Lanes of all ones where the lane is negative, else zero: a byte permute that replicates
// the sign bit of byte 1 over bytes 0-1 and that of byte 3 over bytes 2-3.
__device__ __forceinline__ uint32_t p_signmask(uint32_t a) {
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, 0xBB99;" : "=r"(d) : "r"(a));
    return d;
}
// a negated in the lanes where mask is all ones (mask lanes 0 or 0xffff): (a ^ -1) + 1.
__device__ __forceinline__ uint32_t p_cneg(uint32_t a, uint32_t mask) {
    return p_add(a ^ mask, mask & 0x00010001u);
}

// Second sweep of a packed row: the row's sign parity is folded into the two candidate
// magnitudes once (n0, n1: min0 and min1 negated in the lanes whose parity is odd); per
// edge, |lambda| = min0 exactly where |lambda| - min0 - 1 is negative (|lambda| >= min0),
// that lane takes n1, the others n0, and lanes where lambda < 0 are negated (Observation 2).
struct PackedPick {
    uint32_t n0 = 0, n1 = 0, m0p1 = 0;  // m0p1 = -(min0 + 1) lane by lane
    __device__ __forceinline__ void set(uint32_t min0, uint32_t min1, uint32_t sx) {
        const uint32_t pm = p_signmask(sx);
        n0 = p_cneg(min0, pm);
        n1 = p_cneg(min1, pm);
        m0p1 = p_neg(p_add(min0, 0x00010001u));
    }
    // The same, picking the negated messages (-eta): the candidates negated once per row,
    // since the conditional negation of -x is minus that of x.
    __device__ __forceinline__ void set_neg(uint32_t min0, uint32_t min1, uint32_t sx) {
        const uint32_t pm = ~p_signmask(sx);
        n0 = p_cneg(min0, pm);
        n1 = p_cneg(min1, pm);
        m0p1 = p_neg(p_add(min0, 0x00010001u));
    }
    __device__ __forceinline__ uint32_t operator()(uint32_t lam) const {
        const uint32_t sm = p_signmask(lam);
        const uint32_t eq = p_signmask(p_add(p_cneg(lam, sm), m0p1));
        return p_cneg((n1 & eq) | (n0 & ~eq), sm);
    }
};

}  // namespace ldpc_impl
