// Compressed check messages of the streaming variant (padded row layout, FP32 mode).
//
// Every message a check sends in one iteration follows from four things (Section III,
// Observations 1 and 2): the two smallest magnitudes min0 <= min1 of the row's lambdas,
// the first location of min0, and per edge the sign (the row's sign parity XOR the sign
// of that edge's lambda). So a row of d <= 16 edges keeps, per frame,
//   m0 = min0, m1 = min1 (binary32), and
//   w  = bit t set for the edge holding min0 (t < 16) | sign of the message to edge t at
//        bit 16 + t,
// and the message to edge t is +-(bit t of w ? m1 : m0), with the magnitude weighted in the
// learned decoder (max(fma(alpha, m, -beta), 0), alpha and beta of the class of edge t's
// bit). Twelve bytes per row and frame replace four bytes per message slot (8 or 16 per
// row); the arrays are frame-interleaved like every streaming array, element (row i,
// position p) at i Fp + p.
#pragma once

#include <stdint.h>

namespace ldpc_impl {

struct CState {
    float* m0;    // [M][Fp]
    float* m1;    // [M][Fp]
    uint32_t* w;  // [M][Fp]
};

// The three arrays laid out one after the other from `base` (12 M Fp bytes).
__host__ __device__ inline CState cstate_at(void* base, int64_t M, int64_t Fp) {
    float* m0 = static_cast<float*>(base);
    return CState{m0, m0 + M * Fp, reinterpret_cast<uint32_t*>(m0 + 2 * M * Fp)};
}

// Magnitude of the message to edge t (before any weighting).
__device__ __forceinline__ float cmsg_mag(float m0, float m1, uint32_t w, int t) {
    return ((w >> t) & 1u) ? m1 : m0;
}

// The message to edge t: magnitude m (>= 0) with the sign kept at bit 16 + t of w.
__device__ __forceinline__ float cmsg_signed(float m, uint32_t w, int t) {
    return __uint_as_float(__float_as_uint(m) | ((w << (15 - t)) & 0x80000000u));
}

// Learned weighting of a magnitude: max(fma(alpha, m, -beta), 0) in binary32.
__device__ __forceinline__ float cmsg_weight(float m, float wa, float wb) {
    const float x = __fmaf_rn(wa, m, -wb);
    return x > 0.0f ? x : 0.0f;
}

}  // namespace ldpc_impl
