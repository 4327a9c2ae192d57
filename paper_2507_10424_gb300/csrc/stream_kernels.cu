// Streaming variant: edge messages eta live in HBM in a frame-interleaved
// structure-of-arrays layout, element (edge e, frame f) at e * Fp + f. A thread owns V
// consecutive frames (one 16-byte vector: 4 x fp32 or 8 x int16) of one row or column,
// so each warp moves 512 contiguous bytes per edge whatever the structure of H.
//
// Per flooding iteration k (Algorithm 1):
//   k_check: for every check i and frame: lambda_e = s_j - eta_e (eq. eta_update with
//            eta^prev), Observation 1 (min0, first location, min1) and Observation 2 (sign
//            product as XOR), then eta_e = +-(min1 at the location, min0 elsewhere).
//            The same pass XORs the hard decisions of the gathered s_j: that is the
//            syndrome of the previous iteration's decision (eq. 1-2).
//   k_var:   for every bit j and frame: s_j = r_j + sum of eta over M_j, ascending rows
//            (eq. lambda_j); frames whose previous syndrome was zero are frozen there.
// A final syndrome-only pass gives the status of frames that never stopped early.
#include "../../include/ldpc.h"
#include "ldpc_internal.h"

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

// ------------------------------------------------------------------------------------
// Per-frame state
// ------------------------------------------------------------------------------------
__global__ void k_init_state(uint8_t* state, int32_t* done_iter, int Fp, int frames) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f < Fp) {
        state[f] = f < frames;
        done_iter[f] = -1;
    }
}

// llr [frames][N] (frame-major) -> r, s [N][Fp] (frame-interleaved); 32 x 32 tiles.
template <int MODE>
__global__ void k_load(const void* llr, int llr_i8, int frames, int N, typename Tr<MODE>::R* r,
                       typename Tr<MODE>::T* s, int Fp) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int f = f0 + y, j = j0 + threadIdx.x;
        float v = 0.0f;
        if (f < frames && j < N) {
            size_t idx = (size_t)f * N + j;
            v = llr_i8 ? (float)((const int8_t*)llr)[idx] : ((const float*)llr)[idx];
        }
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int j = j0 + y, f = f0 + threadIdx.x;
        if (j < N && f < Fp) {
            float v = tile[threadIdx.x][y];
            size_t idx = (size_t)j * Fp + f;
            if (MODE == kModeFP32) {
                r[idx] = (R)v;
                s[idx] = (T)v;
            } else {
                int8_t q = llr_i8 ? (int8_t)v : quantize(v);
                r[idx] = (R)q;
                s[idx] = (T)q;
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
    if (do_syn) {
        z &= act;
        if (z) {
#pragma unroll
            for (int v = 0; v < V; v++)
                if ((z >> v) & 1) unsat[f0 + v] = 1;
        }
    }
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
// Variable-node pass. Block = 4 warps = 4 columns; lane = one frame vector.
// test_prev: the previous decision's syndrome (in unsat) decides whether a frame stops.
// ------------------------------------------------------------------------------------
template <int MODE, int VW = Tr<MODE>::V>
__global__ void __launch_bounds__(128) k_var(const int32_t* __restrict__ col_ptr,
                                             const int32_t* __restrict__ col_edge, int N,
                                             const typename Tr<MODE>::R* __restrict__ r,
                                             typename Tr<MODE>::T* s,
                                             const typename Tr<MODE>::T* __restrict__ eta, int Fp,
                                             uint8_t* state, int32_t* done_iter,
                                             const uint8_t* __restrict__ unsat, int test_prev,
                                             int k, int* n_done, int frames) {
    using T = typename Tr<MODE>::T;
    using R = typename Tr<MODE>::R;
    using A = typename Tr<MODE>::A;
    constexpr int V = VW;
    using VT = Vec<T, V>;
    using VR = Vec<R, V>;
    using VS = Vec<uint8_t, V>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int j = blockIdx.x * 4 + warp;
    const int f0 = (blockIdx.y * 32 + lane) * V;
    if (j >= N) return;
    if (*(volatile const int*)n_done >= frames) return;
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
                    done_iter[f0 + v] = k - 1;
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
    for (int t = t0; t < t1; t++) {
        const int e = __ldg(col_edge + t);
        const VT ev = *reinterpret_cast<const VT*>(eta + (size_t)e * Fp + f0);
#pragma unroll
        for (int v = 0; v < V; v++) acc[v] = acc[v] + (A)ev.x[v];
    }
    T* sp = s + (size_t)j * Fp + f0;
    if (upd == (1u << V) - 1u) {
        VT out;
#pragma unroll
        for (int v = 0; v < V; v++) {
            if (MODE == kModeFP32) out.x[v] = (T)acc[v];
            else out.x[v] = (T)sat16((int32_t)acc[v]);
        }
        *reinterpret_cast<VT*>(sp) = out;
    } else {
#pragma unroll
        for (int v = 0; v < V; v++)
            if ((upd >> v) & 1) sp[v] = (MODE == kModeFP32) ? (T)acc[v] : (T)sat16((int32_t)acc[v]);
    }
}

// s [N][Fp] -> bits (and soft) [frames][N]; 32 x 32 tiles.
template <int MODE>
__global__ void k_store(const typename Tr<MODE>::T* s, int Fp, int N, int frames, uint8_t* bits,
                        float* soft, int paper) {
    using A = typename Tr<MODE>::A;
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int j = j0 + y, f = f0 + threadIdx.x;
        float v = 0.0f;
        if (j < N && f < frames) v = (float)s[(size_t)j * Fp + f];
        tile[y][threadIdx.x] = v;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        int f = f0 + y, j = j0 + threadIdx.x;
        if (f < frames && j < N) {
            float v = tile[threadIdx.x][y];  // exact for fp32 and int16 values
            size_t idx = (size_t)f * N + j;
            bits[idx] = (uint8_t)slice((A)v, paper);
            if (soft) soft[idx] = (MODE == kModeFP32) ? v : v * 0.25f;
        }
    }
}

__global__ void k_finish(const int32_t* done_iter, const uint8_t* unsat_final, int frames, int L,
                         int32_t* out_iters, uint8_t* out_ok) {
    int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= frames) return;
    int d = done_iter[f];
    out_iters[f] = d >= 0 ? d : L;
    if (out_ok) out_ok[f] = d >= 0 ? 1 : (unsat_final[f] == 0);
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
    k_init_state<<<(Fp + 255) / 256, 256, 0, st>>>(state, w.done_iter, Fp, a.frames);
    launches++;
    k_load<MODE><<<dim3((a.N + 31) / 32, Fp / 32), dim3(32, 8), 0, st>>>(a.llr, a.llr_is_i8, a.frames,
                                                                        a.N, r, s, Fp);
    launches++;
    const dim3 gc((a.M + 3) / 4, Fp / (32 * V)), gv((a.N + 3) / 4, Fp / (32 * V));
    for (int k = 1; k <= a.L; k++) {
        const int test_prev = a.early_stop && ((k - 1) % a.check_every == 0);
        uint8_t* un = w.unsat + (size_t)k * Fp;
        if (MODE == kModeFP32 && a.w_rows > 0) {
            const int row = (k < a.w_rows ? k : a.w_rows) - 1;
            const IterWeights wt{g.col_class, a.w_alpha + (size_t)row * a.n_classes,
                                 a.w_beta + (size_t)row * a.n_classes};
            if (k == 1)
                k_check<MODE, true, false, true, V><<<gc, 128, 0, st>>>(
                    g.row_ptr, g.col_idx, a.M, s, eta, Fp, state, un, test_prev, w.n_done, a.frames,
                    a.paper_slicer, wt);
            else
                k_check<MODE, false, false, true, V><<<gc, 128, 0, st>>>(
                    g.row_ptr, g.col_idx, a.M, s, eta, Fp, state, un, test_prev, w.n_done, a.frames,
                    a.paper_slicer, wt);
        } else if (k == 1)
            k_check<MODE, true, false, false, V><<<gc, 128, 0, st>>>(g.row_ptr, g.col_idx, a.M, s, eta, Fp,
                                                           state, un, test_prev, w.n_done,
                                                           a.frames, a.paper_slicer);
        else
            k_check<MODE, false, false, false, V><<<gc, 128, 0, st>>>(g.row_ptr, g.col_idx, a.M, s, eta, Fp,
                                                            state, un, test_prev, w.n_done,
                                                            a.frames, a.paper_slicer);
        k_var<MODE, V><<<gv, 128, 0, st>>>(g.col_ptr, g.col_edge, a.N, r, s, eta, Fp, state,
                                        w.done_iter, un, test_prev, k, w.n_done, a.frames);
        launches += 2;
    }
    uint8_t* unf = w.unsat + (size_t)(a.L + 1) * Fp;
    k_check<MODE, false, true, false, V><<<gc, 128, 0, st>>>(g.row_ptr, g.col_idx, a.M, s, eta, Fp, state,
                                                   unf, 1, w.n_done, a.frames, a.paper_slicer);
    // (the final pass returns at once when every frame has stopped: their status is known)
    k_store<MODE><<<dim3((a.N + 31) / 32, (a.frames + 31) / 32), dim3(32, 8), 0, st>>>(
        s, Fp, a.N, a.frames, a.out_bits, a.out_soft, a.paper_slicer);
    k_finish<<<(a.frames + 255) / 256, 256, 0, st>>>(w.done_iter, unf, a.frames, a.L, a.out_iters,
                                                     a.out_ok);
    launches += 3;
    if (cudaGetLastError() != cudaSuccess) return LDPC_ERR_CUDA;
    return launches;
}

}  // namespace

size_t stream_bytes(int mode, int32_t N, int64_t E, int32_t Fp, int32_t L) {
    size_t tb = mode == kModeFP32 ? 4 : 2, rb = mode == kModeFP32 ? 4 : 1;
    return (size_t)E * Fp * tb + (size_t)N * Fp * (tb + rb) + (size_t)Fp * 5 + (size_t)(L + 2) * Fp + 256;
}

StreamWork stream_carve(int mode, void* mem, int32_t N, int64_t E, int32_t Fp, int32_t L) {
    // Fp is a multiple of 256, so every region below starts 256-byte aligned
    const size_t tb = mode == kModeFP32 ? 4 : 2, rb = mode == kModeFP32 ? 4 : 1;
    char* p = (char*)mem;
    StreamWork w;
    w.Fp = Fp;
    w.eta = p;
    p += (size_t)E * Fp * tb;
    w.s = p;
    p += (size_t)N * Fp * tb;
    w.r = p;
    p += (size_t)N * Fp * rb;
    w.done_iter = (int32_t*)p;
    p += (size_t)Fp * 4;
    w.state = (uint8_t*)p;
    p += (size_t)Fp;
    w.unsat = (uint8_t*)p;
    p += (size_t)(L + 2) * Fp;
    w.n_done = (int32_t*)p;
    return w;
}

int stream_decode(int mode, const DevGraph& g, const DecodeArgs& a, const StreamWork& w,
                  cudaStream_t st, int vw) {
    // vw: frames per lane (0 = the 16-byte vector of the mode); w.Fp is a multiple of 32 vw.
    if (mode == kModeFP32) {
        switch (vw) {
            case 1: return run<kModeFP32, 1>(g, a, w, st);
            case 2: return run<kModeFP32, 2>(g, a, w, st);
            case 0:
            case Tr<kModeFP32>::V: return run<kModeFP32, Tr<kModeFP32>::V>(g, a, w, st);
            default: return LDPC_ERR_INVALID_ARG;
        }
    }
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
