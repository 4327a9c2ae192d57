// Training path of the learned (normalised / offset) Min-Sum decoder: an unrolled forward
// of T flooding iterations that keeps, per iteration, only the compressed state of every
// check (min0, min1, the first location of the minimum, the location of the second
// minimum, the sign parity, and one sign bit per edge), and the hand-written adjoint that
// rebuilds each iteration's messages from that state instead of storing them.
//
// Forward iteration t (1-based), per check i and frame (eq. eta_update with the learned
// magnitude): lambda_e = s_j - eta_e; m_e = min1 at the location of the minimum, else
// min0 (Observation 1); g_e = fma(alpha[t][c], m_e, -beta[t][c]) with c the class of bit j;
// eta_e = S_e * max(g_e, 0) with S_e the extrinsic sign (Observation 2); then per bit
// s_j = r_j + sum of eta in ascending row order (eq. lambda_j).
//
// Adjoint of iteration t, given ds^t (loss gradient w.r.t. s^t) and dlambda^(t+1):
//   deta_e = ds^t_j - dlambda^(t+1)_e               (eta_e feeds s^t_j and lambda^(t+1)_e)
//   dg_e = deta_e * S_e if g_e > 0 else 0           (signs are piecewise constant)
//   dalpha[t][c] += dg_e * m_e,  dbeta[t][c] -= dg_e
//   dm_e = dg_e * alpha[t][c] flows to the edge whose |lambda| is m_e: the minimum's
//   location for every other edge, the second minimum's location for the minimum itself
//   (a subgradient through min / argmin): dlambda^t = sign(lambda) * that sum, else 0;
//   ds^(t-1)_j = sum of dlambda^t over the edges of bit j.
// Layout: frame-interleaved, element (row/edge/bit x, frame f) at x * Fp + f; a warp
// covers 32 consecutive frames of one check or bit. The saved state of a check is min0,
// min1 and one word: for codes whose rows have at most 16 edges the word also holds the
// row's sign bits (loc | loc2 << 4 | parity << 8 | sign of lambda_k << (16 + k)), so each
// iteration keeps 12 bytes per check and frame; longer rows keep loc | loc2 << 8 |
// parity << 16 and one sign byte per edge.
#include <algorithm>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace {

using namespace ldpc_impl;

struct TrainWork {
    int32_t Fp;
    float *r, *s, *eta, *dlam, *ds;
    uint8_t* sg;     // [T][E][Fp] sign bit of lambda (rows of more than 16 edges only)
    float* mn0;      // [T][M][Fp]
    float* mn1;      // [T][M][Fp]
    uint32_t* info;  // [T][M][Fp]: the check's word (see above)
};

// Rows of at most 16 edges keep their sign bits in the check's word.
constexpr int kPackedSignsMaxRow = 16;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carve the workspace; returns the bytes needed (and fills w when base != nullptr).
size_t carve(int32_t M, int32_t N, int64_t E, int32_t F, int32_t T, bool packed, char* base,
             TrainWork* w) {
    const int32_t Fp = (F + 31) & ~31;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char* p = base ? base + o : nullptr;
        o += al256(bytes);
        return p;
    };
    char* r = take((size_t)N * Fp * 4);
    char* s = take((size_t)N * Fp * 4);
    char* eta = take((size_t)E * Fp * 4);
    char* dlam = take((size_t)E * Fp * 4);
    char* ds = take((size_t)N * Fp * 4);
    char* sg = packed ? nullptr : take((size_t)T * E * Fp);
    char* mn0 = take((size_t)T * M * Fp * 4);
    char* mn1 = take((size_t)T * M * Fp * 4);
    char* info = take((size_t)T * M * Fp * 4);
    if (w) {
        w->Fp = Fp;
        w->r = (float*)r;
        w->s = (float*)s;
        w->eta = (float*)eta;
        w->dlam = (float*)dlam;
        w->ds = (float*)ds;
        w->sg = (uint8_t*)sg;
        w->mn0 = (float*)mn0;
        w->mn1 = (float*)mn1;
        w->info = (uint32_t*)info;
    }
    return o;
}

// [F][N] -> [N][Fp] (and the copy into s); frames past F are zero. acc: add into dst.
__global__ void k_lw_in(const float* src, int F, int N, float* dst, float* dst2, int Fp,
                        int acc = 0) {
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int f = f0 + y, j = j0 + threadIdx.x;
        tile[y][threadIdx.x] = (f < F && j < N) ? src[(size_t)f * N + j] : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = j0 + y, f = f0 + threadIdx.x;
        if (j < N && f < Fp) {
            const size_t o = (size_t)j * Fp + f;
            dst[o] = acc ? dst[o] + tile[threadIdx.x][y] : tile[threadIdx.x][y];
            if (dst2) dst2[o] = tile[threadIdx.x][y];
        }
    }
}

// [N][Fp] -> [F][N]
__global__ void k_lw_out(const float* src, int Fp, int N, int F, float* dst) {
    __shared__ float tile[32][33];
    const int j0 = blockIdx.x * 32, f0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int j = j0 + y, f = f0 + threadIdx.x;
        tile[y][threadIdx.x] = (j < N && f < F) ? src[(size_t)j * Fp + f] : 0.0f;
    }
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += blockDim.y) {
        const int f = f0 + y, j = j0 + threadIdx.x;
        if (f < F && j < N) dst[(size_t)f * N + j] = tile[threadIdx.x][y];
    }
}

struct LwArgs {
    const int32_t *row_ptr, *col_idx, *col_ptr, *col_edge;
    const uint8_t* col_class;
    int32_t M, N, C, Fp;
    int64_t E;
    const float *alpha, *beta;  // [T][C]
};

// Forward check pass of iteration t with saving; block = 4 checks x 32 frames.
// PK: the row's sign bits go to its word (rows of at most 16 edges).
template <bool FIRST, bool PK>
__global__ void __launch_bounds__(128) k_lw_check(LwArgs a, TrainWork w, int t) {
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int f = blockIdx.y * 32 + (threadIdx.x & 31);
    if (i >= a.M) return;
    const int Fp = a.Fp;
    const int e0 = __ldg(a.row_ptr + i), d = __ldg(a.row_ptr + i + 1) - e0;
    uint8_t* sg = PK ? nullptr : w.sg + (size_t)(t - 1) * (size_t)a.E * Fp;
    float min0 = __int_as_float(0x7f800000), min1 = min0;
    int loc = 0, loc2 = 0;
    uint32_t par = 0, sgw = 0;
    for (int k = 0; k < d; k++) {
        const int e = e0 + k, c = __ldg(a.col_idx + e);
        const float lam = FIRST ? w.s[(size_t)c * Fp + f] : w.s[(size_t)c * Fp + f] - w.eta[(size_t)e * Fp + f];
        const float m = fabsf(lam);
        const uint32_t neg = lam < 0.0f;
        par ^= neg;
        if (PK) sgw |= neg << k;
        else sg[(size_t)e * Fp + f] = (uint8_t)neg;
        if (m < min0) {
            min1 = min0;
            loc2 = loc;
            min0 = m;
            loc = k;
        } else if (m < min1) {
            min1 = m;
            loc2 = k;
        }
    }
    const size_t ri = (size_t)(t - 1) * a.M * Fp + (size_t)i * Fp + f;
    w.mn0[ri] = min0;
    w.mn1[ri] = min1;
    w.info[ri] = PK ? (uint32_t)loc | ((uint32_t)loc2 << 4) | (par << 8) | (sgw << 16)
                    : (uint32_t)loc | ((uint32_t)loc2 << 8) | (par << 16);
    const float* al = a.alpha + (size_t)(t - 1) * a.C;
    const float* be = a.beta + (size_t)(t - 1) * a.C;
    for (int k = 0; k < d; k++) {
        const int e = e0 + k, cls = __ldg(a.col_class + __ldg(a.col_idx + e));
        const float g = __fmaf_rn(__ldg(al + cls), k == loc ? min1 : min0, -__ldg(be + cls));
        const float mag = g > 0.0f ? g : 0.0f;
        const uint32_t neg = PK ? (sgw >> k) & 1u : sg[(size_t)e * Fp + f];
        w.eta[(size_t)e * Fp + f] = (par ^ neg) ? -mag : mag;
    }
}

// Forward bit pass: s = r + sum of eta in ascending row order.
__global__ void __launch_bounds__(128) k_lw_var(LwArgs a, TrainWork w) {
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int f = blockIdx.y * 32 + (threadIdx.x & 31);
    if (j >= a.N) return;
    const int Fp = a.Fp;
    float acc = w.r[(size_t)j * Fp + f];
    for (int q = __ldg(a.col_ptr + j); q < __ldg(a.col_ptr + j + 1); q++)
        acc = acc + w.eta[(size_t)__ldg(a.col_edge + q) * Fp + f];
    w.s[(size_t)j * Fp + f] = acc;
}

// Adjoint of the check pass of iteration t; LAST: t = T (no dlambda^(t+1)).
template <bool LAST, bool PK>
__global__ void __launch_bounds__(128) k_lw_bwd_row(LwArgs a, TrainWork w, int t, int F,
                                                    float* grad_alpha, float* grad_beta) {
    extern __shared__ float gacc[];  // [2][C]
    for (int q = threadIdx.x; q < 2 * a.C; q += blockDim.x) gacc[q] = 0.0f;
    __syncthreads();
    const int i = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int f = blockIdx.y * 32 + (threadIdx.x & 31);
    const int Fp = a.Fp;
    if (i < a.M && f < F) {
        const int e0 = __ldg(a.row_ptr + i), d = __ldg(a.row_ptr + i + 1) - e0;
        const uint8_t* sg = PK ? nullptr : w.sg + (size_t)(t - 1) * (size_t)a.E * Fp;
        const size_t ri = (size_t)(t - 1) * a.M * Fp + (size_t)i * Fp + f;
        const float min0 = w.mn0[ri], min1 = w.mn1[ri];
        const uint32_t info = w.info[ri];
        const int loc = PK ? info & 0xf : info & 0xff, loc2 = PK ? (info >> 4) & 0xf : (info >> 8) & 0xff;
        const uint32_t par = (info >> (PK ? 8 : 16)) & 1u;
        auto neg_of = [&](int k, int e) -> uint32_t {  // sign bit of lambda of the row's k-th edge
            return PK ? (info >> (16 + k)) & 1u : sg[(size_t)e * Fp + f];
        };
        const float* al = a.alpha + (size_t)(t - 1) * a.C;
        const float* be = a.beta + (size_t)(t - 1) * a.C;
        float acc_loc = 0.0f, acc_loc2 = 0.0f;
        for (int k = 0; k < d; k++) {
            const int e = e0 + k, c = __ldg(a.col_idx + e);
            const int cls = __ldg(a.col_class + c);
            float deta = w.ds[(size_t)c * Fp + f];
            if (!LAST) deta -= w.dlam[(size_t)e * Fp + f];
            const float m = k == loc ? min1 : min0;
            const float alpha = __ldg(al + cls);
            const float g = __fmaf_rn(alpha, m, -__ldg(be + cls));
            if (g > 0.0f) {
                const float dg = (par ^ neg_of(k, e)) ? -deta : deta;
                atomicAdd(&gacc[cls], dg * m);
                atomicAdd(&gacc[a.C + cls], -dg);
                if (k != loc) acc_loc += dg * alpha;
                else acc_loc2 += dg * alpha;
            }
        }
        for (int k = 0; k < d; k++) {
            const int e = e0 + k;
            float v = 0.0f;
            if (k == loc) v = acc_loc;
            else if (k == loc2) v = acc_loc2;
            if (neg_of(k, e)) v = -v;  // d|lambda| / dlambda = sign(lambda), sign(0) = +1
            w.dlam[(size_t)e * Fp + f] = v;
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 2 * a.C; q += blockDim.x) {
        const float v = gacc[q];
        if (v != 0.0f) atomicAdd(q < a.C ? grad_alpha + (size_t)(t - 1) * a.C + q
                                         : grad_beta + (size_t)(t - 1) * a.C + (q - a.C), v);
    }
}

// ds^(t-1)_j = sum over the edges of bit j of dlambda^t.
__global__ void __launch_bounds__(128) k_lw_bwd_col(LwArgs a, TrainWork w, int F) {
    const int j = blockIdx.x * 4 + (threadIdx.x >> 5);
    const int f = blockIdx.y * 32 + (threadIdx.x & 31);
    if (j >= a.N) return;
    const int Fp = a.Fp;
    float acc = 0.0f;
    if (f < F)
        for (int q = __ldg(a.col_ptr + j); q < __ldg(a.col_ptr + j + 1); q++)
            acc += w.dlam[(size_t)__ldg(a.col_edge + q) * Fp + f];
    w.ds[(size_t)j * Fp + f] = acc;
}

bool packed_signs(const HandleView& v) { return v.dg->max_dc <= kPackedSignsMaxRow; }

int check_common(const HandleView& v, int32_t frames, int32_t iters, const void* alpha,
                 const void* beta, const void* work, uint64_t work_bytes) {
    if (frames <= 0 || iters <= 0 || frames > 65535 * 32) return LDPC_ERR_INVALID_ARG;
    if (!alpha || !beta || !work) return LDPC_ERR_BAD_POINTER;
    if (v.dg->n_classes <= 0 || v.dg->max_dc > 255) return LDPC_ERR_UNSUPPORTED;
    const size_t need = carve(v.M, v.N, v.E, frames, iters, packed_signs(v), nullptr, nullptr);
    if (work_bytes < need) return LDPC_ERR_INVALID_ARG;
    return LDPC_OK;
}

LwArgs make_args(const HandleView& v, int32_t Fp, const float* alpha, const float* beta) {
    LwArgs a;
    a.row_ptr = v.dg->row_ptr;
    a.col_idx = v.dg->col_idx;
    a.col_ptr = v.dg->col_ptr;
    a.col_edge = v.dg->col_edge;
    a.col_class = v.dg->col_class;
    a.M = v.M;
    a.N = v.N;
    a.C = v.dg->n_classes;
    a.Fp = Fp;
    a.E = v.E;
    a.alpha = alpha;
    a.beta = beta;
    return a;
}

}  // namespace

extern "C" {

int ldpc_train_workspace_size(ldpc_t* h, int32_t frames, int32_t iters, uint64_t* bytes) {
    HandleView v;
    if (handle_view(h, &v) != LDPC_OK || !bytes) return LDPC_ERR_BAD_POINTER;
    if (frames <= 0 || iters <= 0) return LDPC_ERR_INVALID_ARG;
    *bytes = carve(v.M, v.N, v.E, frames, iters, packed_signs(v), nullptr, nullptr);
    return LDPC_OK;
}

int ldpc_train_forward(ldpc_t* h, const float* llr, int32_t frames, int32_t iters,
                       const float* alpha, const float* beta, float* soft, int32_t soft_every,
                       void* work, uint64_t work_bytes) {
    HandleView v;
    if (handle_view(h, &v) != LDPC_OK || !llr || !soft) return LDPC_ERR_BAD_POINTER;
    int rc = check_common(v, frames, iters, alpha, beta, work, work_bytes);
    if (rc != LDPC_OK) return rc;
    TrainWork w;
    const bool pk = packed_signs(v);
    carve(v.M, v.N, v.E, frames, iters, pk, (char*)work, &w);
    const LwArgs a = make_args(v, w.Fp, alpha, beta);
    cudaStream_t st = v.stream;
    k_lw_in<<<dim3((v.N + 31) / 32, w.Fp / 32), dim3(32, 8), 0, st>>>(llr, frames, v.N, w.r, w.s, w.Fp);
    const dim3 gc((v.M + 3) / 4, w.Fp / 32), gv((v.N + 3) / 4, w.Fp / 32);
    const dim3 go((v.N + 31) / 32, (frames + 31) / 32), bo(32, 8);
    int launches = 1;
    for (int t = 1; t <= iters; t++) {
        if (pk) {
            if (t == 1) k_lw_check<true, true><<<gc, 128, 0, st>>>(a, w, t);
            else k_lw_check<false, true><<<gc, 128, 0, st>>>(a, w, t);
        } else {
            if (t == 1) k_lw_check<true, false><<<gc, 128, 0, st>>>(a, w, t);
            else k_lw_check<false, false><<<gc, 128, 0, st>>>(a, w, t);
        }
        k_lw_var<<<gv, 128, 0, st>>>(a, w);
        launches += 2;
        if (soft_every || t == iters) {
            k_lw_out<<<go, bo, 0, st>>>(w.s, w.Fp, v.N, frames,
                                        soft + (soft_every ? (size_t)(t - 1) * frames * v.N : 0));
            launches++;
        }
    }
    *v.last_launches = launches;
    return cudaGetLastError() == cudaSuccess ? LDPC_OK : LDPC_ERR_CUDA;
}

int ldpc_train_backward(ldpc_t* h, int32_t frames, int32_t iters, const float* alpha,
                        const float* beta, const float* grad_soft, int32_t soft_every,
                        float* grad_alpha, float* grad_beta, void* work, uint64_t work_bytes) {
    HandleView v;
    if (handle_view(h, &v) != LDPC_OK || !grad_soft || !grad_alpha || !grad_beta)
        return LDPC_ERR_BAD_POINTER;
    int rc = check_common(v, frames, iters, alpha, beta, work, work_bytes);
    if (rc != LDPC_OK) return rc;
    TrainWork w;
    const bool pk = packed_signs(v);
    carve(v.M, v.N, v.E, frames, iters, pk, (char*)work, &w);
    const LwArgs a = make_args(v, w.Fp, alpha, beta);
    cudaStream_t st = v.stream;
    const size_t gbytes = (size_t)iters * a.C * sizeof(float);
    if (cudaMemsetAsync(grad_alpha, 0, gbytes, st) != cudaSuccess ||
        cudaMemsetAsync(grad_beta, 0, gbytes, st) != cudaSuccess)
        return LDPC_ERR_CUDA;
    const dim3 gi((v.N + 31) / 32, w.Fp / 32), bi(32, 8);
    const size_t plane = (size_t)frames * v.N;
    // ds^T = the loss gradient of the last posteriors
    k_lw_in<<<gi, bi, 0, st>>>(grad_soft + (soft_every ? (size_t)(iters - 1) * plane : 0), frames,
                               v.N, w.ds, nullptr, w.Fp);
    const dim3 gc((v.M + 3) / 4, w.Fp / 32), gv((v.N + 3) / 4, w.Fp / 32);
    const size_t sm = 2 * a.C * sizeof(float);
    int launches = 1;
    for (int t = iters; t >= 1; t--) {
        auto row = t == iters ? (pk ? k_lw_bwd_row<true, true> : k_lw_bwd_row<true, false>)
                              : (pk ? k_lw_bwd_row<false, true> : k_lw_bwd_row<false, false>);
        row<<<gc, 128, sm, st>>>(a, w, t, frames, grad_alpha, grad_beta);
        launches++;
        if (t > 1) {
            k_lw_bwd_col<<<gv, 128, 0, st>>>(a, w, frames);  // ds^(t-1) through lambda^t
            launches++;
            if (soft_every) {  // plus the loss gradient of the posteriors of iteration t-1
                k_lw_in<<<gi, bi, 0, st>>>(grad_soft + (size_t)(t - 2) * plane, frames, v.N, w.ds,
                                           nullptr, w.Fp, 1);
                launches++;
            }
        }
    }
    *v.last_launches = launches;
    return cudaGetLastError() == cudaSuccess ? LDPC_OK : LDPC_ERR_CUDA;
}

}  // extern "C"
