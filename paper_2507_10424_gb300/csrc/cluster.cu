// Cluster variant: codes whose messages do not fit one SM's shared memory are decoded by
// a thread-block cluster of C CTAs that keeps one tile of FT frames on chip across its C
// SMs (distributed shared memory). Algorithm 1's flooding iterations run as in the
// resident variant, with the rows and columns split between the cluster's CTAs:
//   CTA q holds, for the FT interleaved frames of the tile,
//     eta[row slot]      the messages of its own rows (sliced layout of its rows),
//     s[position], r[position]   posteriors and channel values of its own columns;
//   phase A (its rows): lambda = s - eta with s gathered from the column owners' shared
//     memory, Observation 1 (min0, min1) and Observation 2 (XOR of sign bits), then the
//     new messages, written locally; the sweep XORs the decisions of the gathered s (the
//     syndrome, eq. 1-2) into a per-CTA word;
//   phase B (its columns): s = r + the column's messages in ascending row order, gathered
//     from the row owners' shared memory (eq. lambda_j).
// Cluster barriers separate the phases. The early-stop test ORs the C syndrome words, so
// every CTA takes the same decision. Channel values are read once and decisions written
// once per frame, each CTA for its own columns.
#include <cooperative_groups.h>

#include "resident.cuh"

namespace ldpc_impl {
namespace clusterv {
using namespace resident;
namespace cg = cooperative_groups;

constexpr int kClThreads = 1024;

struct ClArgs {
    const int32_t* meta;
    const int32_t* r_base;
    const uint8_t* r_deg;
    const uint32_t* r_ref;
    const uint8_t* r_cls;
    const int32_t* c_base;
    const uint8_t* c_deg;
    const uint32_t* c_ref;
    const uint16_t* pos_of_col;
    int32_t E_cap, P_cap, N;
    int32_t w_rows, n_classes;  // learned weights (FP32), w_rows = 0: plain Min-Sum
    const float* w_alpha;
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

// Byte offsets of eta, s and r in every CTA's shared memory (identical across the cluster,
// so one offset addresses the same array in any CTA).
struct ClLayout {
    uint32_t eta, s, r, total;
};
__host__ __device__ inline ClLayout cl_layout(int vec_bytes, int E_cap, int P_cap) {
    ClLayout L;
    L.eta = 0;
    L.s = al16((uint32_t)E_cap * vec_bytes);
    L.r = L.s + al16((uint32_t)P_cap * vec_bytes);
    L.total = L.r + al16((uint32_t)P_cap * vec_bytes);
    return L;
}

template <int MODE>
__device__ __forceinline__ typename RT<MODE>::A cl_chan(const ClArgs& a, size_t idx) {
    if (MODE == kModeFP32) return __ldg((const float*)a.llr + idx);
    if (a.llr_i8) return (int32_t)__ldg((const int8_t*)a.llr + idx);
    return (int32_t)rquant(__ldg((const float*)a.llr + idx));
}

// The entry `ref` = (rank << 16) | index of an array that sits at `local` in this CTA and
// at the same offset in every CTA of the cluster.
template <typename VT>
__device__ __forceinline__ VT cl_load(const cg::cluster_group& cl, VT* local, uint32_t ref) {
    return *cl.map_shared_rank(local + (ref & 0xffffu), ref >> 16);
}

struct Part {  // this CTA's part of the layout
    int j0, j1, n_rtasks, n_ctasks;
    const int32_t* r_base;
    const uint8_t* r_deg;
    const uint32_t* r_ref;
    const uint8_t* r_cls;
    const int32_t* c_base;
    const uint8_t* c_deg;
    const uint32_t* c_ref;
};

// Phase A over this CTA's rows; same sweeps as the resident variant (min1 where |lambda|
// equals min0, so the first location needs no tracking), with s gathered across the cluster.
template <int MODE, int FT, bool FIRST, bool SYN, bool UPD, bool PAPER, bool W>
__device__ __forceinline__ void cl_phase_a(const cg::cluster_group& cl, const Part& pt,
                                           VecR<typename RT<MODE>::T, FT>* eta,
                                           VecR<typename RT<MODE>::T, FT>* s, const float* walpha,
                                           const float* wbeta, uint32_t* unsat_w) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    constexpr int UNR = FT >= 4 ? 2 : 4;
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int task = snake(k, nth);
        if (task >= pt.n_rtasks) break;
        const int d = pt.r_deg[task];
        if (d == 0) continue;
        const int base = pt.r_base[task >> 5] + (task & 31);
        A min0[FT], min1[FT];
        uint32_t sx[FT], zx[FT];
#pragma unroll
        for (int f = 0; f < FT; f++) {
            min0[f] = rbig(A());
            min1[f] = rbig(A());
            sx[f] = 0;
            zx[f] = 0;
        }
#pragma unroll UNR
        for (int t = 0; t < d; t++) {
            const int slot = base + 32 * t;
            const VT sv = cl_load(cl, s, __ldg(pt.r_ref + slot));
            if (SYN) {
#pragma unroll
                for (int f = 0; f < FT; f++) zx[f] ^= dec_bits<PAPER>((A)sv.x[f]);
            }
            if (UPD) {
                VT ev;
                if (!FIRST) ev = eta[slot];
                VT lv;
#pragma unroll
                for (int f = 0; f < FT; f++) {
                    const A lam = FIRST ? (A)sv.x[f] : lam_sat((A)sv.x[f], (A)ev.x[f]);
                    const A m = rabs(lam);
                    min1[f] = min(min1[f], max(min0[f], m));
                    min0[f] = min(min0[f], m);
                    sx[f] ^= bits_of(lam);
                    lv.x[f] = (T)lam;
                }
                eta[slot] = lv;  // stash lambda for sweep 2
            }
        }
        if (SYN) {
            uint32_t z = 0;
#pragma unroll
            for (int f = 0; f < FT; f++) z |= (zx[f] >> 31) << f;
            if (z) atomicOr(unsat_w, z);
        }
        if (UPD) {
#pragma unroll UNR
            for (int t = 0; t < d; t++) {
                const int slot = base + 32 * t;
                const VT lv = eta[slot];
                float wa = 1.0f, wb = 0.0f;
                if constexpr (W) {
                    const int c = __ldg(pt.r_cls + slot);
                    wa = __ldg(walpha + c);
                    wb = __ldg(wbeta + c);
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
                eta[slot] = out;
            }
        }
    }
}

template <int MODE, int FT, bool PAPER, bool W>
__device__ __forceinline__ void cl_phase_a_any(bool first, bool syn, bool upd,
                                               const cg::cluster_group& cl, const Part& pt,
                                               VecR<typename RT<MODE>::T, FT>* eta,
                                               VecR<typename RT<MODE>::T, FT>* s,
                                               const float* wa, const float* wb, uint32_t* uw) {
#define LDPC_CL_PHASE_A(F, S, U) cl_phase_a<MODE, FT, F, S, U, PAPER, W>(cl, pt, eta, s, wa, wb, uw)
    if (first) {
        if (!upd) LDPC_CL_PHASE_A(true, true, false);
        else if (syn) LDPC_CL_PHASE_A(true, true, true);
        else LDPC_CL_PHASE_A(true, false, true);
    } else {
        if (!upd) LDPC_CL_PHASE_A(false, true, false);
        else if (syn) LDPC_CL_PHASE_A(false, true, true);
        else LDPC_CL_PHASE_A(false, false, true);
    }
#undef LDPC_CL_PHASE_A
}

// Phase B over this CTA's column positions, messages gathered across the cluster.
template <int MODE, int FT>
__device__ __forceinline__ void cl_phase_b(const cg::cluster_group& cl, const Part& pt,
                                           VecR<typename RT<MODE>::T, FT>* eta,
                                           VecR<typename RT<MODE>::T, FT>* s,
                                           const VecR<typename RT<MODE>::T, FT>* r) {
    using T = typename RT<MODE>::T;
    using A = typename RT<MODE>::A;
    using VT = VecR<T, FT>;
    const int nth = blockDim.x;
    for (int k = 0;; k++) {
        const int p = snake(k, nth);
        if (p >= pt.n_ctasks) break;
        const int d = pt.c_deg[p];
        if (d == 0) continue;  // padding, or a bit in no check: s stays r
        const int base = pt.c_base[p >> 5] + (p & 31);
        const VT rv = r[p];
        A acc[FT];
#pragma unroll
        for (int f = 0; f < FT; f++) acc[f] = (A)rv.x[f];
#pragma unroll 4
        for (int t = 0; t < d; t++) {
            const VT ev = cl_load(cl, eta, __ldg(pt.c_ref + base + 32 * t));
#pragma unroll
            for (int f = 0; f < FT; f++) acc[f] = acc[f] + (A)ev.x[f];
        }
        VT out;
#pragma unroll
        for (int f = 0; f < FT; f++) out.x[f] = (T)rsat_out(acc[f]);
        s[p] = out;
    }
}

// Decisions (and posteriors) of this CTA's columns for the frames in `mask`; rank 0 also
// writes the iteration counts and statuses.
template <int MODE, int FT>
__device__ __forceinline__ void cl_emit(const ClArgs& a, const Part& pt, int rank,
                                        const VecR<typename RT<MODE>::T, FT>* s, int fbase,
                                        uint32_t mask, int iters, uint32_t okm) {
    using A = typename RT<MODE>::A;
    const int N = a.N;
    for (int j = pt.j0 + (int)threadIdx.x; j < pt.j1; j += blockDim.x) {
        const auto v = s[a.pos_of_col[j]];
#pragma unroll
        for (int f = 0; f < FT; f++) {
            if (!((mask >> f) & 1u)) continue;
            const size_t o = (size_t)(fbase + f) * N + j;
            const A x = (A)v.x[f];
            a.out_bits[o] = (uint8_t)rslice(x, a.paper);
            if (a.out_soft) a.out_soft[o] = (MODE == kModeFP32) ? (float)x : (float)x * 0.25f;
        }
    }
    if (rank == 0) {
#pragma unroll
        for (int f = 0; f < FT; f++)
            if (threadIdx.x == f && ((mask >> f) & 1u)) {
                a.out_iters[fbase + f] = iters;
                if (a.out_ok) a.out_ok[fbase + f] = (okm >> f) & 1u;
            }
    }
}

// Persistent: rank 0 of each cluster takes tiles from the work counter. Every branch that
// decides whether a cluster barrier is reached depends only on values all CTAs of the
// cluster share (tile number, iteration, the ORed syndrome words), so the CTAs reach the
// same barriers.
template <int MODE, int FT, bool PAPER, bool W>
__global__ void __launch_bounds__(kClThreads, 1) k_cluster(const ClArgs a) {
    using T = typename RT<MODE>::T;
    using VT = VecR<T, FT>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t unsat_w[2];
    __shared__ uint32_t unsat_all;
    __shared__ int tile_sh;
    const cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank(), C = (int)cl.num_blocks();
    const ClLayout lay = cl_layout((int)sizeof(VT), a.E_cap, a.P_cap);
    VT* eta = reinterpret_cast<VT*>(smem_raw + lay.eta);
    VT* s = reinterpret_cast<VT*>(smem_raw + lay.s);
    VT* r = reinterpret_cast<VT*>(smem_raw + lay.r);
    const int32_t* m = a.meta + rank * kClMeta;
    Part pt;
    pt.j0 = m[kClJ0];
    pt.j1 = m[kClJ1];
    pt.n_rtasks = m[kClRTasks];
    pt.n_ctasks = m[kClCTasks];
    pt.r_base = a.r_base + m[kClRBase];
    pt.r_deg = a.r_deg + m[kClRDeg];
    pt.r_ref = a.r_ref + m[kClRRef];
    pt.r_cls = a.r_cls + m[kClRRef];
    pt.c_base = a.c_base + m[kClCBase];
    pt.c_deg = a.c_deg + m[kClCDeg];
    pt.c_ref = a.c_ref + m[kClCRef];
    const int N = a.N;

    for (;;) {
        if (rank == 0 && threadIdx.x == 0) tile_sh = atomicAdd(a.tile_counter, 1);
        cl.sync();
        const int tile = *cl.map_shared_rank(&tile_sh, 0);
        cl.sync();  // every CTA has read the tile number before rank 0 may leave or reuse it
        if (tile >= a.n_tiles) break;
        const int fbase = tile * FT, nf = min(FT, a.frames - fbase);
        for (int j = pt.j0 + (int)threadIdx.x; j < pt.j1; j += blockDim.x) {
            VT v;
#pragma unroll
            for (int f = 0; f < FT; f++)  // "+ 0" turns -0.0 into +0.0 and changes no other value
                v.x[f] = f < nf ? (T)(cl_chan<MODE>(a, (size_t)(fbase + f) * N + j) + 0) : T(0);
            const int p = a.pos_of_col[j];
            s[p] = v;
            r[p] = v;
        }
        if (threadIdx.x == 0) {
            unsat_w[0] = 0;
            unsat_w[1] = 0;
        }
        uint32_t active = (1u << nf) - 1u;
        cl.sync();  // every posterior of the tile is in place before any CTA gathers

        for (int k = 0;; k++) {
            const int par = k & 1;
            const bool last = (k == a.L);
            const bool syn = last || (a.early_stop && (k % a.check_every == 0));
            const float* wa = nullptr;
            const float* wb = nullptr;
            if (W) {  // weights of iteration k + 1 (the last row serves the later iterations)
                const int row = min(k + 1, a.w_rows) - 1;
                wa = a.w_alpha + row * a.n_classes;
                wb = a.w_beta + row * a.n_classes;
            }
            cl_phase_a_any<MODE, FT, PAPER, W>(k == 0, syn, !last, cl, pt, eta, s, wa, wb,
                                               &unsat_w[par]);
            cl.sync();
            if (syn) {
                if (threadIdx.x < 32) {
                    uint32_t v = (int)threadIdx.x < C ? *cl.map_shared_rank(&unsat_w[par], threadIdx.x) : 0u;
                    v = __reduce_or_sync(0xffffffffu, v);
                    if (threadIdx.x == 0) unsat_all = v;
                }
                __syncthreads();
                const uint32_t conv = active & ~unsat_all;
                if (last) {
                    cl_emit<MODE, FT>(a, pt, rank, s, fbase, active, a.L, conv);
                    break;
                }
                if (conv) {
                    cl_emit<MODE, FT>(a, pt, rank, s, fbase, conv, k, conv);
                    active &= ~conv;
                    if (!active) break;
                    __syncthreads();  // the emitted posteriors are read before phase B rewrites them
                }
            }
            cl_phase_b<MODE, FT>(cl, pt, eta, s, r);
            if (threadIdx.x == 0) unsat_w[par ^ 1] = 0;
            cl.sync();
        }
    }
}

template <int MODE, int FT, bool PAPER, bool W>
int launch(const ClArgs& ca, const ClusterPlan& p, cudaStream_t st, int* clusters_out) {
    auto kern = k_cluster<MODE, FT, PAPER, W>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    if (p.C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess)
        return LDPC_ERR_CUDA;
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.blockDim = dim3((unsigned)p.threads);
    cfg.dynamicSmemBytes = p.smem;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (clusters_out) {  // query only: how many clusters fit on the device at once
        cfg.gridDim = dim3((unsigned)p.C);
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
            cudaGetLastError();
            n = 0;
        }
        *clusters_out = n;
        return LDPC_OK;
    }
    const int clusters = std::max(1, std::min(ca.n_tiles, p.clusters));
    cfg.gridDim = dim3((unsigned)(clusters * p.C));
    if (cudaLaunchKernelEx(&cfg, kern, ca) != cudaSuccess) return LDPC_ERR_CUDA;
    return 1;
}

template <int MODE, bool PAPER, bool W>
int launch_ft(const ClArgs& ca, const ClusterPlan& p, cudaStream_t st, int* q) {
    switch (p.FT) {
        case 1: return launch<MODE, 1, PAPER, W>(ca, p, st, q);
        case 2: return launch<MODE, 2, PAPER, W>(ca, p, st, q);
        case 4: return launch<MODE, 4, PAPER, W>(ca, p, st, q);
    }
    return LDPC_ERR_INVALID_ARG;
}

int dispatch(int mode, const ClArgs& ca, const ClusterPlan& p, cudaStream_t st, int* q) {
    if (mode == kModeFP32) {
        if (ca.w_rows > 0)
            return ca.paper ? launch_ft<kModeFP32, true, true>(ca, p, st, q)
                            : launch_ft<kModeFP32, false, true>(ca, p, st, q);
        return ca.paper ? launch_ft<kModeFP32, true, false>(ca, p, st, q)
                        : launch_ft<kModeFP32, false, false>(ca, p, st, q);
    }
    return ca.paper ? launch_ft<kModeFixed, true, false>(ca, p, st, q)
                    : launch_ft<kModeFixed, false, false>(ca, p, st, q);
}

}  // namespace clusterv

using namespace clusterv;

ClusterPlan cluster_plan(int mode, const DevCluster& dc, int FT, int threads, int w_entries) {
    ClusterPlan p;
    if (!dc.C) return p;
    int device = 0, optin = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return p;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const size_t budget = (size_t)std::max(0, optin - 256);  // static shared memory
    const int tb = mode == kModeFP32 ? 4 : 2;
    if (threads && (threads % 32 || threads < 64 || threads > kClThreads)) return p;
    const int fts[] = {4, 2, 1};
    for (int ft : fts) {
        if (FT && ft != FT) continue;
        if (ft * tb > 16) continue;
        const ClLayout L = cl_layout(ft * tb, dc.E_cap, dc.P_cap);
        if (L.total > budget) continue;
        ClusterPlan c;
        c.ok = 1;
        c.C = dc.C;
        c.FT = ft;
        c.threads = threads ? threads : kClThreads;
        c.smem = L.total;
        ClArgs q{};
        q.w_rows = (mode == kModeFP32 && w_entries > 0) ? 1 : 0;
        int n = 0;
        dispatch(mode, q, c, nullptr, &n);
        if (n < 1) continue;
        c.clusters = n;
        return c;
    }
    return p;
}

int cluster_decode(int mode, const DevCluster& dc, const ClusterPlan& p, const DecodeArgs& a,
                   int32_t* tile_counter, cudaStream_t st) {
    if (!p.ok) return LDPC_ERR_UNSUPPORTED;
    ClArgs ca;
    ca.meta = dc.meta;
    ca.r_base = dc.r_base;
    ca.r_deg = dc.r_deg;
    ca.r_ref = dc.r_ref;
    ca.r_cls = dc.r_cls;
    ca.c_base = dc.c_base;
    ca.c_deg = dc.c_deg;
    ca.c_ref = dc.c_ref;
    ca.pos_of_col = dc.pos_of_col;
    ca.E_cap = dc.E_cap;
    ca.P_cap = dc.P_cap;
    ca.N = a.N;
    ca.w_rows = mode == kModeFP32 ? a.w_rows : 0;
    ca.n_classes = a.n_classes;
    ca.w_alpha = a.w_alpha;
    ca.w_beta = a.w_beta;
    ca.llr = a.llr;
    ca.llr_i8 = a.llr_is_i8;
    ca.frames = a.frames;
    ca.n_tiles = (a.frames + p.FT - 1) / p.FT;
    ca.L = a.L;
    ca.early_stop = a.early_stop;
    ca.check_every = a.check_every;
    ca.paper = a.paper_slicer;
    ca.out_bits = a.out_bits;
    ca.out_iters = a.out_iters;
    ca.out_ok = a.out_ok;
    ca.out_soft = a.out_soft;
    ca.tile_counter = tile_counter;
    if (cudaMemsetAsync(tile_counter, 0, sizeof(int32_t), st) != cudaSuccess) return LDPC_ERR_CUDA;
    return dispatch(mode, ca, p, st, nullptr);
}

}  // namespace ldpc_impl
