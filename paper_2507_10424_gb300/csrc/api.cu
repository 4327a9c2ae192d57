// C ABI of the decoder: handle life cycle, argument checks, workspace, dispatch to the
// resident or streaming kernels, and the host-buffer pipeline.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

using namespace ldpc_impl;

namespace {
thread_local int g_last_error = LDPC_OK;
thread_local int g_last_cuda = 0;

int fail(int status) {
    g_last_error = status;
    return status;
}
int cuda_fail(cudaError_t e) {
    g_last_cuda = (int)e;
    return fail(LDPC_ERR_CUDA);
}
// A failed allocation: clear the runtime's pending error (else the next successful call
// would report it) and map it to a status.
int alloc_fail(cudaError_t e) {
    cudaGetLastError();
    g_last_cuda = (int)e;
    return fail(e == cudaErrorMemoryAllocation ? LDPC_ERR_OOM : LDPC_ERR_CUDA);
}
#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

template <typename T>
int upload(T** dst, const T* src, size_t n) {
    *dst = nullptr;
    cudaError_t e = cudaMalloc((void**)dst, (n ? n : 1) * sizeof(T));  // never a null array
    if (e != cudaSuccess) {
        *dst = nullptr;
        return alloc_fail(e);
    }
    if (src && n) {
        e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return LDPC_OK;
}
}  // namespace

struct ldpc {
    int device = 0, num_sms = 0;
    int mode = kModeFP32, flags = 0, variant = LDPC_VARIANT_AUTO;
    int32_t M = 0, N = 0, max_dc = 0, max_dv = 0;
    int64_t E = 0;
    DevGraph dg;
    ResidentPlan plan[2];
    ResidentTuning tuning;
    std::vector<int32_t> class_degree;
    // learned weights (FP32 mode)
    int32_t w_rows = 0;
    float* w_alpha = nullptr;  // device [w_rows][n_classes], then beta
    // training scratch: accumulators of the weight gradients are the caller's
    cudaStream_t stream = nullptr;
    // streaming workspace
    StreamWork sw;
    int32_t sw_cap = 0, sw_cap_L = -1;
    void* sw_big = nullptr;
    uint8_t* sw_unsat = nullptr;
    void* dense_work = nullptr;  // dense variant workspace
    size_t dense_cap = 0;
    int32_t stream_group = -1;   // streaming: -1 no frame groups, 0 L2-sized groups, > 0 group size
    int l2_bytes = 0;
    int smem_optin = 0;           // shared memory a CTA may opt in to on this device
    int32_t* counters = nullptr;  // [0] resident / cluster tile counter, [1] streaming done
                                  // count, [2] device error word (bounded waits that ran out),
                                  // [4..7] the debug checks' report (two 64-bit words)
    int debug = 0;                // ldpc_set_debug
    int32_t dbg_what = 0;         // the last refused decode's first violation
    int64_t dbg_where = 0;
    // staged streaming check pass: requested warps per CTA and stages (0 = automatic,
    // stages -1 = off) and the tries of each bounded wait
    int32_t st_warps = 0, st_stages = 0, st_vw = 0;
    uint32_t wait_limit = 1u << 16;
    // cluster variant: layouts built on demand from the host graph, one per cluster size
    // 2^i; plans per mode, recomputed after any change of tuning or weights
    HostGraph hg;
    mutable DevCluster dcl[5];
    mutable int dcl_state[5] = {};  // 0 not built, 1 built, -1 cannot be built
    int32_t cl_C = 0, cl_FT = 0, cl_threads = 0;  // requested shape, 0 = automatic
    mutable ClusterPlan cl_plan[2];
    mutable int cl_valid[2] = {};
    int32_t last_launches = 0;
    // frames whose messages the streaming workspace holds after the last decode (a
    // streaming decode without early stop or frame groups), and that decode's mode; 0 when
    // the last decode left none (ldpc_read_messages)
    int32_t msg_frames = 0, msg_mode = kModeFP32;
    int32_t msg_cmp = 0, msg_L = 0;  // that decode kept compressed messages; its iterations
    int32_t st_msg = 1;              // ldpc_set_stream_messages
    // host pipeline staging (2 slots)
    cudaStream_t h2d = nullptr, d2h = nullptr;
    cudaEvent_t ev_h2d[2] = {}, ev_comp[2] = {}, ev_d2h[2] = {};
    void* stage[2] = {};
    size_t stage_bytes = 0;
};

static void free_graph(DevGraph& g) {
    void* ptrs[] = {g.row_ptr, g.col_idx, g.col_ptr, g.col_edge, g.packed, g.r_base,
                    g.r_deg, g.r_slot_pos, g.c_base, g.c_deg, g.c_slot, g.col_pos,
                    g.col_class, g.r_slot_cls, g.ell_col, g.ell_deg, g.ell_cslot, g.ell_cls};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    g = DevGraph();
}

static void free_cluster(DevCluster& c) {
    void* ptrs[] = {c.meta, c.r_base, c.c_base, c.r_deg, c.c_deg, c.r_ref, c.c_ref, c.r_cls, c.pos_of_col};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c = DevCluster();
}

static void free_stream_work(ldpc_t* h) {
    if (h->sw_big) cudaFree(h->sw_big);
    if (h->sw_unsat) cudaFree(h->sw_unsat);
    h->sw_big = nullptr;
    h->sw_unsat = nullptr;
    h->sw = StreamWork();
    h->sw_cap = 0;
    h->sw_cap_L = -1;
}

// Largest batch of one streaming decode (its grids put frame blocks on the y dimension).
constexpr int32_t kMaxStreamFrames = 65535 * 32;

// Warps per CTA of the staged check pass: the caller's, else the default; but an FP32 code
// on rows of 16 slots keeps its messages compressed only with fewer warps (their stages do
// not fit 12 warps' shared memory, and the decode would fall back to per-edge messages), so
// there the automatic choice is the largest of 8 and 4 warps that fits (QC N=2304, 65536
// frames, 10 iterations: 16.8 ms compressed with 8 warps against 23.3 ms per edge).
static int32_t stage_warps_of(const ldpc_t* h) {
    if (h->st_warps > 0) return h->st_warps;
    if (h->mode != kModeFP32 || !h->st_msg || h->dg.ell_D == 0 || h->st_stages < 0) return kStageWarpsDefault;
    if (h->w_rows > 0 && h->dg.n_classes > 256) return kStageWarpsDefault;
    const int stages = h->st_stages > 0 ? h->st_stages : kStagesDefault;
    const int vw = h->st_vw ? h->st_vw : 4;
    for (int32_t w : {kStageWarpsDefault, 8, 4})
        if (staged_smem_bytes(kModeFP32, vw, h->dg.ell_D, true, w, stages, h->w_rows > 0) <=
            (size_t)h->smem_optin)
            return w;
    return kStageWarpsDefault;
}

// The staged check pass settings of a handle, applied to a streaming workspace.
static void apply_staging(const ldpc_t* h, StreamWork& w) {
    w.err = h->counters + 2;
    w.num_sms = h->num_sms;
    w.stage_warps = stage_warps_of(h);
    w.stages = h->st_stages < 0 ? 0 : (h->st_stages > 0 ? h->st_stages : kStagesDefault);
    w.stage_vw = h->st_vw;
    w.wait_limit = h->wait_limit;
    w.msg_compressed = h->st_msg;
}

static int ensure_stream_work(ldpc_t* h, int32_t frames, int32_t L, int32_t granule = 256) {
    if (frames > kMaxStreamFrames) return fail(LDPC_ERR_INVALID_ARG);
    const int32_t Fp = (frames + granule - 1) / granule * granule;
    if (Fp > h->sw_cap) {
        if (h->sw_big) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->sw_big);
            h->sw_big = nullptr;
        }
        const size_t tb = 4, rb = 4;  // sized for fp32; the fixed mode uses less
        const size_t eta = (size_t)h->dg.eta_slots * Fp * tb, sb = (size_t)h->N * Fp * tb,
                     rr = (size_t)h->N * Fp * rb, hd = (size_t)h->N * (Fp / 4);
        const size_t total = eta + sb + rr + hd + (size_t)Fp * 12 + (size_t)Fp + 1280;
        cudaError_t e = cudaMalloc(&h->sw_big, total);
        if (e != cudaSuccess) {
            h->sw_big = nullptr;
            h->sw_cap = 0;
            return alloc_fail(e);
        }
        char* p = (char*)h->sw_big;
        h->sw.eta = p;
        p += (eta + 255) & ~(size_t)255;
        h->sw.s = p;
        p += (sb + 255) & ~(size_t)255;
        h->sw.r = p;
        p += (rr + 255) & ~(size_t)255;
        h->sw.hd = (uint8_t*)p;
        p += (hd + 255) & ~(size_t)255;
        h->sw.done_iter = (int32_t*)p;
        p += (size_t)Fp * 4;
        h->sw.pos2frame = (int32_t*)p;
        p += (size_t)Fp * 4;
        h->sw.new_pos = (int32_t*)p;
        p += (size_t)Fp * 4;
        h->sw.state = (uint8_t*)p;
        p += (size_t)Fp;
        h->sw.comp = (int32_t*)p;  // Fp is a multiple of 32: 16-byte aligned
        h->sw_cap = Fp;
        h->sw_cap_L = -1;  // unsat depends on Fp too
    }
    if (L > h->sw_cap_L) {
        if (h->sw_unsat) {
            cudaStreamSynchronize(h->stream);
            cudaFree(h->sw_unsat);
            h->sw_unsat = nullptr;
        }
        cudaError_t e = cudaMalloc((void**)&h->sw_unsat, (size_t)(L + 2) * h->sw_cap);
        if (e != cudaSuccess) {
            h->sw_unsat = nullptr;
            h->sw_cap_L = -1;
            return alloc_fail(e);
        }
        h->sw_cap_L = L;
    }
    h->sw.Fp = Fp;
    h->sw.unsat = h->sw_unsat;
    h->sw.n_done = h->counters + 1;
    apply_staging(h, h->sw);
    return LDPC_OK;
}

// Resident plans for both modes under the current tuning and weights.
static void replan(ldpc_t* h) {
    h->cl_valid[0] = h->cl_valid[1] = 0;
    if (!h->dg.sliced) return;
    const int we = h->w_rows * h->dg.n_classes;
    h->plan[kModeFP32] = resident_plan(kModeFP32, h->dg, h->N, h->device, h->tuning, we);
    h->plan[kModeFixed] = resident_plan(kModeFixed, h->dg, h->N, h->device, h->tuning, 0);
}

// The cluster layout for cluster size 2^li, built and uploaded on first use.
static bool cluster_layout(const ldpc_t* h, int li) {
    if (h->dcl_state[li]) return h->dcl_state[li] > 0;
    h->dcl_state[li] = -1;
    ClusterGraph cgr;
    if (!build_cluster(h->hg, 1 << li, cgr)) return false;
    DevCluster d;
    d.C = cgr.C;
    d.E_cap = cgr.E_cap;
    d.P_cap = cgr.P_cap;
    if (upload(&d.meta, cgr.meta.data(), cgr.meta.size()) ||
        upload(&d.r_base, cgr.r_base.data(), cgr.r_base.size()) ||
        upload(&d.c_base, cgr.c_base.data(), cgr.c_base.size()) ||
        upload(&d.r_deg, cgr.r_deg.data(), cgr.r_deg.size()) ||
        upload(&d.c_deg, cgr.c_deg.data(), cgr.c_deg.size()) ||
        upload(&d.r_ref, cgr.r_ref.data(), cgr.r_ref.size()) ||
        upload(&d.c_ref, cgr.c_ref.data(), cgr.c_ref.size()) ||
        upload(&d.r_cls, cgr.r_cls.data(), cgr.r_cls.size()) ||
        upload(&d.pos_of_col, cgr.pos_of_col.data(), cgr.pos_of_col.size())) {
        free_cluster(d);
        cudaGetLastError();
        return false;
    }
    h->dcl[li] = d;
    h->dcl_state[li] = 1;
    return true;
}

// Cluster plan of a mode: the requested cluster size, else the smallest real cluster
// (2, 4, 8, 16 CTAs) that holds a tile.
static const ClusterPlan& cluster_plan_of(const ldpc_t* h, int mode) {
    if (h->cl_valid[mode]) return h->cl_plan[mode];
    ClusterPlan best;
    const int we = (mode == kModeFP32 && h->w_rows > 0) ? h->w_rows * h->dg.n_classes : 0;
    for (int li = 0; li <= 4 && !best.ok; li++) {
        const int C = 1 << li;
        if (h->cl_C ? C != h->cl_C : C == 1) continue;
        if (!cluster_layout(h, li)) continue;
        best = cluster_plan(mode, h->dcl[li], h->cl_FT, h->cl_threads, we);
    }
    h->cl_plan[mode] = best;
    h->cl_valid[mode] = 1;
    return h->cl_plan[mode];
}

static int log2_of(int C) {
    int li = 0;
    while ((1 << li) < C) li++;
    return li;
}

// AUTO: resident when a frame fits one SM, else streaming. The cluster variant is never
// chosen automatically: on codes too large for one SM it measured slower than streaming,
// its scattered 2- and 4-byte reads of other CTAs' shared memory being the bottleneck.
static int resolved_variant(const ldpc_t* h) {
    if (h->variant != LDPC_VARIANT_AUTO) return h->variant;
    return h->plan[h->mode].ok ? LDPC_VARIANT_RESIDENT : LDPC_VARIANT_STREAM;
}

static int is_device_ptr(const void* p) {
    if (!p) return 0;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static ldpc_t* create_from_graph(HostGraph& hg, int32_t mode, int32_t flags) {
    ldpc_t* h = new (std::nothrow) ldpc_t();
    if (!h) {
        fail(LDPC_ERR_OOM);
        return nullptr;
    }
    h->mode = mode;
    h->flags = flags;
    const char* dbg_env = std::getenv("LDPC_DEBUG");
    h->debug = ((flags & LDPC_FLAG_DEBUG) || (dbg_env && dbg_env[0] == '1' && dbg_env[1] == 0)) ? 1 : 0;
    h->M = hg.M;
    h->N = hg.N;
    h->E = hg.E;
    h->max_dc = hg.max_dc;
    h->max_dv = hg.max_dv;
    int rc = LDPC_OK;
    auto bail = [&](int status) -> ldpc_t* {
        free_graph(h->dg);
        if (h->counters) cudaFree(h->counters);
        delete h;
        if (status != LDPC_OK) g_last_error = status;
        return nullptr;
    };
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e));
    e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e));
    e = cudaDeviceGetAttribute(&h->l2_bytes, cudaDevAttrL2CacheSize, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e));
    e = cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device);
    if (e != cudaSuccess) return bail(cuda_fail(e));
    // the static scratch array of ldpc_decode_noalloc is mapped now, so that the entry
    // point never maps or allocates anything itself
    if ((rc = noalloc_setup(h->device)) != LDPC_OK) return bail(fail(rc));
    // CSR / CSC
    if ((rc = upload(&h->dg.row_ptr, hg.row_ptr.data(), hg.row_ptr.size())) ||
        (rc = upload(&h->dg.col_idx, hg.col_idx.data(), hg.col_idx.size())) ||
        (rc = upload(&h->dg.col_ptr, hg.col_ptr.data(), hg.col_ptr.size())) ||
        (rc = upload(&h->dg.col_edge, hg.col_edge.data(), hg.col_edge.size())))
        return bail(rc);
    h->dg.max_dc = hg.max_dc;
    h->dg.eta_slots = hg.E;
    // padded row layout of the streaming kernels (rows of at most 16 edges)
    {
        EllGraph eg;
        if (build_ell(hg, eg)) {
            if ((rc = upload(&h->dg.ell_col, eg.ell_col.data(), eg.ell_col.size())) ||
                (rc = upload(&h->dg.ell_deg, eg.ell_deg.data(), eg.ell_deg.size())) ||
                (rc = upload(&h->dg.ell_cslot, eg.ell_cslot.data(), eg.ell_cslot.size())) ||
                (rc = upload(&h->dg.ell_cls, eg.ell_cls.data(), eg.ell_cls.size())))
                return bail(rc);
            h->dg.ell_D = eg.D;
            h->dg.eta_slots = (int64_t)hg.M * eg.D;
        }
    }
    // edge classes (learned weights)
    h->class_degree = hg.class_degree;
    h->dg.n_classes = (int32_t)hg.class_degree.size();
    if (h->dg.n_classes > 255) h->dg.n_classes = 0;  // weights unsupported for such codes
    if ((rc = upload(&h->dg.col_class, hg.col_class.data(), hg.col_class.size()))) return bail(rc);
    // bit-packed rows
    {
        const int64_t W = (hg.N + 31) / 32;
        std::vector<uint32_t> packed((size_t)hg.M * W, 0u);
        for (int32_t i = 0; i < hg.M; i++)
            for (int32_t e2 = hg.row_ptr[i]; e2 < hg.row_ptr[i + 1]; e2++)
                packed[(size_t)i * W + hg.col_idx[e2] / 32] |= 1u << (hg.col_idx[e2] % 32);
        if ((rc = upload(&h->dg.packed, packed.data(), packed.size()))) return bail(rc);
    }
    // sliced layouts for the resident kernel (codes small enough to be resident)
    SlicedGraph sg;
    if (build_sliced(hg, sg)) {
        DevGraph& d = h->dg;
        d.n_rslices = sg.n_rslices;
        d.n_cslices = sg.n_cslices;
        d.E_pad = sg.E_pad;
        d.Ec_pad = sg.Ec_pad;
        if ((rc = upload(&d.r_base, sg.r_base.data(), sg.r_base.size())) ||
            (rc = upload(&d.r_deg, sg.r_deg.data(), sg.r_deg.size())) ||
            (rc = upload(&d.r_slot_pos, sg.r_slot_pos.data(), sg.r_slot_pos.size())) ||
            (rc = upload(&d.c_base, sg.c_base.data(), sg.c_base.size())) ||
            (rc = upload(&d.c_deg, sg.c_deg.data(), sg.c_deg.size())) ||
            (rc = upload(&d.c_slot, sg.c_slot.data(), sg.c_slot.size())) ||
            (rc = upload(&d.col_pos, sg.col_pos.data(), sg.col_pos.size())) ||
            (rc = upload(&d.r_slot_cls, sg.r_slot_cls.data(), sg.r_slot_cls.size())))
            return bail(rc);
        d.sliced = 1;
        h->plan[kModeFP32] = resident_plan(kModeFP32, d, hg.N, h->device);
        h->plan[kModeFixed] = resident_plan(kModeFixed, d, hg.N, h->device);
    }
    e = cudaMalloc((void**)&h->counters, 8 * sizeof(int32_t));
    if (e != cudaSuccess) return bail(alloc_fail(e));
    e = cudaMemset(h->counters, 0, 8 * sizeof(int32_t));
    if (e != cudaSuccess) return bail(cuda_fail(e));
    h->hg = std::move(hg);
    g_last_error = LDPC_OK;
    return h;
}

int ldpc_impl::handle_view(ldpc_t* h, HandleView* v) {
    if (!h || !v) return LDPC_ERR_BAD_POINTER;
    *v = HandleView{h->device, h->mode, h->flags, h->M, h->N, h->E, &h->dg, h->stream,
                    &h->last_launches, h->w_rows, h->w_alpha};
    v->num_sms = h->num_sms;
    v->err = h->counters + 2;
    v->stage_warps = stage_warps_of(h);
    v->stages = h->st_stages < 0 ? 0 : (h->st_stages > 0 ? h->st_stages : kStagesDefault);
    v->stage_vw = h->st_vw;
    v->wait_limit = h->wait_limit;
    v->msg_compressed = h->st_msg;
    return LDPC_OK;
}


extern "C" {

ldpc_t* ldpc_create_ex(int32_t M, int32_t N, int32_t h_format, const void* h_a, const void* h_b,
                       int32_t mode, int32_t flags) {
    if (mode != LDPC_MODE_FP32 && mode != LDPC_MODE_FIXED) {
        fail(LDPC_ERR_INVALID_ARG);
        return nullptr;
    }
    if (flags & ~(LDPC_FLAG_PAPER_SLICER | LDPC_FLAG_DEBUG)) {
        fail(LDPC_ERR_INVALID_ARG);
        return nullptr;
    }
    if (M <= 0 || N <= 0) {
        fail(LDPC_ERR_INVALID_H);
        return nullptr;
    }
    HostGraph hg;
    int rc;
    switch (h_format) {
        case LDPC_H_DENSE_U8: rc = graph_from_dense(M, N, (const uint8_t*)h_a, hg); break;
        case LDPC_H_PACKED_U32: rc = graph_from_packed(M, N, (const uint32_t*)h_a, hg); break;
        case LDPC_H_CSR: rc = graph_from_csr(M, N, (const int64_t*)h_a, (const int32_t*)h_b, hg); break;
        default: rc = LDPC_ERR_INVALID_ARG;
    }
    if (rc != LDPC_OK) {
        fail(rc);
        return nullptr;
    }
    return create_from_graph(hg, mode, flags);
}

ldpc_t* ldpc_create(int32_t M, int32_t N, const uint8_t* H) {
    return ldpc_create_ex(M, N, LDPC_H_DENSE_U8, H, nullptr, LDPC_MODE_FP32, 0);
}

// The debug checks of one decode (ldpc_set_debug): enqueue them, wait, read the report.
static int debug_checks(ldpc_t* h, const void* llr, int llr_is_i8, int32_t frames) {
    auto* rep = reinterpret_cast<unsigned long long*>(h->counters + 4);
    int rc = debug_check_launch(h->dg, h->M, h->N, h->E, llr, llr_is_i8, frames, rep, h->stream);
    if (rc != LDPC_OK) return rc;
    unsigned long long r[2];
    cudaError_t e = cudaMemcpyAsync(r, rep, sizeof(r), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        g_last_cuda = (int)e;
        return LDPC_ERR_CUDA;
    }
    if (r[0] == ~0ull && r[1] == ~0ull) return LDPC_OK;
    h->dbg_what = r[0] != ~0ull ? 1 : 2;
    h->dbg_where = (int64_t)(r[0] != ~0ull ? r[0] : r[1]);
    return LDPC_ERR_DEVICE_CHECK;
}

int ldpc_decode_ex(ldpc_t* h, const void* llr, int32_t llr_dtype, int32_t frames, int32_t max_iter,
                   int32_t early_stop, int32_t check_every, uint8_t* out_bits, int32_t* out_iters,
                   uint8_t* out_ok, float* out_soft) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames < 0 || max_iter < 0 || check_every < 1) return fail(LDPC_ERR_INVALID_ARG);
    if (llr_dtype != LDPC_LLR_F32 && llr_dtype != LDPC_LLR_I8) return fail(LDPC_ERR_INVALID_ARG);
    if (llr_dtype == LDPC_LLR_I8 && h->mode != kModeFixed) return fail(LDPC_ERR_INVALID_ARG);
    if (h->w_rows > 0 && h->mode != kModeFP32) return fail(LDPC_ERR_UNSUPPORTED);
    h->last_launches = 0;
    h->msg_frames = 0;
    if (frames == 0) return LDPC_OK;
    if (!is_device_ptr(llr) || !is_device_ptr(out_bits) || !is_device_ptr(out_iters) ||
        (out_ok && !is_device_ptr(out_ok)) || (out_soft && !is_device_ptr(out_soft)))
        return fail(LDPC_ERR_BAD_POINTER);
    if (h->debug) {
        const int rc = debug_checks(h, llr, llr_dtype == LDPC_LLR_I8, frames);
        if (rc != LDPC_OK) return fail(rc);
    }
    DecodeArgs a;
    a.M = h->M;
    a.N = h->N;
    a.E = (int32_t)h->E;
    a.frames = frames;
    a.L = max_iter;
    a.early_stop = early_stop ? 1 : 0;
    a.check_every = check_every;
    a.paper_slicer = (h->flags & LDPC_FLAG_PAPER_SLICER) ? 1 : 0;
    a.llr_is_i8 = llr_dtype == LDPC_LLR_I8;
    a.llr = llr;
    a.out_bits = out_bits;
    a.out_iters = out_iters;
    a.out_ok = out_ok;
    a.out_soft = out_soft;
    if (h->w_rows > 0 && h->mode == kModeFP32) {
        a.w_rows = h->w_rows;
        a.n_classes = h->dg.n_classes;
        a.w_alpha = h->w_alpha;
        a.w_beta = h->w_alpha + (size_t)h->w_rows * h->dg.n_classes;
    }
    int n;
    if (resolved_variant(h) == LDPC_VARIANT_DENSE) {
        if (h->mode != kModeFP32 || a.w_rows > 0 || a.llr_is_i8) return fail(LDPC_ERR_UNSUPPORTED);
        if (frames > 65535) return fail(LDPC_ERR_INVALID_ARG);
        const size_t need = dense_bytes(h->M, h->N, frames);
        if (need > h->dense_cap) {
            if (h->dense_work) {
                cudaStreamSynchronize(h->stream);
                cudaFree(h->dense_work);
                h->dense_work = nullptr;
                h->dense_cap = 0;
            }
            cudaError_t e = cudaMalloc(&h->dense_work, need);
            if (e != cudaSuccess) {
                h->dense_work = nullptr;
                return alloc_fail(e);
            }
            h->dense_cap = need;
        }
        n = dense_decode(h->dg, a, h->dense_work, h->stream);
    } else if (resolved_variant(h) == LDPC_VARIANT_RESIDENT) {
        if (!h->plan[h->mode].ok) return fail(LDPC_ERR_UNSUPPORTED);
        n = resident_decode(h->mode, h->dg, h->plan[h->mode], a, h->counters, h->num_sms, h->stream);
    } else if (resolved_variant(h) == LDPC_VARIANT_CLUSTER) {
        const ClusterPlan& p = cluster_plan_of(h, h->mode);
        if (!p.ok) return fail(LDPC_ERR_UNSUPPORTED);
        n = cluster_decode(h->mode, h->dcl[log2_of(p.C)], p, a, h->counters, h->stream);
    } else {
        // A batch whose streaming working set (messages, posteriors, channel values) would
        // overflow L2 is decoded in frame groups that fit, one frame per lane, each group
        // through all its iterations before the next: the messages then live in L2.
        const size_t tb = h->mode == kModeFP32 ? 4 : 2, rb = h->mode == kModeFP32 ? 4 : 1;
        const size_t per_frame = (size_t)h->E * tb + (size_t)h->N * (tb + rb);
        const size_t budget = (size_t)h->l2_bytes / 2;
        int32_t group = h->stream_group;
        if (group == 0 && (size_t)frames * per_frame > budget && 32 * per_frame <= budget)
            group = (int32_t)std::max<size_t>(32, budget / per_frame / 32 * 32);
        if (group > 0 && group < frames) {
            // frames per lane: the widest vector (up to 16 bytes) that the group fills
            int vw = 1;
            while (vw * 2 <= (h->mode == kModeFP32 ? 4 : 8) && group % (64 * vw) == 0) vw *= 2;
            int rc = ensure_stream_work(h, group, max_iter, 32 * vw);
            if (rc != LDPC_OK) return rc;
            const size_t in_b = a.llr_is_i8 ? 1 : 4;
            n = 0;
            for (int32_t f0 = 0; f0 < frames && n >= 0; f0 += group) {
                DecodeArgs ag = a;
                ag.frames = std::min(group, frames - f0);
                ag.llr = (const char*)llr + (size_t)f0 * h->N * in_b;
                ag.out_bits = out_bits + (size_t)f0 * h->N;
                ag.out_iters = out_iters + f0;
                ag.out_ok = out_ok ? out_ok + f0 : nullptr;
                ag.out_soft = out_soft ? out_soft + (size_t)f0 * h->N : nullptr;
                const int k = stream_decode(h->mode, h->dg, ag, h->sw, h->stream, vw);
                n = k < 0 ? k : n + k;
            }
        } else {
            int rc = ensure_stream_work(h, frames, max_iter);
            if (rc != LDPC_OK) return rc;
            int32_t used_cmp = 0;
            StreamWork w = h->sw;
            w.used_compressed = &used_cmp;
            n = stream_decode(h->mode, h->dg, a, w, h->stream);
            if (n >= 0 && !a.early_stop) {  // no compaction: position = frame
                h->msg_frames = frames;
                h->msg_mode = h->mode;
                h->msg_cmp = used_cmp;
                h->msg_L = max_iter;
            }
        }
    }
    if (n < 0) {
        cudaError_t e = cudaGetLastError();
        return e != cudaSuccess ? cuda_fail(e) : fail(n);
    }
    h->last_launches = n;
    return LDPC_OK;
}

int ldpc_decode(ldpc_t* h, const float* llr, int32_t frames, int32_t max_iter, uint8_t* out_bits,
                int32_t* out_iters) {
    return ldpc_decode_ex(h, llr, LDPC_LLR_F32, frames, max_iter, 1, 1, out_bits, out_iters, nullptr,
                          nullptr);
}

int ldpc_decode_i8(ldpc_t* h, const int8_t* llr_q, int32_t frames, int32_t max_iter,
                   uint8_t* out_bits, int32_t* out_iters) {
    if (h && h->mode != kModeFixed) return fail(LDPC_ERR_INVALID_ARG);
    return ldpc_decode_ex(h, llr_q, LDPC_LLR_I8, frames, max_iter, 1, 1, out_bits, out_iters,
                          nullptr, nullptr);
}

int ldpc_decode_host(ldpc_t* h, const void* llr_host, int32_t llr_dtype, int32_t frames,
                     int32_t max_iter, int32_t early_stop, int32_t check_every, uint8_t* bits_host,
                     int32_t* iters_host, uint8_t* ok_host, float* soft_host) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames < 0 || max_iter < 0 || check_every < 1) return fail(LDPC_ERR_INVALID_ARG);
    if (llr_dtype != LDPC_LLR_F32 && llr_dtype != LDPC_LLR_I8) return fail(LDPC_ERR_INVALID_ARG);
    if (frames == 0) return LDPC_OK;
    if (!llr_host || !bits_host || !iters_host) return fail(LDPC_ERR_BAD_POINTER);
    const int N = h->N;
    const size_t in_b = llr_dtype == LDPC_LLR_F32 ? 4 : 1;
    // chunk so that several chunks are in flight and each still fills the GPU
    int32_t chunk = std::max<int32_t>(1024, std::min<int32_t>(frames, (frames + 3) / 4));
    chunk = std::min<int32_t>(chunk, std::max<int32_t>(1024, (int32_t)((512ull << 20) / (N * in_b))));
    // Chunk sizes: nothing overlaps the first chunk's input copy or the last chunk's output
    // copy, so the schedule ramps up from an eighth of the chunk (doubling: the next
    // chunk's input copy still hides behind the decode of the current one) and back down
    // at the end.
    std::vector<int32_t> sizes;
    {
        const int32_t first = std::max<int32_t>(1024, chunk / 8);  // still fills the GPU
        std::vector<int32_t> ramp;  // first, 2 first, ... up to half a chunk
        for (int32_t c = first; 2 * c <= chunk; c *= 2) ramp.push_back(c);
        int64_t ramp_sum = 0;
        for (int32_t c : ramp) ramp_sum += c;
        int32_t left = frames;
        if ((int64_t)frames >= 2 * ramp_sum + chunk) {
            for (int32_t c : ramp) sizes.push_back(c);
            left -= (int32_t)ramp_sum;
            while (left > ramp_sum) {
                const int32_t c = (int32_t)std::min<int64_t>(chunk, left - ramp_sum);
                sizes.push_back(c);
                left -= c;
            }
            for (auto it = ramp.rbegin(); it != ramp.rend(); ++it) {
                sizes.push_back(*it);
                left -= *it;
            }
        } else {  // too few frames for a ramp: even chunks
            for (; left > 0; left -= std::min(chunk, left)) sizes.push_back(std::min(chunk, left));
        }
    }
    const size_t per_frame = (size_t)N * in_b + (size_t)N + 4 + 1 + (soft_host ? (size_t)N * 4 : 0);
    const size_t need = ((size_t)chunk * per_frame + 4096);
    if (!h->h2d) {
        CK(cudaStreamCreateWithFlags(&h->h2d, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&h->d2h, cudaStreamNonBlocking));
        for (int s = 0; s < 2; s++) {
            CK(cudaEventCreateWithFlags(&h->ev_h2d[s], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ev_comp[s], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&h->ev_d2h[s], cudaEventDisableTiming));
        }
    }
    if (need > h->stage_bytes) {
        for (int s = 0; s < 2; s++) {
            if (h->stage[s]) {
                cudaStreamSynchronize(h->d2h);
                cudaFree(h->stage[s]);
                h->stage[s] = nullptr;
            }
            cudaError_t e = cudaMalloc(&h->stage[s], need);
            if (e != cudaSuccess) {
                h->stage[s] = nullptr;
                h->stage_bytes = 0;
                return alloc_fail(e);
            }
        }
        h->stage_bytes = need;
    }
    int launches = 0;
    int32_t f0 = 0;
    for (int c = 0; c < (int)sizes.size(); f0 += sizes[c], c++) {
        const int s = c & 1;
        const int32_t nf = sizes[c];
        char* base = (char*)h->stage[s];
        void* d_llr = base;
        uint8_t* d_bits = (uint8_t*)(base + (((size_t)chunk * N * in_b + 255) & ~(size_t)255));
        int32_t* d_iters = (int32_t*)((char*)d_bits + (((size_t)chunk * N + 255) & ~(size_t)255));
        uint8_t* d_ok = (uint8_t*)(d_iters + ((chunk + 63) & ~63));
        float* d_soft = soft_host ? (float*)(d_ok + ((chunk + 255) & ~255)) : nullptr;
        if (c >= 2) CK(cudaStreamWaitEvent(h->h2d, h->ev_d2h[s], 0));
        CK(cudaMemcpyAsync(d_llr, (const char*)llr_host + (size_t)f0 * N * in_b, (size_t)nf * N * in_b,
                           cudaMemcpyHostToDevice, h->h2d));
        CK(cudaEventRecord(h->ev_h2d[s], h->h2d));
        CK(cudaStreamWaitEvent(h->stream, h->ev_h2d[s], 0));
        int rc = ldpc_decode_ex(h, d_llr, llr_dtype, nf, max_iter, early_stop, check_every, d_bits,
                                d_iters, ok_host ? d_ok : nullptr, d_soft);
        if (rc != LDPC_OK) return rc;
        launches += h->last_launches;
        CK(cudaEventRecord(h->ev_comp[s], h->stream));
        CK(cudaStreamWaitEvent(h->d2h, h->ev_comp[s], 0));
        CK(cudaMemcpyAsync(bits_host + (size_t)f0 * N, d_bits, (size_t)nf * N, cudaMemcpyDeviceToHost, h->d2h));
        CK(cudaMemcpyAsync(iters_host + f0, d_iters, (size_t)nf * 4, cudaMemcpyDeviceToHost, h->d2h));
        if (ok_host) CK(cudaMemcpyAsync(ok_host + f0, d_ok, (size_t)nf, cudaMemcpyDeviceToHost, h->d2h));
        if (soft_host)
            CK(cudaMemcpyAsync(soft_host + (size_t)f0 * N, d_soft, (size_t)nf * N * 4,
                               cudaMemcpyDeviceToHost, h->d2h));
        CK(cudaEventRecord(h->ev_d2h[s], h->d2h));
    }
    CK(cudaStreamSynchronize(h->d2h));
    h->last_launches = launches;
    return LDPC_OK;
}

int ldpc_set_stream(ldpc_t* h, void* cuda_stream) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    h->stream = (cudaStream_t)cuda_stream;
    return LDPC_OK;
}

int ldpc_set_mode(ldpc_t* h, int32_t mode) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (mode != LDPC_MODE_FP32 && mode != LDPC_MODE_FIXED) return fail(LDPC_ERR_INVALID_ARG);
    h->mode = mode;
    return LDPC_OK;
}

int ldpc_set_tuning(ldpc_t* h, int32_t frames_per_tile, int32_t threads, int32_t index_placement) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if ((frames_per_tile != 0 && frames_per_tile != 1 && frames_per_tile != 2 && frames_per_tile != 4) ||
        threads < 0 || threads % 32 || index_placement < 0 || index_placement > 2)
        return fail(LDPC_ERR_INVALID_ARG);
    if (!h->dg.sliced) return fail(LDPC_ERR_UNSUPPORTED);
    ResidentTuning t;
    t.FT = frames_per_tile;
    t.threads = threads;
    t.idx = index_placement;
    const ResidentPlan p = resident_plan(h->mode, h->dg, h->N, h->device, t,
                                         h->mode == kModeFP32 ? h->w_rows * h->dg.n_classes : 0);
    if (!p.ok) return fail(LDPC_ERR_UNSUPPORTED);
    h->tuning = t;
    replan(h);
    return LDPC_OK;
}

// What the autotuners time: zeros without early stop (the work then does not depend on
// the values), or the caller's frames (device FP32 [frames][N]) with its early-stop
// settings, whose frames stop at different iterations.
struct TuneData {
    const float* llr = nullptr;  // nullptr: zeros, no early stop
    int32_t early_stop = 0;
    int32_t check_every = 1;
};

// Streaming codes: time the staged check pass's shapes (and the unstaged kernel) on
// min(frames, 2048) frames through the regular decode path, and keep the fastest.
static int autotune_stream(ldpc_t* h, int32_t frames, int32_t max_iter, float* best_ms,
                           const TuneData& td) {
    if (!h->dg.ell_D) return fail(LDPC_ERR_UNSUPPORTED);  // only the padded layout has shapes
    const int32_t F = std::min<int32_t>(frames, 2048);
    void* llr = nullptr;
    uint8_t* bits = nullptr;
    int32_t* iters = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (llr) cudaFree(llr);
        if (bits) cudaFree(bits);
        if (iters) cudaFree(iters);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if ((!td.llr && cudaMalloc(&llr, (size_t)F * h->N * 4) != cudaSuccess) ||
        cudaMalloc((void**)&bits, (size_t)F * h->N) != cudaSuccess ||
        cudaMalloc((void**)&iters, (size_t)F * 4) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(LDPC_ERR_OOM);
    }
    if (!td.llr && cudaMemsetAsync(llr, 0, (size_t)F * h->N * 4, h->stream) != cudaSuccess) {
        cleanup();
        return fail(LDPC_ERR_CUDA);
    }
    const void* x = td.llr ? (const void*)td.llr : llr;
    const int32_t keep[3] = {h->st_warps, h->st_stages, h->st_vw};
    // (warps, stages, frames per lane): full and half-width lanes (half-width stages let rows
    // of 16 slots fit more warps), and the unstaged kernel
    // (shapes whose shared memory does not fit run the unstaged kernel and lose)
    static const int32_t shapes[][3] = {{8, 3, 0}, {12, 2, 0}, {6, 3, 0}, {4, 4, 0}, {8, 2, 0},
                                        {12, 3, 0}, {8, 4, 0}, {4, 2, 0}, {6, 2, 0}, {12, 2, 2},
                                        {8, 3, 2}, {0, -1, 0}};
    constexpr int n_shapes = (int)(sizeof(shapes) / sizeof(shapes[0]));
    // FP32 on the padded layout: every staged shape with compressed and with per-edge
    // messages (the unstaged kernel keeps per-edge messages)
    const int n_fmt = h->mode == kModeFP32 ? 2 : 1;
    const int32_t keep_msg = h->st_msg;
    float best = -1.0f;
    int bi = -1;
    for (int k = 0; k < n_shapes * n_fmt; k++) {
        const int sh = k % n_shapes;
        if (k >= n_shapes && shapes[sh][1] < 0) continue;
        h->st_msg = n_fmt == 2 ? (k < n_shapes ? 1 : 0) : keep_msg;
        h->st_warps = shapes[sh][0];
        h->st_stages = shapes[sh][1];
        h->st_vw = shapes[sh][2] ? (h->mode == kModeFP32 ? 2 : 4) : 0;
        float ms = 0.0f;
        auto run = [&]() {
            return ldpc_decode_ex(h, x, LDPC_LLR_F32, F, max_iter, td.early_stop, td.check_every,
                                  bits, iters, nullptr, nullptr) != LDPC_OK;
        };
        bool bad = run();
        bad = bad || cudaEventRecord(e0, h->stream) != cudaSuccess;
        for (int r = 0; r < 2 && !bad; r++) bad = run();
        bad = bad || cudaEventRecord(e1, h->stream) != cudaSuccess ||
              cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
        if (bad) {
            cudaGetLastError();
            continue;
        }
        if (best < 0.0f || ms < best) {
            best = ms;
            bi = k;
        }
    }
    cleanup();
    if (bi < 0) {
        h->st_warps = keep[0];
        h->st_stages = keep[1];
        h->st_vw = keep[2];
        h->st_msg = keep_msg;
        apply_staging(h, h->sw);
        return fail(LDPC_ERR_UNSUPPORTED);
    }
    h->st_msg = n_fmt == 2 ? (bi < n_shapes ? 1 : 0) : keep_msg;
    h->st_warps = shapes[bi % n_shapes][0];
    h->st_stages = shapes[bi % n_shapes][1];
    h->st_vw = shapes[bi % n_shapes][2] ? (h->mode == kModeFP32 ? 2 : 4) : 0;
    apply_staging(h, h->sw);
    if (best_ms) *best_ms = best / 2.0f;
    return LDPC_OK;
}

static int autotune(ldpc_t* h, int32_t frames, int32_t max_iter, float* best_ms,
                    const TuneData& td) {
    if (resolved_variant(h) == LDPC_VARIANT_STREAM)
        return autotune_stream(h, frames, max_iter, best_ms, td);
    if (!h->dg.sliced || !h->plan[h->mode].ok) return fail(LDPC_ERR_UNSUPPORTED);
    // the caller's frames: up to a full 65536-frame batch (how many tiles fill the SMs
    // decides the shape); zeros: a quarter of that
    const int32_t F = std::min<int32_t>(frames, td.llr ? 65536 : 16384);
    void* llr = nullptr;
    uint8_t* bits = nullptr;
    int32_t* iters = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        if (llr) cudaFree(llr);
        if (bits) cudaFree(bits);
        if (iters) cudaFree(iters);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if ((!td.llr && cudaMalloc(&llr, (size_t)F * h->N * 4) != cudaSuccess) ||
        cudaMalloc((void**)&bits, (size_t)F * h->N) != cudaSuccess ||
        cudaMalloc((void**)&iters, (size_t)F * 4) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        cudaGetLastError();
        return fail(LDPC_ERR_OOM);
    }
    if (!td.llr && cudaMemsetAsync(llr, 0, (size_t)F * h->N * 4, h->stream) != cudaSuccess) {
        cleanup();
        return fail(LDPC_ERR_CUDA);
    }
    DecodeArgs a;
    a.M = h->M;
    a.N = h->N;
    a.E = (int32_t)h->E;
    a.frames = F;
    a.L = max_iter;
    a.early_stop = td.early_stop;
    a.check_every = td.check_every;
    a.paper_slicer = (h->flags & LDPC_FLAG_PAPER_SLICER) ? 1 : 0;
    a.llr_is_i8 = 0;
    a.llr = td.llr ? (const void*)td.llr : llr;
    a.out_bits = bits;
    a.out_iters = iters;
    a.out_ok = nullptr;
    a.out_soft = nullptr;
    if (h->w_rows > 0 && h->mode == kModeFP32) {
        a.w_rows = h->w_rows;
        a.n_classes = h->dg.n_classes;
        a.w_alpha = h->w_alpha;
        a.w_beta = h->w_alpha + (size_t)h->w_rows * h->dg.n_classes;
    }
    float best = -1.0f;
    ResidentTuning best_t = h->tuning;
    for (int ft : {1, 2, 4})
    for (int ip : {1, 2})
        for (int th = 0; th <= 1024; th += 64) {  // 0: the default for the tile
            ResidentTuning t;
            t.FT = ft;
            t.threads = th;
            t.idx = ip;
            const ResidentPlan p = resident_plan(h->mode, h->dg, h->N, h->device, t,
                                                 h->mode == kModeFP32 ? h->w_rows * h->dg.n_classes : 0);
            if (!p.ok) continue;
            float ms = 0.0f;
            bool bad = resident_decode(h->mode, h->dg, p, a, h->counters, h->num_sms, h->stream) < 0;
            bad = bad || cudaEventRecord(e0, h->stream) != cudaSuccess;
            for (int r = 0; r < 2 && !bad; r++)
                bad = resident_decode(h->mode, h->dg, p, a, h->counters, h->num_sms, h->stream) < 0;
            bad = bad || cudaEventRecord(e1, h->stream) != cudaSuccess ||
                  cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
            if (bad) {
                cudaGetLastError();
                continue;  // a shape the device cannot run is skipped
            }
            if (best < 0.0f || ms < best) {
                best = ms;
                best_t = t;
            }
        }
    cleanup();
    if (best < 0.0f) return fail(LDPC_ERR_UNSUPPORTED);
    h->tuning = best_t;
    replan(h);
    if (best_ms) *best_ms = best / 2.0f;
    return LDPC_OK;
}

int ldpc_autotune(ldpc_t* h, int32_t frames, int32_t max_iter, float* best_ms) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames <= 0 || max_iter < 0) return fail(LDPC_ERR_INVALID_ARG);
    return autotune(h, frames, max_iter, best_ms, TuneData{});
}

int ldpc_autotune_data(ldpc_t* h, const float* llr, int32_t frames, int32_t max_iter,
                       int32_t early_stop, int32_t check_every, float* best_ms) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames <= 0 || max_iter < 0 || check_every < 1 || (early_stop != 0 && early_stop != 1))
        return fail(LDPC_ERR_INVALID_ARG);
    if (!is_device_ptr(llr)) return fail(LDPC_ERR_BAD_POINTER);
    TuneData td;
    td.llr = llr;
    td.early_stop = early_stop;
    td.check_every = check_every;
    return autotune(h, frames, max_iter, best_ms, td);
}

int ldpc_get_tuning(const ldpc_t* h, int32_t* frames_per_tile, int32_t* threads,
                    int32_t* index_placement) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    const ResidentPlan& p = h->plan[h->mode];
    if (!p.ok) return fail(LDPC_ERR_UNSUPPORTED);
    if (frames_per_tile) *frames_per_tile = p.FT;
    if (threads) *threads = p.threads;
    if (index_placement) *index_placement = p.idx_smem ? 1 : 2;
    return LDPC_OK;
}

int ldpc_classes(const ldpc_t* h, int32_t* n_classes, int32_t* degrees) {
    if (!h || !n_classes) return fail(LDPC_ERR_BAD_POINTER);
    *n_classes = h->dg.n_classes;
    if (degrees)
        for (int32_t c = 0; c < h->dg.n_classes; c++) degrees[c] = h->class_degree[c];
    return LDPC_OK;
}

int ldpc_set_weights(ldpc_t* h, int32_t n_rows, const float* alpha, const float* beta) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (n_rows < 0 || n_rows > 4096) return fail(LDPC_ERR_INVALID_ARG);
    if (n_rows > 0 && (!alpha || !beta)) return fail(LDPC_ERR_BAD_POINTER);
    if (n_rows > 0 && h->dg.n_classes == 0) return fail(LDPC_ERR_UNSUPPORTED);
    cudaStreamSynchronize(h->stream);
    if (h->w_alpha) cudaFree(h->w_alpha);
    h->w_alpha = nullptr;
    h->w_rows = 0;
    if (n_rows == 0) {
        replan(h);
        return LDPC_OK;
    }
    const size_t n = (size_t)n_rows * h->dg.n_classes;
    std::vector<float> tab(2 * n);
    std::copy(alpha, alpha + n, tab.begin());
    std::copy(beta, beta + n, tab.begin() + n);
    int rc = upload(&h->w_alpha, tab.data(), tab.size());
    if (rc != LDPC_OK) return rc;
    h->w_rows = n_rows;
    replan(h);
    return LDPC_OK;
}

int ldpc_set_stream_group(ldpc_t* h, int32_t frames_per_group) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames_per_group < -1 || (frames_per_group > 0 && frames_per_group % 32)) return fail(LDPC_ERR_INVALID_ARG);
    h->stream_group = frames_per_group;
    return LDPC_OK;
}

int ldpc_set_stream_staging(ldpc_t* h, int32_t warps_per_cta, int32_t stages, int32_t frames_per_lane) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (warps_per_cta < 0 || warps_per_cta > 12 || stages < -1 || stages == 1 || stages > 8 ||
        (frames_per_lane != 0 && frames_per_lane != 1 && frames_per_lane != 2 && frames_per_lane != 4 &&
         frames_per_lane != 8))
        return fail(LDPC_ERR_INVALID_ARG);
    h->st_warps = warps_per_cta;
    h->st_stages = stages;
    h->st_vw = frames_per_lane;
    apply_staging(h, h->sw);
    return LDPC_OK;
}

int ldpc_set_stream_messages(ldpc_t* h, int32_t compressed) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (compressed != 0 && compressed != 1) return fail(LDPC_ERR_INVALID_ARG);
    h->st_msg = compressed;
    apply_staging(h, h->sw);
    return LDPC_OK;
}

int ldpc_get_stream_messages(const ldpc_t* h, int32_t* compressed) {
    if (!h || !compressed) return fail(LDPC_ERR_BAD_POINTER);
    *compressed = 0;
    if (!h->st_msg || h->mode != kModeFP32 || h->dg.ell_D == 0 || h->st_stages < 0) return LDPC_OK;
    if (h->w_rows > 0 && h->dg.n_classes > 256) return LDPC_OK;
    // the staged kernel must fit (else the decode keeps per-edge messages)
    StreamWork w;
    apply_staging(h, w);
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
        cudaGetLastError();
        return LDPC_OK;
    }
    const size_t need = staged_smem_bytes(kModeFP32, w.stage_vw ? w.stage_vw : 4, h->dg.ell_D, true,
                                          w.stage_warps, w.stages, h->w_rows > 0);
    *compressed = need <= (size_t)optin ? 1 : 0;
    return LDPC_OK;
}

int ldpc_get_stream_staging(const ldpc_t* h, int32_t* warps_per_cta, int32_t* stages,
                            int32_t* frames_per_lane) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (warps_per_cta) *warps_per_cta = stage_warps_of(h);
    if (stages) *stages = h->st_stages < 0 ? 0 : (h->st_stages > 0 ? h->st_stages : kStagesDefault);
    if (frames_per_lane) *frames_per_lane = h->st_vw;
    return LDPC_OK;
}

int ldpc_read_messages(ldpc_t* h, int32_t frames, float* out) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (frames < 0) return fail(LDPC_ERR_INVALID_ARG);
    if (frames == 0) return LDPC_OK;
    if (h->msg_frames == 0) return fail(LDPC_ERR_UNSUPPORTED);
    if (frames > h->msg_frames) return fail(LDPC_ERR_INVALID_ARG);
    if (!is_device_ptr(out)) return fail(LDPC_ERR_BAD_POINTER);
    const float *wa = nullptr, *wb = nullptr;  // weights of the decode's last iteration
    if (h->msg_cmp && h->w_rows > 0 && h->msg_L > 0) {
        const int row = std::min(h->msg_L, h->w_rows) - 1;
        wa = h->w_alpha + (size_t)row * h->dg.n_classes;
        wb = h->w_alpha + (size_t)h->w_rows * h->dg.n_classes + (size_t)row * h->dg.n_classes;
    }
    const int n = stream_read_messages(h->msg_mode, h->dg, h->M, h->E, h->sw, frames, out, h->stream,
                                       h->msg_cmp, wa, wb);
    if (n < 0) {
        cudaError_t e = cudaGetLastError();
        return e != cudaSuccess ? cuda_fail(e) : fail(n);
    }
    return LDPC_OK;
}

int ldpc_check_device(ldpc_t* h) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e);
    int32_t word = 0;
    e = cudaMemcpy(&word, h->counters + 2, sizeof(word), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    if (word == 0) return LDPC_OK;
    e = cudaMemset(h->counters + 2, 0, sizeof(int32_t));
    if (e != cudaSuccess) return cuda_fail(e);
    return fail(LDPC_ERR_TIMEOUT);
}

int ldpc_set_debug(ldpc_t* h, int32_t on) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (on != 0 && on != 1) return fail(LDPC_ERR_INVALID_ARG);
    h->debug = on;
    return LDPC_OK;
}

int ldpc_debug_report(ldpc_t* h, int32_t* what, int64_t* where) {
    if (!h || !what || !where) return fail(LDPC_ERR_BAD_POINTER);
    *what = h->dbg_what;
    *where = h->dbg_where;
    h->dbg_what = 0;
    h->dbg_where = 0;
    return LDPC_OK;
}

int ldpc_set_wait_limit(ldpc_t* h, int32_t tries) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (tries < 0) return fail(LDPC_ERR_INVALID_ARG);
    h->wait_limit = (uint32_t)tries;
    apply_staging(h, h->sw);
    return LDPC_OK;
}

int ldpc_set_cluster_shape(ldpc_t* h, int32_t cluster_size, int32_t frames_per_tile, int32_t threads) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    const bool c_ok = cluster_size == 0 || cluster_size == 1 || cluster_size == 2 || cluster_size == 4 ||
                      cluster_size == 8 || cluster_size == 16;
    const bool f_ok = frames_per_tile == 0 || frames_per_tile == 1 || frames_per_tile == 2 || frames_per_tile == 4;
    const bool t_ok = threads == 0 || (threads % 32 == 0 && threads >= 64 && threads <= 1024);
    if (!c_ok || !f_ok || !t_ok) return fail(LDPC_ERR_INVALID_ARG);
    h->cl_C = cluster_size;
    h->cl_FT = frames_per_tile;
    h->cl_threads = threads;
    h->cl_valid[0] = h->cl_valid[1] = 0;
    return LDPC_OK;
}

int ldpc_get_cluster_shape(const ldpc_t* h, int32_t* cluster_size, int32_t* frames_per_tile,
                           int32_t* threads, int32_t* clusters) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    const ClusterPlan& p = cluster_plan_of(h, h->mode);
    if (!p.ok) return fail(LDPC_ERR_UNSUPPORTED);
    if (cluster_size) *cluster_size = p.C;
    if (frames_per_tile) *frames_per_tile = p.FT;
    if (threads) *threads = p.threads;
    if (clusters) *clusters = p.clusters;
    return LDPC_OK;
}

int ldpc_set_variant(ldpc_t* h, int32_t variant) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (variant < LDPC_VARIANT_AUTO || variant > LDPC_VARIANT_CLUSTER) return fail(LDPC_ERR_INVALID_ARG);
    if (variant == LDPC_VARIANT_RESIDENT && !h->plan[h->mode].ok) return fail(LDPC_ERR_UNSUPPORTED);
    if (variant == LDPC_VARIANT_CLUSTER && !cluster_plan_of(h, h->mode).ok) return fail(LDPC_ERR_UNSUPPORTED);
    h->variant = variant;
    return LDPC_OK;
}

int ldpc_get_variant(const ldpc_t* h, int32_t* variant) {
    if (!h || !variant) return fail(LDPC_ERR_BAD_POINTER);
    *variant = resolved_variant(h);
    return LDPC_OK;
}

int ldpc_reserve(ldpc_t* h, int32_t max_frames) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (max_frames < 0) return fail(LDPC_ERR_INVALID_ARG);
    if (resolved_variant(h) == LDPC_VARIANT_STREAM && max_frames > 0)
        return ensure_stream_work(h, max_frames, std::max(h->sw_cap_L, 64));
    return LDPC_OK;
}

int ldpc_info(const ldpc_t* h, int32_t* M, int32_t* N, int64_t* E, int32_t* max_dc, int32_t* max_dv) {
    if (!h) return fail(LDPC_ERR_BAD_POINTER);
    if (M) *M = h->M;
    if (N) *N = h->N;
    if (E) *E = h->E;
    if (max_dc) *max_dc = h->max_dc;
    if (max_dv) *max_dv = h->max_dv;
    return LDPC_OK;
}

int ldpc_last_kernel_count(const ldpc_t* h, int32_t* count) {
    if (!h || !count) return fail(LDPC_ERR_BAD_POINTER);
    *count = h->last_launches;
    return LDPC_OK;
}

int ldpc_last_error(void) { return g_last_error; }
int ldpc_last_cuda_error(void) { return g_last_cuda; }

const char* ldpc_strerror(int status) {
    switch (status) {
        case LDPC_OK: return "ok";
        case LDPC_ERR_INVALID_ARG: return "invalid argument";
        case LDPC_ERR_INVALID_H: return "invalid parity matrix";
        case LDPC_ERR_BAD_POINTER: return "bad pointer (NULL, or host memory where device memory is required)";
        case LDPC_ERR_OOM: return "out of memory";
        case LDPC_ERR_CUDA: return "CUDA runtime error";
        case LDPC_ERR_TIMEOUT: return "a bounded wait inside a kernel ran out";
        case LDPC_ERR_DEVICE_CHECK: return "the debug checks found a NaN LLR or an index out of range";
        case LDPC_ERR_UNSUPPORTED: return "unsupported for this code or device";
    }
    return "unknown status";
}

void ldpc_destroy(ldpc_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->h2d) {
        cudaStreamSynchronize(h->h2d);
        cudaStreamSynchronize(h->d2h);
        for (int s = 0; s < 2; s++) {
            if (h->stage[s]) cudaFree(h->stage[s]);
            cudaEventDestroy(h->ev_h2d[s]);
            cudaEventDestroy(h->ev_comp[s]);
            cudaEventDestroy(h->ev_d2h[s]);
        }
        cudaStreamDestroy(h->h2d);
        cudaStreamDestroy(h->d2h);
    }
    free_stream_work(h);
    free_graph(h->dg);
    for (auto& c : h->dcl) free_cluster(c);
    if (h->counters) cudaFree(h->counters);
    if (h->w_alpha) cudaFree(h->w_alpha);
    if (h->dense_work) cudaFree(h->dense_work);
    delete h;
}

}  // extern "C"
