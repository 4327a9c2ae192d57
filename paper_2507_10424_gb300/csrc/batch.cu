// Batched decoding of several codes of uneven size in one persistent launch.
//
// One kernel decodes the frames of every code in the batch: its CTAs take tiles (code,
// frame) from a single atomic work counter, largest codes first, and run every flooding
// iteration of the tile with the resident variant's tile body (decode_tile). A code whose
// frame fits the launch's shared memory keeps eta, s and r there. A code too large for
// that is, by default, decoded by the streaming kernels on one of two streams forked from
// the batch's stream (so they can fill the SMs that the persistent kernel's last tiles
// leave idle, and the launch gaps of each other's passes); optionally it joins the persistent launch instead, with eta, s and r in
// the CTA's own slot of a global scratch buffer. The index arrays of every code are read
// from global memory. FP32 mode.
//
// The launch (a memset of the work counter, the kernel, and the streaming kernels of the
// large codes between a fork and a join event) touches only buffers fixed when the batch
// is prepared, so it can be recorded once in a CUDA graph and replayed
// (ldpc_batch_capture / ldpc_batch_replay).
#include <algorithm>
#include <new>
#include <vector>

#include "resident.cuh"

namespace ldpc_impl {
namespace resident {
namespace {

struct CodeDesc {
    ResArgs a;        // graph, sizes, inputs and outputs of this code for the call
    int32_t in_smem;  // eta, s, r of a tile in shared memory (else in the CTA's scratch slot)
    int32_t ft;       // frames interleaved per tile: 1, 2 or 4
};

struct Tile {
    int32_t code, f0;
};

// The tile body for FT interleaved frames at `base` (shared memory or a scratch slot).
template <int FT, bool PAPER, bool ES>
__device__ __forceinline__ void multi_tile(const ResArgs& a, const Idx& ix, char* base,
                                           uint32_t* unsat_w, int f0) {
    using VT = VecR<float, FT>;
    VT* eta = reinterpret_cast<VT*>(base);
    VT* s = eta + a.E_pad;
    VT* r = s + a.n_csl * 32;
    decode_tile<kModeFP32, FT, PAPER, false, VT, true, ES>(a, ix, eta, s, r, unsat_w, f0, min(FT, a.frames - f0),
                                             nullptr, nullptr, a.n_rsl * 32);
}

// ES: the early-stop form of the tile body (the syndrome gathered by the row pass).
template <bool PAPER, bool ES>
__global__ void __launch_bounds__(kMaxThreads, 1) k_multi(const CodeDesc* codes, const Tile* tiles,
                                                          int n_tiles, int32_t* counter,
                                                          char* scratch, size_t slot_bytes) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t unsat_w[2];
    __shared__ int tile_sh;
    __shared__ CodeDesc cd;
    for (;;) {
        if (threadIdx.x == 0) {
            tile_sh = atomicAdd(counter, 1);
            unsat_w[0] = 0;
            unsat_w[1] = 0;
        }
        __syncthreads();
        const int t = tile_sh;
        if (t >= n_tiles) break;
        const Tile tl = tiles[t];
        if (threadIdx.x == 0) cd = codes[tl.code];
        __syncthreads();
        const ResArgs& a = cd.a;
        const Idx ix{a.r_base, a.r_deg, a.r_slot_pos, a.c_base, a.c_deg, a.c_slot, a.col_pos,
                     nullptr, nullptr, nullptr};
        if (cd.in_smem) {
            char* base = reinterpret_cast<char*>(smem_raw);
            if (cd.ft == 4) multi_tile<4, PAPER, ES>(a, ix, base, unsat_w, tl.f0);
            else if (cd.ft == 2) multi_tile<2, PAPER, ES>(a, ix, base, unsat_w, tl.f0);
            else multi_tile<1, PAPER, ES>(a, ix, base, unsat_w, tl.f0);
        } else {
            char* base = scratch + (size_t)blockIdx.x * slot_bytes;
            if (cd.ft == 2) multi_tile<2, PAPER, ES>(a, ix, base, unsat_w, tl.f0);
            else multi_tile<1, PAPER, ES>(a, ix, base, unsat_w, tl.f0);
        }
        __syncthreads();
    }
}

size_t frame_bytes(const DevGraph& g) { return ((size_t)g.E_pad + 2 * (size_t)g.n_cslices * 32) * 4; }

}  // namespace
}  // namespace resident
}  // namespace ldpc_impl

using namespace ldpc_impl;
using namespace ldpc_impl::resident;

struct ldpc_batch {
    int device = 0, num_sms = 0;
    std::vector<ldpc_t*> codes;
    std::vector<HandleView> views;
    std::vector<CodeDesc> desc;  // host copies
    std::vector<int32_t> frames;
    std::vector<int32_t> fit_ft;  // most frames per tile that fit shared memory (in_smem codes)
    std::vector<size_t> fbytes;   // bytes of one frame's eta, s and r
    int ft_cap = 4;               // frames per tile at most (ldpc_batch_set_tile_frames)
    int paper = 0;
    int es = 0;                   // the prepared decode tests the syndrome every iteration
    CodeDesc* d_desc = nullptr;
    Tile* d_tiles = nullptr;
    int32_t n_tiles = 0, tiles_cap = 0;
    int32_t* d_counter = nullptr;
    char* d_scratch = nullptr;
    size_t slot_bytes = 0, smem = 0;
    int threads = 512, grid = 0;
    cudaStream_t stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t last_launches = 0, captured_launches = 0;
    // codes too large for shared memory: streaming kernels (1) or the persistent launch (0)
    int large_stream = 1;
    // SMs of the persistent kernel while streamed codes run beside it (0: all of them);
    // the streaming kernels' persistent passes then size their grids to the other SMs
    int32_t sm_split = 0;
    struct Streamed {
        int32_t code;
        DecodeArgs a;
        StreamWork w;
        void* mem = nullptr;
        size_t bytes = 0;
    };
    std::vector<Streamed> streamed;
    // the streamed codes alternate between two side streams (their passes fill each
    // other's launch gaps and tails)
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr, join2 = nullptr;
};

static void batch_free(ldpc_batch_t* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& x : b->streamed)
        if (x.mem) cudaFree(x.mem);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->side2) cudaStreamDestroy(b->side2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    if (b->join2) cudaEventDestroy(b->join2);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_tiles) cudaFree(b->d_tiles);
    if (b->d_counter) cudaFree(b->d_counter);
    if (b->d_scratch) cudaFree(b->d_scratch);
    delete b;
}

using MultiKernel = void (*)(const CodeDesc*, const Tile*, int, int32_t*, char*, size_t);

// The standard slicer has the early-stop form; the paper's slicer tests the syndrome in
// a pass of its own.
static MultiKernel multi_kernel(const ldpc_batch_t* b) {
    if (b->paper) return k_multi<true, false>;
    return b->es ? k_multi<false, true> : k_multi<false, false>;
}

static int batch_occupancy(ldpc_batch_t* b, int threads, int* grid) {
    auto kern = multi_kernel(b);
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem) != cudaSuccess)
        return LDPC_ERR_CUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, b->smem) != cudaSuccess ||
        per_sm < 1)
        return LDPC_ERR_UNSUPPORTED;
    *grid = b->num_sms * per_sm;
    return LDPC_OK;
}

// Enqueue the launch (capturable): the streaming decodes of the large codes on the two
// side streams between a fork and join events, the work counter reset and the persistent
// kernel on the batch's stream. Returns the number of kernels enqueued, or a negative status.
static int batch_enqueue(ldpc_batch_t* b) {
    int launches = 0;
    const bool side = !b->streamed.empty();
    const bool two = b->streamed.size() > 1;
    if (side) {
        if (cudaEventRecord(b->fork, b->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->side, b->fork, 0) != cudaSuccess ||
            (two && cudaStreamWaitEvent(b->side2, b->fork, 0) != cudaSuccess))
            return LDPC_ERR_CUDA;
        for (size_t k = 0; k < b->streamed.size(); k++) {
            const auto& x = b->streamed[k];
            if (x.a.frames == 0) continue;
            const int n = stream_decode(kModeFP32, *b->views[x.code].dg, x.a, x.w, (k & 1) ? b->side2 : b->side);
            if (n < 0) return n;
            launches += n;
        }
    }
    if (cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), b->stream) != cudaSuccess) return LDPC_ERR_CUDA;
    if (b->n_tiles > 0) {
        int grid = std::min(b->grid, b->n_tiles);
        if (side && b->sm_split > 0)  // leave the other SMs to the streaming kernels
            grid = std::min(grid, b->sm_split * std::max(1, b->grid / std::max(1, b->num_sms)));
        multi_kernel(b)<<<grid, b->threads, b->smem, b->stream>>>(b->d_desc, b->d_tiles, b->n_tiles,
                                                                  b->d_counter, b->d_scratch,
                                                                  b->slot_bytes);
        launches++;
    }
    if (side && (cudaEventRecord(b->join, b->side) != cudaSuccess ||
                 cudaStreamWaitEvent(b->stream, b->join, 0) != cudaSuccess))
        return LDPC_ERR_CUDA;
    if (two && (cudaEventRecord(b->join2, b->side2) != cudaSuccess ||
                cudaStreamWaitEvent(b->stream, b->join2, 0) != cudaSuccess))
        return LDPC_ERR_CUDA;
    return cudaGetLastError() == cudaSuccess ? launches : LDPC_ERR_CUDA;
}

extern "C" {

ldpc_batch_t* ldpc_batch_create(int32_t n_codes, ldpc_t* const* codes) {
    if (n_codes <= 0 || n_codes > 4096 || !codes) return nullptr;
    ldpc_batch_t* b = new (std::nothrow) ldpc_batch();
    if (!b) return nullptr;
    int optin = 0;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return nullptr;
    }
    const size_t budget = (size_t)std::max(0, optin - 1024);
    size_t slot = 0;
    constexpr int kScratchFT = 2;  // frames per tile of the codes kept in global scratch
    for (int32_t c = 0; c < n_codes; c++) {
        HandleView v;
        if (handle_view(codes[c], &v) != LDPC_OK || !v.dg->sliced || v.device != b->device) {
            delete b;
            return nullptr;
        }
        if (c == 0) b->paper = (v.flags & LDPC_FLAG_PAPER_SLICER) ? 1 : 0;
        if (b->paper != ((v.flags & LDPC_FLAG_PAPER_SLICER) ? 1 : 0)) {  // one slicer per batch
            delete b;
            return nullptr;
        }
        b->codes.push_back(codes[c]);
        b->views.push_back(v);
        const size_t fb = frame_bytes(*v.dg);
        CodeDesc d{};
        d.in_smem = fb <= budget;
        d.ft = 1;
        if (d.in_smem) {
            d.ft = 4 * fb <= budget ? 4 : (2 * fb <= budget ? 2 : 1);
            b->smem = std::max(b->smem, (size_t)d.ft * fb);
        }
        b->fit_ft.push_back(d.ft);
        b->fbytes.push_back(fb);
        if (!d.in_smem) {
            d.ft = kScratchFT;
            slot = std::max(slot, (size_t)kScratchFT * fb);
        }
        b->desc.push_back(d);
        b->frames.push_back(0);
    }
    b->slot_bytes = (slot + 255) & ~(size_t)255;
    cudaError_t e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join2, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_desc, sizeof(CodeDesc) * n_codes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(int32_t));
    if (e == cudaSuccess && batch_occupancy(b, b->threads, &b->grid) != LDPC_OK) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess && b->slot_bytes) e = cudaMalloc((void**)&b->d_scratch, b->slot_bytes * b->grid);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(b);
        return nullptr;
    }
    return b;
}

int ldpc_batch_set_stream(ldpc_batch_t* b, void* stream) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    b->stream = (cudaStream_t)stream;
    return LDPC_OK;
}

int ldpc_batch_set_io(ldpc_batch_t* b, int32_t code, const float* llr, int32_t frames,
                      uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok, float* out_soft) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (code < 0 || code >= (int32_t)b->codes.size() || frames < 0) return LDPC_ERR_INVALID_ARG;
    if (frames > 0 && (!llr || !out_bits || !out_iters)) return LDPC_ERR_BAD_POINTER;
    const HandleView& v = b->views[code];
    const DevGraph& g = *v.dg;
    ResArgs& a = b->desc[code].a;
    a = ResArgs{};
    a.r_base = g.r_base;
    a.r_deg = g.r_deg;
    a.r_slot_pos = g.r_slot_pos;
    a.c_base = g.c_base;
    a.c_deg = g.c_deg;
    a.c_slot = g.c_slot;
    a.col_pos = g.col_pos;
    a.r_slot_cls = g.r_slot_cls;
    a.n_rsl = g.n_rslices;
    a.n_csl = g.n_cslices;
    a.E_pad = g.E_pad;
    a.Ec_pad = g.Ec_pad;
    a.N = v.N;
    a.llr = llr;
    a.frames = frames;
    a.paper = b->paper;
    a.out_bits = out_bits;
    a.out_iters = out_iters;
    a.out_ok = out_ok;
    a.out_soft = out_soft;
    b->frames[code] = frames;
    return LDPC_OK;
}

// Upload the descriptors and the tile list for max_iter / early_stop (synchronous).
int ldpc_batch_prepare(ldpc_batch_t* b, int32_t max_iter, int32_t early_stop) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (max_iter < 0) return LDPC_ERR_INVALID_ARG;
    const int es = early_stop ? 1 : 0;
    if (es != b->es) {  // the other kernel form: its occupancy sets the grid
        const int keep = b->es;
        b->es = es;
        const int rc = ldpc_batch_set_threads(b, b->threads);
        if (rc != LDPC_OK) {
            b->es = keep;
            return rc;
        }
    }
    std::vector<int32_t> order(b->codes.size());
    for (size_t c = 0; c < order.size(); c++) {
        order[c] = (int32_t)c;
        ResArgs& a = b->desc[c].a;
        a.L = max_iter;
        a.early_stop = early_stop ? 1 : 0;
        a.check_every = 1;
    }
    // largest frames first: the last tiles to start are the short ones
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return b->views[x].E > b->views[y].E;
    });
    std::vector<Tile> tiles;
    std::vector<ldpc_batch::Streamed> keep;
    for (int32_t c : order) {
        if (b->large_stream && !b->desc[c].in_smem) {
            // the streaming decode of this code: workspace sized for its frames and max_iter
            ldpc_batch::Streamed x;
            for (auto& old : b->streamed)
                if (old.code == c) {
                    x = old;
                    old.mem = nullptr;
                }
            const ResArgs& ra = b->desc[c].a;
            const HandleView& v = b->views[c];
            const int32_t Fp = (b->frames[c] + 255) & ~255;
            const size_t need = stream_bytes(kModeFP32, v.N, v.dg->eta_slots, Fp, max_iter);
            if (need > x.bytes) {
                if (x.mem) {
                    cudaStreamSynchronize(b->side);
                    cudaStreamSynchronize(b->side2);
                    cudaFree(x.mem);
                }
                x.mem = nullptr;
                x.bytes = 0;
                if (cudaMalloc(&x.mem, need) != cudaSuccess) {
                    cudaGetLastError();
                    for (auto& y : keep) cudaFree(y.mem);
                    return LDPC_ERR_OOM;
                }
                x.bytes = need;
            }
            x.code = c;
            x.w = stream_carve(kModeFP32, x.mem, v.N, v.dg->eta_slots, Fp, max_iter);
            x.w.err = v.err;  // the code handle's device error word (ldpc_check_device)
            x.w.num_sms = b->sm_split > 0 ? std::max(1, v.num_sms - b->sm_split) : v.num_sms;
            x.w.stage_warps = v.stage_warps;
            x.w.stages = v.stages;
            x.w.stage_vw = v.stage_vw;
            x.w.wait_limit = v.wait_limit;
            x.w.msg_compressed = v.msg_compressed;
            DecodeArgs& a = x.a;
            a = DecodeArgs();
            a.M = v.M;
            a.N = v.N;
            a.E = (int32_t)v.E;
            a.frames = b->frames[c];
            a.L = max_iter;
            a.early_stop = early_stop ? 1 : 0;
            a.check_every = 1;
            a.paper_slicer = b->paper;
            a.llr_is_i8 = 0;
            a.llr = ra.llr;
            a.out_bits = ra.out_bits;
            a.out_iters = ra.out_iters;
            a.out_ok = ra.out_ok;
            a.out_soft = ra.out_soft;
            keep.push_back(x);
            continue;
        }
        for (int32_t f = 0; f < b->frames[c]; f += b->desc[c].ft) tiles.push_back(Tile{c, f});
    }
    for (auto& old : b->streamed)
        if (old.mem) {
            cudaStreamSynchronize(b->side);
            cudaStreamSynchronize(b->side2);
            cudaFree(old.mem);
        }
    b->streamed = keep;
    if (b->exec) {  // a recorded launch refers to the old work list: record again
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    if ((int32_t)tiles.size() > b->tiles_cap) {
        if (b->d_tiles) cudaFree(b->d_tiles);
        b->d_tiles = nullptr;
        if (cudaMalloc((void**)&b->d_tiles, sizeof(Tile) * tiles.size()) != cudaSuccess) {
            cudaGetLastError();
            b->tiles_cap = 0;
            return LDPC_ERR_OOM;
        }
        b->tiles_cap = (int32_t)tiles.size();
    }
    b->n_tiles = (int32_t)tiles.size();
    if (cudaStreamSynchronize(b->stream) != cudaSuccess ||
        cudaMemcpy(b->d_desc, b->desc.data(), sizeof(CodeDesc) * b->desc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        (b->n_tiles && cudaMemcpy(b->d_tiles, tiles.data(), sizeof(Tile) * tiles.size(), cudaMemcpyHostToDevice) != cudaSuccess))
        return LDPC_ERR_CUDA;
    return LDPC_OK;
}

int ldpc_batch_launch(ldpc_batch_t* b) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    const int n = batch_enqueue(b);
    b->last_launches = n < 0 ? 0 : n;
    return n < 0 ? n : LDPC_OK;
}

int ldpc_batch_set_large_codes(ldpc_batch_t* b, int32_t streaming) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (streaming != 0 && streaming != 1) return LDPC_ERR_INVALID_ARG;
    b->large_stream = streaming;
    return LDPC_OK;  // takes effect at the next ldpc_batch_prepare
}

int ldpc_batch_set_sm_split(ldpc_batch_t* b, int32_t sms) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (sms < 0 || sms >= b->num_sms) return LDPC_ERR_INVALID_ARG;
    b->sm_split = sms;
    return LDPC_OK;  // takes effect at the next ldpc_batch_prepare
}

int ldpc_batch_get_sm_split(const ldpc_batch_t* b, int32_t* sms) {
    if (!b || !sms) return LDPC_ERR_BAD_POINTER;
    *sms = b->sm_split;
    return LDPC_OK;
}

int ldpc_batch_decode(ldpc_batch_t* b, int32_t max_iter, int32_t early_stop) {
    const int rc = ldpc_batch_prepare(b, max_iter, early_stop);
    return rc != LDPC_OK ? rc : ldpc_batch_launch(b);
}

int ldpc_batch_capture(ldpc_batch_t* b) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (!b->stream) return LDPC_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return LDPC_ERR_CUDA;
    const int n = batch_enqueue(b);
    const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
    if (n >= 0) b->captured_launches = n;
    if (n < 0 || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return LDPC_ERR_CUDA;
    }
    const cudaError_t e2 = cudaGraphInstantiate(&b->exec, g, 0);
    cudaGraphDestroy(g);
    if (e2 != cudaSuccess) {
        b->exec = nullptr;
        cudaGetLastError();
        return LDPC_ERR_CUDA;
    }
    return LDPC_OK;
}

int ldpc_batch_replay(ldpc_batch_t* b) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (!b->exec) return LDPC_ERR_INVALID_ARG;
    b->last_launches = b->captured_launches;
    return cudaGraphLaunch(b->exec, b->stream) == cudaSuccess ? LDPC_OK : LDPC_ERR_CUDA;
}

int ldpc_batch_set_threads(ldpc_batch_t* b, int32_t threads) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (threads < 64 || threads > kMaxThreads || threads % 32) return LDPC_ERR_INVALID_ARG;
    int grid = 0;
    const int rc = batch_occupancy(b, threads, &grid);
    if (rc != LDPC_OK) return rc;
    if (grid > b->grid && b->slot_bytes) {  // more CTAs need more scratch slots
        char* p = nullptr;
        if (cudaMalloc((void**)&p, b->slot_bytes * grid) != cudaSuccess) {
            cudaGetLastError();
            return LDPC_ERR_OOM;
        }
        cudaStreamSynchronize(b->stream);
        cudaFree(b->d_scratch);
        b->d_scratch = p;
    }
    b->threads = threads;
    b->grid = grid;
    if (b->exec) {  // a recorded launch keeps its old shape: record again
        cudaGraphExecDestroy(b->exec);
        b->exec = nullptr;
    }
    return LDPC_OK;
}

int ldpc_batch_set_tile_frames(ldpc_batch_t* b, int32_t max_frames_per_tile) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    const int cap = max_frames_per_tile;
    if (cap != 1 && cap != 2 && cap != 4) return LDPC_ERR_INVALID_ARG;
    const int keep_cap = b->ft_cap;
    const size_t keep_smem = b->smem;
    std::vector<int32_t> keep_ft;
    size_t smem = 0;
    for (size_t c = 0; c < b->desc.size(); c++) {
        keep_ft.push_back(b->desc[c].ft);
        if (!b->desc[c].in_smem) continue;
        b->desc[c].ft = std::min(b->fit_ft[c], cap);
        smem = std::max(smem, (size_t)b->desc[c].ft * b->fbytes[c]);
    }
    b->ft_cap = cap;
    b->smem = smem;
    const int rc = ldpc_batch_set_threads(b, b->threads);  // the grid follows the new smem
    if (rc != LDPC_OK) {
        b->ft_cap = keep_cap;
        b->smem = keep_smem;
        for (size_t c = 0; c < b->desc.size(); c++) b->desc[c].ft = keep_ft[c];
    }
    return rc;  // the tiles follow at the next ldpc_batch_prepare
}

int ldpc_batch_get_tile_frames(const ldpc_batch_t* b, int32_t* max_frames_per_tile) {
    if (!b || !max_frames_per_tile) return LDPC_ERR_BAD_POINTER;
    *max_frames_per_tile = b->ft_cap;
    return LDPC_OK;
}

int ldpc_batch_autotune(ldpc_batch_t* b, int32_t max_iter, int32_t early_stop, int32_t* best_threads,
                        float* best_ms) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return LDPC_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return LDPC_ERR_CUDA;
    }
    float best = -1.0f;
    const int keep_t = b->threads, keep_cap = b->ft_cap;
    int best_t = keep_t, best_cap = keep_cap;
    int rc = LDPC_OK;
    // frames per tile at most x CTA size: with early stop a tile runs until its last frame
    // stops, so narrower tiles can win although they share less of each index read
    for (int cap : {4, 2, 1}) {
        if (ldpc_batch_set_tile_frames(b, cap) != LDPC_OK) continue;
        rc = ldpc_batch_prepare(b, max_iter, early_stop);
        if (rc != LDPC_OK) break;
        for (int th = 128; th <= kMaxThreads; th += 128) {
            if (ldpc_batch_set_threads(b, th) != LDPC_OK) continue;
            float ms = 0.0f;
            bool bad = batch_enqueue(b) < 0 || cudaEventRecord(e0, b->stream) != cudaSuccess;
            for (int r = 0; r < 2 && !bad; r++) bad = batch_enqueue(b) < 0;
            bad = bad || cudaEventRecord(e1, b->stream) != cudaSuccess ||
                  cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
            if (bad) {
                cudaGetLastError();
                continue;
            }
            if (best < 0.0f || ms < best) {
                best = ms;
                best_t = th;
                best_cap = cap;
            }
        }
    }
    // with codes streamed beside the persistent kernel: the SMs it keeps (the resident
    // tiles are bound on chip, the streaming passes by DRAM, so disjoint SM sets can run
    // both near their own limits)
    const int32_t keep_split = b->sm_split;
    int32_t best_split = keep_split;
    if (rc == LDPC_OK && best >= 0.0f && ldpc_batch_set_tile_frames(b, best_cap) == LDPC_OK &&
        ldpc_batch_set_threads(b, best_t) == LDPC_OK) {
        for (int q : {0, 8, 6, 5, 4, 3}) {  // 0: no split; else num_sms / q SMs
            const int32_t split = q ? std::max(1, b->num_sms / q) : 0;
            b->sm_split = split;
            if (ldpc_batch_prepare(b, max_iter, early_stop) != LDPC_OK) continue;
            if (b->streamed.empty() && split) break;  // nothing runs beside the kernel
            float ms = 0.0f;
            bool bad = batch_enqueue(b) < 0 || cudaEventRecord(e0, b->stream) != cudaSuccess;
            for (int r = 0; r < 2 && !bad; r++) bad = batch_enqueue(b) < 0;
            bad = bad || cudaEventRecord(e1, b->stream) != cudaSuccess ||
                  cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess;
            if (bad) {
                cudaGetLastError();
                continue;
            }
            if (ms < best) {
                best = ms;
                best_split = split;
            }
        }
    }
    b->sm_split = best_split;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != LDPC_OK || best < 0.0f) {  // leave the shape the caller had
        b->sm_split = keep_split;
        ldpc_batch_set_tile_frames(b, keep_cap);
        ldpc_batch_set_threads(b, keep_t);
        return rc != LDPC_OK ? rc : LDPC_ERR_UNSUPPORTED;
    }
    rc = ldpc_batch_set_tile_frames(b, best_cap);
    if (rc == LDPC_OK) rc = ldpc_batch_set_threads(b, best_t);
    if (rc == LDPC_OK) rc = ldpc_batch_prepare(b, max_iter, early_stop);
    if (best_threads) *best_threads = best_t;
    if (best_ms) *best_ms = best / 2.0f;
    return rc;
}

int ldpc_batch_info(const ldpc_batch_t* b, int32_t* n_codes, int32_t* n_tiles, int32_t* threads,
                    int32_t* codes_in_shared_memory) {
    if (!b) return LDPC_ERR_BAD_POINTER;
    if (n_codes) *n_codes = (int32_t)b->codes.size();
    if (n_tiles) *n_tiles = b->n_tiles;
    if (threads) *threads = b->threads;
    if (codes_in_shared_memory) {
        int32_t n = 0;
        for (const auto& d : b->desc) n += d.in_smem;
        *codes_in_shared_memory = n;
    }
    return LDPC_OK;
}

void ldpc_batch_destroy(ldpc_batch_t* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    batch_free(b);
}

}  // extern "C"
