// Decoding without device allocation: ldpc_decode_noalloc.
//
// Some callers cannot call cudaMalloc while they decode: a serving loop that must not
// stall on the allocator (cudaMalloc and cudaFree can synchronise the whole device),
// a process whose device memory is already fully reserved by another allocator (a
// framework's caching pool), or an embedding that forbids allocation after start-up.
// For them this entry point runs the streaming kernels with their scratch (edge
// messages, posteriors, channel values, per-frame flags) carved from one statically
// sized device array that the library defines, instead of the handle's workspace.
//
// The array is a file-scope __device__ variable: in host code its name is only a
// stand-in, so its device address is looked up with cudaGetSymbolAddress once per
// device, with that device current. The lookup is what maps the array (under CUDA's lazy
// module loading this translation unit's module, and the array with it, is loaded on its
// first use), so it runs when a handle is created on the device (noalloc_setup, called
// by ldpc_create / ldpc_create_ex), never inside ldpc_decode_noalloc itself.
#include <mutex>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace {

constexpr size_t kScratchBytes = LDPC_NOALLOC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the static scratch array on `device` (which must be current).
cudaError_t scratch_address(int device, void** out) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[device] = p;
    }
    *out = g_scratch_addr[device];
    return cudaSuccess;
}

}  // namespace

// Maps the scratch array on `device` (current) and caches its address: called once per
// handle creation. Returns LDPC_OK, LDPC_ERR_OOM when the array cannot be mapped for lack
// of memory, or LDPC_ERR_CUDA; the runtime's pending error is cleared on failure.
int ldpc_impl::noalloc_setup(int device) {
    if (device < 0 || device >= kMaxDevices) return LDPC_OK;  // the entry point refuses these
    void* p = nullptr;
    const cudaError_t e = scratch_address(device, &p);
    if (e == cudaSuccess) return LDPC_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? LDPC_ERR_OOM : LDPC_ERR_CUDA;
}

namespace {

int is_device(const void* p) {
    if (!p) return 0;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" int ldpc_decode_noalloc(ldpc_t* h, const void* llr, int32_t llr_dtype, int32_t frames,
                                   int32_t max_iter, int32_t early_stop, int32_t check_every,
                                   uint8_t* out_bits, int32_t* out_iters, uint8_t* out_ok,
                                   float* out_soft) {
    using namespace ldpc_impl;
    HandleView v;
    if (handle_view(h, &v) != LDPC_OK) return LDPC_ERR_BAD_POINTER;
    if (frames < 0 || max_iter < 0 || check_every < 1) return LDPC_ERR_INVALID_ARG;
    if (llr_dtype != LDPC_LLR_F32 && llr_dtype != LDPC_LLR_I8) return LDPC_ERR_INVALID_ARG;
    if (llr_dtype == LDPC_LLR_I8 && v.mode != kModeFixed) return LDPC_ERR_INVALID_ARG;
    if (v.w_rows > 0 && v.mode != kModeFP32) return LDPC_ERR_UNSUPPORTED;
    *v.last_launches = 0;
    if (frames == 0) return LDPC_OK;
    int device = -1;
    if (cudaGetDevice(&device) != cudaSuccess || device != v.device || device >= kMaxDevices)
        return LDPC_ERR_INVALID_ARG;
    if (!is_device(llr) || !is_device(out_bits) || !is_device(out_iters) ||
        (out_ok && !is_device(out_ok)) || (out_soft && !is_device(out_soft)))
        return LDPC_ERR_BAD_POINTER;
    // the scratch this request needs, laid out as the streaming workspace
    if (frames > (int32_t)(kScratchBytes / 8)) return LDPC_ERR_INVALID_ARG;  // cannot fit
    const int32_t Fp = (frames + 255) & ~255;
    const size_t tb = v.mode == kModeFP32 ? 4 : 2, rb = v.mode == kModeFP32 ? 4 : 1;
    const size_t o_eta = 0;
    const size_t o_s = o_eta + al256((size_t)v.dg->eta_slots * Fp * tb);
    const size_t o_r = o_s + al256((size_t)v.N * Fp * tb);
    const size_t o_done = o_r + al256((size_t)v.N * Fp * rb);
    const size_t o_p2f = o_done + al256((size_t)Fp * 4);
    const size_t o_newpos = o_p2f + al256((size_t)Fp * 4);
    const size_t o_state = o_newpos + al256((size_t)Fp * 4);
    const size_t o_unsat = o_state + al256((size_t)Fp);
    const size_t o_count = o_unsat + al256((size_t)(max_iter + 2) * Fp);
    const size_t need = o_count + 256;
    if (need > kScratchBytes) return LDPC_ERR_INVALID_ARG;  // request larger than the array
    char* base = nullptr;
    {  // set at handle creation on this device (noalloc_setup); no lookup happens here
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        base = (char*)g_scratch_addr[device];
    }
    if (!base) return LDPC_ERR_UNSUPPORTED;
    StreamWork w;
    w.Fp = Fp;
    w.eta = base + o_eta;
    w.s = base + o_s;
    w.r = base + o_r;
    w.done_iter = (int32_t*)(base + o_done);
    w.state = (uint8_t*)(base + o_state);
    w.unsat = (uint8_t*)(base + o_unsat);
    w.n_done = (int32_t*)(base + o_count);
    w.pos2frame = (int32_t*)(base + o_p2f);
    w.new_pos = (int32_t*)(base + o_newpos);
    w.comp = w.n_done + 4;  // in the 256 bytes after the done counter
    w.err = v.err;  // the handle's device error word (ldpc_check_device)
    w.num_sms = v.num_sms;
    w.stage_warps = v.stage_warps;
    w.stages = v.stages;
    w.stage_vw = v.stage_vw;
    w.wait_limit = v.wait_limit;
    w.msg_compressed = v.msg_compressed;
    DecodeArgs a;
    a.M = v.M;
    a.N = v.N;
    a.E = (int32_t)v.E;
    a.frames = frames;
    a.L = max_iter;
    a.early_stop = early_stop ? 1 : 0;
    a.check_every = check_every;
    a.paper_slicer = (v.flags & LDPC_FLAG_PAPER_SLICER) ? 1 : 0;
    a.llr_is_i8 = llr_dtype == LDPC_LLR_I8;
    a.llr = llr;
    a.out_bits = out_bits;
    a.out_iters = out_iters;
    a.out_ok = out_ok;
    a.out_soft = out_soft;
    if (v.w_rows > 0) {  // learned weights set on the handle
        a.w_rows = v.w_rows;
        a.n_classes = v.dg->n_classes;
        a.w_alpha = v.w_alpha;
        a.w_beta = v.w_alpha + (size_t)v.w_rows * v.dg->n_classes;
    }
    // the kernels clear the done counter and the syndrome flags and set the frame state
    const int n = stream_decode(v.mode, *v.dg, a, w, v.stream);
    if (n < 0) {  // a failed launch leaves its error pending: clear it and report it
        const cudaError_t e = cudaGetLastError();
        return e != cudaSuccess ? LDPC_ERR_CUDA : n;
    }
    *v.last_launches = n;
    return LDPC_OK;
}
