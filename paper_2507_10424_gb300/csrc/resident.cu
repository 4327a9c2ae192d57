// Resident variant, host side: the launch plan (frames per tile, index placement,
// register budget of the row sweep, CTA size) and the decode entry used by the C ABI.
#include "resident.cuh"

namespace ldpc_impl {
using namespace resident;

ResidentPlan resident_plan(int mode, const DevGraph& dg, int32_t N, int device,
                           const ResidentTuning& tune, int w_entries) {
    ResidentPlan p;
    if (!dg.sliced) return p;
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    const int tb = mode == kModeFP32 ? 4 : 2;
    const size_t budget = (size_t)std::max(0, optin - 256);  // static shared memory
    // up to four interleaved frames (registers); index arrays in shared memory preferred
    const int fts[] = {4, 2, 1};
    for (int idx = 1; idx >= 0 && !p.ok; idx--)
        for (int ft : fts) {
            if ((tune.idx == 1 && !idx) || (tune.idx == 2 && idx)) continue;
            if (ft * tb > 16 || (!idx && ft > 2)) continue;
            if (tune.FT && ft != tune.FT) continue;
            const ResLayout L = res_layout(tb, ft, dg.E_pad, dg.Ec_pad, dg.n_rslices, dg.n_cslices, N, idx,
                                           mode == kModeFP32 ? w_entries : 0);
            if (L.total <= budget) {
                p.ok = 1;
                p.FT = ft;
                p.idx_smem = idx;
                p.smem = L.total;
                break;
            }
        }
    if (!p.ok) return p;
    if (tune.threads) {
        if (tune.threads % 32 || tune.threads < 64 || tune.threads > kMaxThreads) return ResidentPlan();
        p.threads = tune.threads;
        return p;
    }
    // threads: balance latency hiding (resident warps per SM, counted up to 24) against
    // the padding of the last round of row and column tasks (rows weigh twice: two sweeps)
    int per_sm = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    const int ctas_smem = std::max(1, (int)(per_sm / (p.smem + 1024)));
    const int rt = dg.n_rslices * 32;
    const double useful = 2.0 * rt + N;
    double best = -1.0;
    for (int t = 256; t <= kMaxThreads; t += 32) {
        const int ctas = std::min(ctas_smem, 2048 / t);
        const double warps = std::min(24.0, (double)ctas * t / 32.0);
        const double padded = 2.0 * ((rt + t - 1) / t) * t + (double)((N + t - 1) / t) * t;
        const double score = warps * useful / padded;
        if (score > best + 1e-9) {
            best = score;
            p.threads = t;
        }
    }
    return p;
}

int resident_decode(int mode, const DevGraph& dg, const ResidentPlan& p, const DecodeArgs& a,
                    int32_t* tile_counter, int num_sms, cudaStream_t st) {
    ResArgs ra;
    ra.r_base = dg.r_base;
    ra.r_deg = dg.r_deg;
    ra.r_slot_pos = dg.r_slot_pos;
    ra.c_base = dg.c_base;
    ra.c_deg = dg.c_deg;
    ra.c_slot = dg.c_slot;
    ra.col_pos = dg.col_pos;
    ra.r_slot_cls = dg.r_slot_cls;
    ra.w_rows = mode == kModeFP32 ? a.w_rows : 0;
    ra.n_classes = a.n_classes;
    ra.w_alpha = a.w_alpha;
    ra.w_beta = a.w_beta;
    ra.n_rsl = dg.n_rslices;
    ra.n_csl = dg.n_cslices;
    ra.E_pad = dg.E_pad;
    ra.Ec_pad = dg.Ec_pad;
    ra.N = a.N;
    ra.llr = a.llr;
    ra.llr_i8 = a.llr_is_i8;
    ra.frames = a.frames;
    ra.n_tiles = (a.frames + p.FT - 1) / p.FT;
    ra.L = a.L;
    ra.early_stop = a.early_stop;
    ra.check_every = a.check_every;
    ra.paper = a.paper_slicer;
    ra.out_bits = a.out_bits;
    ra.out_iters = a.out_iters;
    ra.out_ok = a.out_ok;
    ra.out_soft = a.out_soft;
    ra.tile_counter = tile_counter;
    if (cudaMemsetAsync(tile_counter, 0, sizeof(int32_t), st) != cudaSuccess) return LDPC_ERR_CUDA;
    if (use_es(ra))
        return mode == kModeFP32 ? dispatch_fp32_es(ra, p, num_sms, st)
                                 : dispatch_fixed_es(ra, p, num_sms, st);
    return mode == kModeFP32 ? dispatch_fp32(ra, p, num_sms, st) : dispatch_fixed(ra, p, num_sms, st);
}

}  // namespace ldpc_impl
