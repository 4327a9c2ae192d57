// Internal declarations of the GB300 Min-Sum decoder library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/ldpc.h"

namespace ldpc_impl {

constexpr int kModeFP32 = 0;
constexpr int kModeFixed = 1;
constexpr int kSat = 32767;  // symmetric saturation limit of fixed-point messages

// ---------------------------------------------------------------------------------------
// Host-side graph of H: the check sets N_i (CSR) and bit sets M_j (CSC), Section II-B.
// Edge id = CSR position; columns ascend within a row, rows ascend within a column.
// ---------------------------------------------------------------------------------------
struct HostGraph {
    int32_t M = 0, N = 0;
    int64_t E = 0;
    std::vector<int32_t> row_ptr;   // M+1
    std::vector<int32_t> col_idx;   // E
    std::vector<int32_t> col_ptr;   // N+1
    std::vector<int32_t> col_edge;  // E: CSR edge ids of column j, ascending row
    int32_t max_dc = 0, max_dv = 0;
    // edge classes for learned weights: class of bit j = index of its column weight among
    // the sorted distinct column weights
    std::vector<int32_t> class_degree;  // n_classes
    std::vector<uint8_t> col_class;     // N
};
void assign_classes(HostGraph& g);

// Each returns LDPC_OK or an LDPC_ERR_* status.
int graph_from_dense(int32_t M, int32_t N, const uint8_t* H, HostGraph& g);
int graph_from_packed(int32_t M, int32_t N, const uint32_t* rows, HostGraph& g);
int graph_from_csr(int32_t M, int32_t N, const int64_t* row_ptr, const int32_t* col_idx,
                   HostGraph& g);

// ---------------------------------------------------------------------------------------
// Sliced layouts of the resident kernel. Rows and columns are each sorted by degree
// (descending, stable) and grouped into slices of 32 lanes; the k-th edge of lane l of
// slice s sits at base[s] + 32 k + l, so a warp's 32 lanes touch 32 consecutive entries.
//   row side:    r_slot_pos[row slot]  = sorted position of the edge's column
//   column side: c_slot[column slot]   = row slot of the edge (edges in ascending row order)
//   col_pos[j]                         = sorted position of column j
// Posteriors and channel values are stored by sorted column position.
// ---------------------------------------------------------------------------------------
struct SlicedGraph {
    int32_t n_rslices = 0, n_cslices = 0;
    int32_t E_pad = 0, Ec_pad = 0;      // row-side and column-side slots incl. padding
    std::vector<int32_t> r_base;        // n_rslices + 1
    std::vector<uint8_t> r_deg;         // 32 * n_rslices (0 for missing rows)
    std::vector<uint16_t> r_slot_pos;   // E_pad
    std::vector<int32_t> c_base;        // n_cslices + 1
    std::vector<uint8_t> c_deg;         // 32 * n_cslices (0 for missing columns)
    std::vector<uint16_t> c_slot;       // Ec_pad
    std::vector<uint16_t> col_pos;      // N
    std::vector<uint8_t> r_slot_cls;    // E_pad: class of the edge's bit (0 for padding)
};
// Returns false when the code cannot use 16-bit slot ids or 8-bit degrees.
bool build_sliced(const HostGraph& g, SlicedGraph& sg);

// ---------------------------------------------------------------------------------------
// Padded row layout of the streaming kernels (codes whose rows have at most 16 edges):
// every row owns D = 8 or 16 message slots, the t-th edge of row i at slot i D + t, so a
// row's columns and messages sit at known offsets and load without a row-pointer lookup.
//   ell_col[i D + t]  column of the t-th edge (t < deg(i)); padding repeats a valid column
//   ell_deg[i]        deg(i)
//   ell_cslot[q]      slot of the q-th edge of the CSC order (ascending rows per column)
//   ell_cls[i D + t]  learned-weight class of the edge's bit (0 for padding)
// ---------------------------------------------------------------------------------------
struct EllGraph {
    int32_t D = 0;
    std::vector<int32_t> ell_col;
    std::vector<uint8_t> ell_deg;
    std::vector<int32_t> ell_cslot;
    std::vector<uint8_t> ell_cls;
};
// Returns false when a row has more than 16 edges (the layout is then not used).
bool build_ell(const HostGraph& g, EllGraph& eg);

// ---------------------------------------------------------------------------------------
// Cluster layout: the C CTAs of a thread-block cluster share a tile of frames. CTA (rank)
// q owns a contiguous range of rows and one of columns, each cut at about E q / C edges,
// and lays them out like the sliced layout above: the messages of its rows and the
// posteriors / channel values of its columns sit in its own shared memory. A reference
// (rank << 16) | index names an entry in the shared memory of CTA `rank`:
//   r_ref[row slot]    -> (owner of the edge's column, that column's position)
//   c_ref[column slot] -> (owner of the edge's row, the edge's row slot), ascending rows
// meta[q][...] gives CTA q's column range and the offsets of its parts of the arrays.
// ---------------------------------------------------------------------------------------
enum ClMeta { kClJ0, kClJ1, kClRTasks, kClCTasks, kClRBase, kClRDeg, kClRRef, kClCBase, kClCDeg,
              kClCRef, kClMeta };
struct ClusterGraph {
    int32_t C = 0;
    int32_t E_cap = 0, P_cap = 0;      // largest per-CTA row-slot / column-position counts
    std::vector<int32_t> meta;         // [C][kClMeta]
    std::vector<int32_t> r_base, c_base;
    std::vector<uint8_t> r_deg, c_deg;
    std::vector<uint32_t> r_ref, c_ref;
    std::vector<uint8_t> r_cls;        // class of the edge's bit, by row slot (as r_ref)
    std::vector<uint16_t> pos_of_col;  // N: position of column j in its owner's layout
};
// Returns false when a CTA's part needs more than 16-bit slot ids or 8-bit degrees.
bool build_cluster(const HostGraph& g, int C, ClusterGraph& cg);

// Device copy of a cluster layout.
struct DevCluster {
    int32_t C = 0, E_cap = 0, P_cap = 0;
    int32_t* meta = nullptr;
    int32_t* r_base = nullptr;
    int32_t* c_base = nullptr;
    uint8_t* r_deg = nullptr;
    uint8_t* c_deg = nullptr;
    uint32_t* r_ref = nullptr;
    uint32_t* c_ref = nullptr;
    uint8_t* r_cls = nullptr;
    uint16_t* pos_of_col = nullptr;
};

// Device copies of the graph.
struct DevGraph {
    // CSR/CSC (streaming kernels)
    int32_t* row_ptr = nullptr;
    int32_t* col_idx = nullptr;
    int32_t* col_ptr = nullptr;
    int32_t* col_edge = nullptr;
    // bit-packed rows, uint32 [M][ceil(N/32)]
    uint32_t* packed = nullptr;
    uint8_t* col_class = nullptr;  // N
    int32_t n_classes = 0;
    // sliced layout (resident kernel)
    int32_t* r_base = nullptr;
    uint8_t* r_deg = nullptr;
    uint16_t* r_slot_pos = nullptr;
    int32_t* c_base = nullptr;
    uint8_t* c_deg = nullptr;
    uint16_t* c_slot = nullptr;
    uint16_t* col_pos = nullptr;
    uint8_t* r_slot_cls = nullptr;
    int32_t n_rslices = 0, n_cslices = 0, E_pad = 0, Ec_pad = 0;
    int32_t sliced = 0;  // the sliced layout exists
    int32_t max_dc = 0;  // longest row (set for every code)
    // padded row layout (streaming kernels); ell_D = 0 when absent
    int32_t* ell_col = nullptr;
    uint8_t* ell_deg = nullptr;
    int32_t* ell_cslot = nullptr;
    uint8_t* ell_cls = nullptr;
    int32_t ell_D = 0;
    // message slots of the streaming workspace: M ell_D with the padded layout, else E
    int64_t eta_slots = 0;
};

// Index arrays the debug checks cover (ids in the report of ldpc_debug_report).
enum class DebugArray : int {
    kRowPtr = 1, kColPtr, kColIdx, kColEdge, kColClass, kRowBase, kColBase, kRowDeg, kColDeg,
    kRowSlotPos, kColSlot, kColPos, kRowSlotCls, kEllCol, kEllDeg, kEllCslot, kEllCls
};
// Enqueue the debug checks of a decode on st (debug.cu): rep[0] receives the smallest flat
// index of a NaN FP32 LLR, rep[1] the smallest (array id << 40 | entry) of an index out of
// range; both stay all ones when nothing is found.
int debug_check_launch(const DevGraph& g, int32_t M, int32_t N, int64_t E, const void* llr, int llr_is_i8,
                       int64_t frames, unsigned long long* rep, cudaStream_t st);

// ---------------------------------------------------------------------------------------
// Launch parameters shared by the variants.
// ---------------------------------------------------------------------------------------
struct DecodeArgs {
    int32_t M, N, E;
    int32_t frames;
    int32_t L;            // max iterations
    int32_t early_stop;   // 0/1
    int32_t check_every;  // >= 1
    int32_t paper_slicer; // 0/1
    int32_t llr_is_i8;    // input element type
    const void* llr;      // [frames][N] float or int8
    uint8_t* out_bits;    // [frames][N]
    int32_t* out_iters;   // [frames]
    uint8_t* out_ok;      // nullable
    float* out_soft;      // nullable
    // learned weights (FP32 mode): w_rows > 0 -> magnitudes max(fma(alpha, m, -beta), 0),
    // row min(iteration, w_rows) - 1 of the [w_rows][n_classes] device tables
    int32_t w_rows = 0, n_classes = 0;
    const float* w_alpha = nullptr;
    const float* w_beta = nullptr;
};

// Streaming variant workspace (frame-interleaved, frame stride Fp).
struct StreamWork {
    int32_t Fp = 0;
    void* r = nullptr;         // [N][Fp] float / int8
    void* s = nullptr;         // [N][Fp] float / int16
    void* eta = nullptr;       // [eta_slots][Fp] float / int16
    int32_t* done_iter = nullptr;  // [Fp] by frame: iteration at which it stopped, -1 while running
    uint8_t* state = nullptr;      // [Fp] by position: 1 while the frame there is being decoded
    // frame compaction (early stop): the frame at each position (-1: none), the new position
    // of each running frame, and [0] compaction pending, [1] positions in use, [2] frames kept
    int32_t* pos2frame = nullptr;  // [Fp]
    int32_t* new_pos = nullptr;    // [Fp]
    int32_t* comp = nullptr;       // [4]
    uint8_t* unsat = nullptr;      // [(L+2)][Fp]
    int32_t* n_done = nullptr;     // [1]
    // decisions of the last bit pass, one byte per lane of 4 or 8 frames: [N][Fp / 4] bytes
    // (nullable: the final syndrome and the output bits are then taken from s)
    uint8_t* hd = nullptr;
    // staged check pass (padded row layout only): warps per CTA and shared-memory stages
    // per warp, 0 stages = the register kernel; err: device error word (kernels set it,
    // the host reads and clears it); wait_limit: tries of each bounded wait
    int32_t* err = nullptr;
    int32_t stage_warps = 0, stages = 0;
    int32_t stage_vw = 0;  // frames per lane of the staged kernel (0: the run's vector width)
    uint32_t wait_limit = 1u << 16;
    int32_t num_sms = 0;
    // FP32 codes on the padded row layout: keep each row's messages compressed (min0,
    // min1, location and signs; cmsg.cuh) when the staged check pass runs (1), or keep one
    // message per edge slot (0); used_compressed (host, nullable) receives the choice made
    int32_t msg_compressed = 1;
    int32_t* used_compressed = nullptr;
};
// Default staging of the streaming check pass (the shape chosen on GB300).
constexpr int32_t kStageWarpsDefault = 12, kStagesDefault = 2;

// Shared memory of the staged check pass: per warp, `stages` stages of chunks of 32 vw
// elements of the mode's message type (2 D chunks with per-edge messages: the gathered s
// and the old messages; D + 3 with compressed ones: s and the row's three state arrays),
// per stage a 4-byte word per lane and D weight classes and an 8-byte mbarrier; with
// learned weights, two 256-entry tables for the CTA.
inline size_t staged_smem_bytes(int mode, int vw, int D, bool cmp, int warps, int stages, bool weights) {
    const size_t chunk = (size_t)32 * vw * (mode == kModeFP32 ? 4 : 2);
    const size_t stage = (size_t)(cmp ? D + 3 : 2 * D) * chunk;
    const size_t meta = (size_t)32 * 4 + (size_t)D * 4;
    return (size_t)warps * stages * (stage + meta + 8) + (weights ? (size_t)2 * 256 * 4 : 0);
}

// Launchers; return the number of kernels enqueued, or a negative status.
// vw: frames per lane (0: a 16-byte vector, 4 fp32 / 8 int16; else 1, 2, 4 or 8 with the
// frame stride w.Fp a multiple of 32 vw)
int stream_decode(int mode, const DevGraph& dg, const DecodeArgs& a, const StreamWork& w,
                  cudaStream_t st, int vw = 0);
// The messages eta of the first `frames` frames held in w (a decode without early stop or
// frame groups: positions are frames) -> out, device float [frames][E] in CSR edge order,
// in LLR units. Returns the kernels enqueued (1) or a negative status.
// cmp: w holds compressed messages (cmsg.cuh), rebuilt with the weights w_alpha / w_beta
// (device, [n_classes]) of the decode's last iteration when the decode was weighted.
int stream_read_messages(int mode, const DevGraph& g, int32_t M, int64_t E, const StreamWork& w,
                         int32_t frames, float* out, cudaStream_t st, int cmp = 0,
                         const float* w_alpha = nullptr, const float* w_beta = nullptr);
// slots: the graph's eta_slots (message slots per frame).
size_t stream_bytes(int mode, int32_t N, int64_t slots, int32_t Fp, int32_t L);
// The workspace of stream_bytes(mode, N, slots, Fp, L) bytes at mem (Fp a multiple of 256).
StreamWork stream_carve(int mode, void* mem, int32_t N, int64_t slots, int32_t Fp, int32_t L);

// Dense variant (the paper's m x n map-reduce form, a baseline): workspace bytes and launcher.
size_t dense_bytes(int32_t M, int32_t N, int32_t frames);
int dense_decode(const DevGraph& g, const DecodeArgs& a, void* work, cudaStream_t st);

struct ResidentPlan {
    int ok = 0;           // the code fits
    int FT = 0;           // frames per tile (interleaved in shared memory)
    int idx_smem = 0;     // index arrays copied to shared memory
    int threads = 0;      // CTA size
    int ctas_per_sm = 0;
    size_t smem = 0;      // dynamic shared memory per CTA
};
// Requested plan parameters; 0 = chosen automatically.
struct ResidentTuning {
    int FT = 0, threads = 0;
    int idx = 0;  // index arrays: 0 automatic, 1 shared memory, 2 global memory
};
ResidentPlan resident_plan(int mode, const DevGraph& dg, int32_t N, int device,
                           const ResidentTuning& tune = ResidentTuning(), int w_entries = 0);
int resident_decode(int mode, const DevGraph& dg, const ResidentPlan& p, const DecodeArgs& a,
                    int32_t* tile_counter, int num_sms, cudaStream_t st);

// Cluster variant: C CTAs (a thread-block cluster) per tile of FT frames.
struct ClusterPlan {
    int ok = 0;
    int C = 0, FT = 0, threads = 0;
    int clusters = 0;     // clusters resident at once on the device
    size_t smem = 0;      // dynamic shared memory per CTA
};
// The plan for cluster size C (a layout built for C) and frames per tile FT (0: the most
// that fit); threads 0 = 1024.
ClusterPlan cluster_plan(int mode, const DevCluster& dc, int FT, int threads, int w_entries);
int cluster_decode(int mode, const DevCluster& dc, const ClusterPlan& p, const DecodeArgs& a,
                   int32_t* tile_counter, cudaStream_t st);

// Read access to a handle's graph and settings for entry points outside api.cu.
struct HandleView {
    int device, mode, flags;
    int32_t M, N;
    int64_t E;
    const DevGraph* dg;
    cudaStream_t stream;
    int32_t* last_launches;
    int32_t w_rows;          // learned weights in force (FP32 mode), 0 if none
    const float* w_alpha;    // device [w_rows][n_classes], beta follows
    int32_t num_sms = 0;
    int32_t* err = nullptr;  // device error word of the handle
    int32_t stage_warps = 0, stages = 0;  // staged streaming check pass (stages 0 = off)
    int32_t stage_vw = 0;
    uint32_t wait_limit = 0;
    int32_t msg_compressed = 1;  // ldpc_set_stream_messages
};
int handle_view(::ldpc_t* h, HandleView* v);

// Maps the static scratch array of ldpc_decode_noalloc on `device` (the current device)
// and caches its address; handle creation calls it. LDPC_OK or a negative status.
int noalloc_setup(int device);

}  // namespace ldpc_impl
