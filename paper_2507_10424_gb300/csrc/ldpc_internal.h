// Internal declarations of the GB300 Min-Sum decoder library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

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
};

// Each returns LDPC_OK or an LDPC_ERR_* status.
int graph_from_dense(int32_t M, int32_t N, const uint8_t* H, HostGraph& g);
int graph_from_packed(int32_t M, int32_t N, const uint32_t* rows, HostGraph& g);
int graph_from_csr(int32_t M, int32_t N, const int64_t* row_ptr, const int32_t* col_idx,
                   HostGraph& g);

// ---------------------------------------------------------------------------------------
// Sliced layout used by the resident kernel: rows sorted by degree (descending, stable),
// grouped into slices of 32; slot (row lane l of slice s, k-th edge) sits at
// slice_base[s] + 32 k + l, so that the 32 lanes of a warp touch 32 consecutive words.
// ---------------------------------------------------------------------------------------
struct SlicedGraph {
    int32_t n_slices = 0;
    int32_t E_pad = 0;                // total slots incl. padding
    std::vector<int32_t> slice_base;  // n_slices + 1
    std::vector<uint8_t> row_deg;     // 32 * n_slices (0 for missing rows)
    std::vector<uint16_t> slot_col;   // E_pad: column of each slot (0 for padding)
    std::vector<int32_t> col_ptr;     // N+1
    std::vector<uint16_t> col_slot16; // E: slot ids of column j's edges, ascending row (E_pad < 65536)
    std::vector<int32_t> col_slot32;  // same, when E_pad >= 65536
};
void build_sliced(const HostGraph& g, SlicedGraph& sg);

// Device copies of the graph.
struct DevGraph {
    // CSR/CSC (streaming kernels)
    int32_t* row_ptr = nullptr;
    int32_t* col_idx = nullptr;
    int32_t* col_ptr = nullptr;
    int32_t* col_edge = nullptr;
    // bit-packed rows, uint32 [M][ceil(N/32)]
    uint32_t* packed = nullptr;
    // sliced layout (resident kernel)
    int32_t* s_slice_base = nullptr;
    uint8_t* s_row_deg = nullptr;
    uint16_t* s_slot_col = nullptr;
    int32_t* s_col_ptr = nullptr;
    uint16_t* s_col_slot16 = nullptr;
    int32_t* s_col_slot32 = nullptr;
    int32_t n_slices = 0, E_pad = 0;
};

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
};

// Streaming variant workspace (frame-interleaved, frame stride Fp).
struct StreamWork {
    int32_t Fp = 0;
    void* r = nullptr;         // [N][Fp] float / int8
    void* s = nullptr;         // [N][Fp] float / int16
    void* eta = nullptr;       // [E][Fp] float / int16
    int32_t* done_iter = nullptr;  // [Fp]: iteration at which the frame stopped, -1 while running
    uint8_t* state = nullptr;      // [Fp]: 1 while the frame is being decoded
    uint8_t* unsat = nullptr;      // [(L+2)][Fp]
    int32_t* n_done = nullptr;     // [1]
};

// Launchers; return the number of kernels enqueued, or a negative status.
int stream_decode(int mode, const DevGraph& dg, const DecodeArgs& a, const StreamWork& w,
                  cudaStream_t st);
size_t stream_bytes(int mode, int32_t N, int64_t E, int32_t Fp, int32_t L);

struct ResidentPlan {
    int ok = 0;           // the code fits
    int FT = 0;           // frames per tile
    int threads = 0;      // CTA size
    int ctas_per_sm = 0;
    size_t smem = 0;      // dynamic shared memory per CTA
};
ResidentPlan resident_plan(int mode, const DevGraph& dg, int32_t M, int32_t N, int device);
int resident_decode(int mode, const DevGraph& dg, const ResidentPlan& p, const DecodeArgs& a,
                    int32_t* tile_counter, int num_sms, cudaStream_t st);

}  // namespace ldpc_impl
