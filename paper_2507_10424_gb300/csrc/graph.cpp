// H ingestion: dense, bit-packed or CSR input -> the check sets N_i (CSR) and bit sets
// M_j (CSC) of Section II-B, plus the sliced layout of the resident kernel.
#include <algorithm>
#include <numeric>

#include "../../include/ldpc.h"
#include "ldpc_internal.h"

namespace ldpc_impl {

// Finish a graph whose row_ptr/col_idx hold sorted, duplicate-free rows.
static int finish_graph(HostGraph& g) {
    const int32_t M = g.M, N = g.N;
    g.E = g.row_ptr[M];
    g.max_dc = 0;
    for (int32_t i = 0; i < M; i++) {
        int32_t d = g.row_ptr[i + 1] - g.row_ptr[i];
        if (d == 1) return LDPC_ERR_INVALID_H;  // minimum over an empty set
        g.max_dc = std::max(g.max_dc, d);
    }
    g.col_ptr.assign(N + 1, 0);
    for (int64_t e = 0; e < g.E; e++) g.col_ptr[g.col_idx[e] + 1]++;
    for (int32_t j = 0; j < N; j++) g.col_ptr[j + 1] += g.col_ptr[j];
    g.col_edge.resize(g.E);
    std::vector<int32_t> fill(g.col_ptr.begin(), g.col_ptr.end() - 1);
    for (int32_t i = 0; i < M; i++)  // rows in ascending order -> ascending rows per column
        for (int32_t e = g.row_ptr[i]; e < g.row_ptr[i + 1]; e++) g.col_edge[fill[g.col_idx[e]]++] = e;
    g.max_dv = 0;
    for (int32_t j = 0; j < N; j++) g.max_dv = std::max(g.max_dv, g.col_ptr[j + 1] - g.col_ptr[j]);
    return LDPC_OK;
}

int graph_from_dense(int32_t M, int32_t N, const uint8_t* H, HostGraph& g) {
    if (M <= 0 || N <= 0) return LDPC_ERR_INVALID_ARG;
    if (!H) return LDPC_ERR_BAD_POINTER;
    g.M = M;
    g.N = N;
    g.row_ptr.assign(M + 1, 0);
    int64_t E = 0;
    for (int32_t i = 0; i < M; i++) {
        const uint8_t* row = H + (int64_t)i * N;
        for (int32_t j = 0; j < N; j++) {
            if (row[j] > 1) return LDPC_ERR_INVALID_H;
            E += row[j];
        }
        if (E >= (int64_t)INT32_MAX) return LDPC_ERR_INVALID_H;
        g.row_ptr[i + 1] = (int32_t)E;
    }
    g.col_idx.resize(E);
    int64_t e = 0;
    for (int32_t i = 0; i < M; i++) {
        const uint8_t* row = H + (int64_t)i * N;
        for (int32_t j = 0; j < N; j++)
            if (row[j]) g.col_idx[e++] = j;
    }
    return finish_graph(g);
}

int graph_from_packed(int32_t M, int32_t N, const uint32_t* rows, HostGraph& g) {
    if (M <= 0 || N <= 0) return LDPC_ERR_INVALID_ARG;
    if (!rows) return LDPC_ERR_BAD_POINTER;
    const int64_t W = (N + 31) / 32;
    g.M = M;
    g.N = N;
    g.row_ptr.assign(M + 1, 0);
    g.col_idx.clear();
    for (int32_t i = 0; i < M; i++) {
        const uint32_t* row = rows + (int64_t)i * W;
        if (N % 32 && (row[W - 1] >> (N % 32)) != 0) return LDPC_ERR_INVALID_H;  // bits past N
        for (int64_t w = 0; w < W; w++) {
            uint32_t x = row[w];
            while (x) {
                int b = __builtin_ctz(x);
                g.col_idx.push_back((int32_t)(w * 32 + b));
                x &= x - 1;
            }
        }
        if ((int64_t)g.col_idx.size() >= (int64_t)INT32_MAX) return LDPC_ERR_INVALID_H;
        g.row_ptr[i + 1] = (int32_t)g.col_idx.size();
    }
    return finish_graph(g);
}

int graph_from_csr(int32_t M, int32_t N, const int64_t* row_ptr, const int32_t* col_idx,
                   HostGraph& g) {
    if (M <= 0 || N <= 0) return LDPC_ERR_INVALID_ARG;
    if (!row_ptr || (!col_idx && row_ptr[M] > 0)) return LDPC_ERR_BAD_POINTER;
    if (row_ptr[0] != 0) return LDPC_ERR_INVALID_H;
    for (int32_t i = 0; i < M; i++)
        if (row_ptr[i + 1] < row_ptr[i]) return LDPC_ERR_INVALID_H;
    if (row_ptr[M] >= (int64_t)INT32_MAX) return LDPC_ERR_INVALID_H;
    g.M = M;
    g.N = N;
    g.row_ptr.assign(M + 1, 0);
    g.col_idx.assign(col_idx, col_idx + row_ptr[M]);
    for (int32_t i = 0; i < M; i++) {
        g.row_ptr[i + 1] = (int32_t)row_ptr[i + 1];
        auto b = g.col_idx.begin() + row_ptr[i], en = g.col_idx.begin() + row_ptr[i + 1];
        std::sort(b, en);
        for (auto it = b; it != en; ++it) {
            if (*it < 0 || *it >= N) return LDPC_ERR_INVALID_H;
            if (it != b && *it == *(it - 1)) return LDPC_ERR_INVALID_H;
        }
    }
    return finish_graph(g);
}

void build_sliced(const HostGraph& g, SlicedGraph& sg) {
    const int32_t M = g.M;
    std::vector<int32_t> order(M);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (g.row_ptr[a + 1] - g.row_ptr[a]) > (g.row_ptr[b + 1] - g.row_ptr[b]);
    });
    sg.n_slices = (M + 31) / 32;
    sg.slice_base.assign(sg.n_slices + 1, 0);
    sg.row_deg.assign((size_t)sg.n_slices * 32, 0);
    for (int32_t s = 0; s < sg.n_slices; s++) {
        int32_t w = 0;
        for (int32_t l = 0; l < 32 && s * 32 + l < M; l++) {
            int32_t i = order[s * 32 + l];
            int32_t d = g.row_ptr[i + 1] - g.row_ptr[i];
            sg.row_deg[s * 32 + l] = (uint8_t)d;
            w = std::max(w, d);
        }
        sg.slice_base[s + 1] = sg.slice_base[s] + 32 * w;
    }
    sg.E_pad = sg.slice_base[sg.n_slices];
    sg.slot_col.assign(sg.E_pad, 0);
    std::vector<int32_t> slot_of_edge(g.E);
    for (int32_t s = 0; s < sg.n_slices; s++)
        for (int32_t l = 0; l < 32 && s * 32 + l < M; l++) {
            int32_t i = order[s * 32 + l];
            for (int32_t k = 0; k < g.row_ptr[i + 1] - g.row_ptr[i]; k++) {
                int32_t slot = sg.slice_base[s] + 32 * k + l;
                int32_t e = g.row_ptr[i] + k;
                sg.slot_col[slot] = (uint16_t)g.col_idx[e];
                slot_of_edge[e] = slot;
            }
        }
    sg.col_ptr = g.col_ptr;
    if (sg.E_pad < 65536) {
        sg.col_slot16.resize(g.E);
        for (int64_t t = 0; t < g.E; t++) sg.col_slot16[t] = (uint16_t)slot_of_edge[g.col_edge[t]];
    } else {
        sg.col_slot32.resize(g.E);
        for (int64_t t = 0; t < g.E; t++) sg.col_slot32[t] = slot_of_edge[g.col_edge[t]];
    }
}

}  // namespace ldpc_impl
