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
    assign_classes(g);
    return LDPC_OK;
}

void assign_classes(HostGraph& g) {
    g.class_degree.clear();
    for (int32_t j = 0; j < g.N; j++) g.class_degree.push_back(g.col_ptr[j + 1] - g.col_ptr[j]);
    std::sort(g.class_degree.begin(), g.class_degree.end());
    g.class_degree.erase(std::unique(g.class_degree.begin(), g.class_degree.end()), g.class_degree.end());
    g.col_class.assign(g.N, 0);
    for (int32_t j = 0; j < g.N; j++)
        g.col_class[j] = (uint8_t)(std::lower_bound(g.class_degree.begin(), g.class_degree.end(),
                                                    g.col_ptr[j + 1] - g.col_ptr[j]) -
                                   g.class_degree.begin());
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

// Degree-sorted order of n items (descending degree, stable).
static std::vector<int32_t> sorted_by_degree(const std::vector<int32_t>& ptr) {
    const int32_t n = (int32_t)ptr.size() - 1;
    std::vector<int32_t> order(n);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (ptr[a + 1] - ptr[a]) > (ptr[b + 1] - ptr[b]);
    });
    return order;
}

// Slices of 32 lanes over `order`; returns the total slot count.
static int32_t make_slices(const std::vector<int32_t>& ptr, const std::vector<int32_t>& order,
                           std::vector<int32_t>& base, std::vector<uint8_t>& deg) {
    const int32_t n = (int32_t)order.size(), ns = (n + 31) / 32;
    base.assign(ns + 1, 0);
    deg.assign((size_t)ns * 32, 0);
    for (int32_t s = 0; s < ns; s++) {
        int32_t w = 0;
        for (int32_t l = 0; l < 32 && s * 32 + l < n; l++) {
            const int32_t x = order[s * 32 + l], d = ptr[x + 1] - ptr[x];
            deg[s * 32 + l] = (uint8_t)d;
            w = std::max(w, d);
        }
        base[s + 1] = base[s] + 32 * w;
    }
    return base[ns];
}

bool build_sliced(const HostGraph& g, SlicedGraph& sg) {
    if (g.N > 65535 || g.max_dc > 255 || g.max_dv > 255) return false;
    const std::vector<int32_t> rorder = sorted_by_degree(g.row_ptr);
    const std::vector<int32_t> corder = sorted_by_degree(g.col_ptr);
    sg.n_rslices = (g.M + 31) / 32;
    sg.n_cslices = (g.N + 31) / 32;
    sg.E_pad = make_slices(g.row_ptr, rorder, sg.r_base, sg.r_deg);
    sg.Ec_pad = make_slices(g.col_ptr, corder, sg.c_base, sg.c_deg);
    if (sg.E_pad >= 65536 || sg.Ec_pad >= 65536) return false;
    sg.col_pos.assign(g.N, 0);
    for (int32_t p = 0; p < g.N; p++) sg.col_pos[corder[p]] = (uint16_t)p;
    // row side: slot of every edge, and the sorted column position it reads
    std::vector<int32_t> slot_of_edge(g.E);
    sg.r_slot_pos.assign(sg.E_pad, 0);
    sg.r_slot_cls.assign(sg.E_pad, 0);
    for (int32_t s = 0; s < sg.n_rslices; s++)
        for (int32_t l = 0; l < 32 && s * 32 + l < g.M; l++) {
            const int32_t i = rorder[s * 32 + l];
            for (int32_t k = 0; k < g.row_ptr[i + 1] - g.row_ptr[i]; k++) {
                const int32_t slot = sg.r_base[s] + 32 * k + l, e = g.row_ptr[i] + k;
                sg.r_slot_pos[slot] = sg.col_pos[g.col_idx[e]];
                sg.r_slot_cls[slot] = g.col_class.empty() ? 0 : g.col_class[g.col_idx[e]];
                slot_of_edge[e] = slot;
            }
        }
    // column side: the row slots of a column's edges in ascending row order
    sg.c_slot.assign(sg.Ec_pad, 0);
    for (int32_t s = 0; s < sg.n_cslices; s++)
        for (int32_t l = 0; l < 32 && s * 32 + l < g.N; l++) {
            const int32_t j = corder[s * 32 + l];
            for (int32_t k = 0; k < g.col_ptr[j + 1] - g.col_ptr[j]; k++)
                sg.c_slot[sg.c_base[s] + 32 * k + l] = (uint16_t)slot_of_edge[g.col_edge[g.col_ptr[j] + k]];
        }
    return true;
}

// Cut items 0 .. n-1 into C contiguous ranges of about equal total degree.
static std::vector<int32_t> cut_by_degree(const std::vector<int32_t>& ptr, int C) {
    const int32_t n = (int32_t)ptr.size() - 1;
    const int64_t E = ptr[n];
    std::vector<int32_t> b(C + 1, n);
    b[0] = 0;
    int32_t x = 0;
    for (int q = 1; q < C; q++) {
        const int64_t target = E * q / C;
        while (x < n && ptr[x] < target) x++;
        b[q] = x;
    }
    return b;
}

// Items lo .. hi-1 sorted by degree (descending, stable).
static std::vector<int32_t> range_by_degree(const std::vector<int32_t>& ptr, int32_t lo, int32_t hi) {
    std::vector<int32_t> order(hi - lo);
    std::iota(order.begin(), order.end(), lo);
    std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
        return (ptr[a + 1] - ptr[a]) > (ptr[b + 1] - ptr[b]);
    });
    return order;
}

bool build_cluster(const HostGraph& g, int C, ClusterGraph& cg) {
    if (C < 1 || C > 16 || g.max_dc > 255 || g.max_dv > 255) return false;
    cg = ClusterGraph();
    cg.C = C;
    cg.meta.assign((size_t)C * kClMeta, 0);
    cg.pos_of_col.assign(g.N, 0);
    const std::vector<int32_t> J = cut_by_degree(g.col_ptr, C), I = cut_by_degree(g.row_ptr, C);
    std::vector<uint8_t> owner(g.N, 0);
    std::vector<std::vector<int32_t>> corder(C), rorder(C);
    for (int q = 0; q < C; q++) {
        corder[q] = range_by_degree(g.col_ptr, J[q], J[q + 1]);
        rorder[q] = range_by_degree(g.row_ptr, I[q], I[q + 1]);
        if (corder[q].size() > 65535) return false;
        for (size_t p = 0; p < corder[q].size(); p++) {
            cg.pos_of_col[corder[q][p]] = (uint16_t)p;
            owner[corder[q][p]] = (uint8_t)q;
        }
    }
    // row side: every edge's slot in its row owner's layout, and the column it reads
    std::vector<uint32_t> slot_ref(g.E);
    for (int q = 0; q < C; q++) {
        int32_t* m = &cg.meta[(size_t)q * kClMeta];
        std::vector<int32_t> base;
        std::vector<uint8_t> deg;
        const int32_t Ep = make_slices(g.row_ptr, rorder[q], base, deg);
        if (Ep > 65536) return false;
        m[kClRTasks] = (int32_t)deg.size();
        m[kClRBase] = (int32_t)cg.r_base.size();
        m[kClRDeg] = (int32_t)cg.r_deg.size();
        m[kClRRef] = (int32_t)cg.r_ref.size();
        const size_t off = cg.r_ref.size();
        cg.r_base.insert(cg.r_base.end(), base.begin(), base.end());
        cg.r_deg.insert(cg.r_deg.end(), deg.begin(), deg.end());
        cg.r_ref.resize(off + Ep, 0);
        cg.r_cls.resize(off + Ep, 0);
        for (size_t t = 0; t < rorder[q].size(); t++) {
            const int32_t i = rorder[q][t], sl = (int32_t)(t / 32), l = (int32_t)(t % 32);
            for (int32_t k = 0; k < g.row_ptr[i + 1] - g.row_ptr[i]; k++) {
                const int32_t slot = base[sl] + 32 * k + l, e = g.row_ptr[i] + k, c = g.col_idx[e];
                cg.r_ref[off + slot] = ((uint32_t)owner[c] << 16) | cg.pos_of_col[c];
                cg.r_cls[off + slot] = g.col_class.empty() ? 0 : g.col_class[c];
                slot_ref[e] = ((uint32_t)q << 16) | (uint32_t)slot;
            }
        }
        cg.E_cap = std::max(cg.E_cap, Ep);
    }
    // column side: the slots of a column's edges in ascending row order
    for (int q = 0; q < C; q++) {
        int32_t* m = &cg.meta[(size_t)q * kClMeta];
        std::vector<int32_t> base;
        std::vector<uint8_t> deg;
        const int32_t Ecp = make_slices(g.col_ptr, corder[q], base, deg);
        m[kClJ0] = J[q];
        m[kClJ1] = J[q + 1];
        m[kClCTasks] = (int32_t)deg.size();
        m[kClCBase] = (int32_t)cg.c_base.size();
        m[kClCDeg] = (int32_t)cg.c_deg.size();
        m[kClCRef] = (int32_t)cg.c_ref.size();
        const size_t off = cg.c_ref.size();
        cg.c_base.insert(cg.c_base.end(), base.begin(), base.end());
        cg.c_deg.insert(cg.c_deg.end(), deg.begin(), deg.end());
        cg.c_ref.resize(off + Ecp, 0);
        for (size_t t = 0; t < corder[q].size(); t++) {
            const int32_t j = corder[q][t], sl = (int32_t)(t / 32), l = (int32_t)(t % 32);
            for (int32_t k = 0; k < g.col_ptr[j + 1] - g.col_ptr[j]; k++)
                cg.c_ref[off + base[sl] + 32 * k + l] = slot_ref[g.col_edge[g.col_ptr[j] + k]];
        }
        cg.P_cap = std::max(cg.P_cap, (int32_t)deg.size());
    }
    return true;
}

bool build_ell(const HostGraph& g, EllGraph& eg) {
    if (g.max_dc > 16) return false;
    const int32_t D = g.max_dc <= 8 ? 8 : 16;
    eg.D = D;
    eg.ell_col.assign((size_t)g.M * D, 0);
    eg.ell_deg.assign(g.M, 0);
    std::vector<int64_t> slot_of_edge(g.E);
    for (int32_t i = 0; i < g.M; i++) {
        const int32_t e0 = g.row_ptr[i], d = g.row_ptr[i + 1] - e0;
        eg.ell_deg[i] = (uint8_t)d;
        for (int32_t t = 0; t < D; t++)  // padding: the row's first column (column 0 if empty)
            eg.ell_col[(size_t)i * D + t] = d == 0 ? 0 : g.col_idx[e0 + (t < d ? t : 0)];
        for (int32_t t = 0; t < d; t++) slot_of_edge[e0 + t] = (int64_t)i * D + t;
    }
    if ((int64_t)g.M * D >= (int64_t)INT32_MAX) return false;
    eg.ell_cslot.resize(g.E);
    for (int64_t q = 0; q < g.E; q++) eg.ell_cslot[q] = (int32_t)slot_of_edge[g.col_edge[q]];
    eg.ell_cls.assign((size_t)g.M * D, 0);
    for (int32_t i = 0; i < g.M; i++)
        for (int32_t t = 0; t < g.row_ptr[i + 1] - g.row_ptr[i]; t++)
            eg.ell_cls[(size_t)i * D + t] = g.col_class[g.col_idx[g.row_ptr[i] + t]];
    return true;
}

}  // namespace ldpc_impl
