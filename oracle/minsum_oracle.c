/*
 * Oracle for flooding Min-Sum decoding of binary LDPC codes (arXiv 2507.10424).
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow CPU restatement of the paper's
 * method, used by the test suite to check the CUDA path and by the benchmark's
 * CPU-baseline leg. It shares no code, header, table or helper with the CUDA path
 * and must never be called from the product path.
 *
 * Everything here follows the paper directly:
 *   - check sets N_i (row support of H) and M_j (column support), Section II-B;
 *   - check-node update, eq. (eta_update): for each edge (i,j),
 *       eta_ij = min_{k in N_i, k != j} |lambda_k - eta_ik^prev|
 *                * prod_{k in N_i, k != j} sign(lambda_k - eta_ik^prev),
 *     with eta^prev = 0 at the first iteration and sign(0) = +1 (Section III);
 *   - the same update through Observations 1 (two smallest magnitudes and the
 *     location of the smallest) and 2 (extrinsic sign = total sign x own sign);
 *   - variable-node update, eq. (lambda_j): s_j = r_j + sum_{i in M_j} eta_ij;
 *   - the hard decision (slice) and the syndrome test H b = 0 over GF(2), eq. (1)-(2);
 *   - Algorithm 1 (graph form) and Algorithm 2 (dense masked map-reduce form).
 *
 * Readings where the paper is silent or inconsistent:
 *   R1 bit decision: b_j = [s_j < 0] (LLR = log P(0)/P(1)); the paper's printed
 *      slicer [s_j > 0] is available as an option (ORC_PAPER_SLICER);
 *   R2 sign(0) = +1, so sigma = [v < 0] and -0.0 counts as positive;
 *   R3 the location of the smallest magnitude is the first (lowest column) position;
 *   R4 the syndrome is tested once before the first iteration (iterations = 0 when the
 *      input already is a codeword), then after every check_every-th iteration;
 *   R5 the returned iteration count is the number of completed iterations;
 *   R6 the column sum starts from r_j and adds eta in ascending row order (left fold);
 *   R7 fixed point: q = clamp(round_half_even(4 llr), -127, 127); lambda, eta and s are
 *      held in [-32767, 32767] with int32 intermediates, saturating lambda and s;
 *   R8 rows of weight 1 are rejected (the minimum over an empty set is undefined).
 *
 * Floating point: the FP32 decoder computes in binary32 with round-to-nearest and no
 * contraction (compile with -ffp-contract=off); a binary64 decoder is provided too.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG (-1)
#define ORC_ERR_H (-2)
#define ORC_ERR_NOMEM (-4)

#define ORC_PAPER_SLICER 1 /* flag: b_j = [s_j > 0] as printed in eq. (slice) */

#define ORC_CHECK_TWOMIN 0 /* Observations 1 and 2 */
#define ORC_CHECK_BRUTE 1  /* eq. (eta_update) taken literally, O(d_c^2) per row */

#define ORC_SAT 32767

typedef struct {
    int32_t M, N;
    int64_t E;
    int64_t *row_ptr; /* M+1: edges of row i are row_ptr[i] .. row_ptr[i+1]-1 */
    int32_t *col_of;  /* E: column of each edge; ascending within a row */
    int64_t *col_ptr; /* N+1 */
    int64_t *edge_of; /* E: edge ids of column j in ascending row order */
} orc_graph;

/* ------------------------------------------------------------------------- */
/* Graph construction: N_i and M_j from H (Section II-B).                     */
/* ------------------------------------------------------------------------- */

void orc_graph_free(orc_graph *g) {
    if (!g) return;
    free(g->row_ptr);
    free(g->col_of);
    free(g->col_ptr);
    free(g->edge_of);
    free(g);
}

static int cmp_i64(const void *a, const void *b) {
    int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
    return (x > y) - (x < y);
}

/* Build from an edge list (row, col); duplicates, out-of-range entries and rows of
 * weight 1 are rejected. */
int orc_graph_create(int32_t M, int32_t N, int64_t E, const int32_t *rows,
                     const int32_t *cols, orc_graph **out) {
    *out = NULL;
    if (M <= 0 || N <= 0 || E < 0) return ORC_ERR_ARG;
    int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    if (!key) return ORC_ERR_NOMEM;
    for (int64_t e = 0; e < E; e++) {
        if (rows[e] < 0 || rows[e] >= M || cols[e] < 0 || cols[e] >= N) {
            free(key);
            return ORC_ERR_H;
        }
        key[e] = (int64_t)rows[e] * N + cols[e];
    }
    qsort(key, (size_t)E, sizeof(int64_t), cmp_i64);
    for (int64_t e = 1; e < E; e++)
        if (key[e] == key[e - 1]) {
            free(key);
            return ORC_ERR_H;
        }
    orc_graph *g = (orc_graph *)calloc(1, sizeof(orc_graph));
    g->M = M;
    g->N = N;
    g->E = E;
    g->row_ptr = (int64_t *)calloc((size_t)M + 1, sizeof(int64_t));
    g->col_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    g->col_ptr = (int64_t *)calloc((size_t)N + 1, sizeof(int64_t));
    g->edge_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E > 0 ? E : 1));
    if (!g->row_ptr || !g->col_of || !g->col_ptr || !g->edge_of) {
        free(key);
        orc_graph_free(g);
        return ORC_ERR_NOMEM;
    }
    /* key is sorted by (row, col): edges enumerate N_i in ascending column order */
    for (int64_t e = 0; e < E; e++) {
        int32_t i = (int32_t)(key[e] / N), j = (int32_t)(key[e] % N);
        g->row_ptr[i + 1]++;
        g->col_of[e] = j;
        g->col_ptr[j + 1]++;
    }
    for (int32_t i = 0; i < M; i++) g->row_ptr[i + 1] += g->row_ptr[i];
    for (int32_t j = 0; j < N; j++) g->col_ptr[j + 1] += g->col_ptr[j];
    /* M_j: scanning edges in row order appends rows to each column in ascending order */
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    memcpy(fill, g->col_ptr, sizeof(int64_t) * (size_t)N);
    for (int64_t e = 0; e < E; e++) g->edge_of[fill[g->col_of[e]]++] = e;
    free(fill);
    free(key);
    for (int32_t i = 0; i < M; i++)
        if (g->row_ptr[i + 1] - g->row_ptr[i] == 1) {
            orc_graph_free(g);
            return ORC_ERR_H;
        }
    *out = g;
    return ORC_OK;
}

/* Build from a dense row-major M x N matrix whose entries must be 0 or 1. */
int orc_graph_from_dense(int32_t M, int32_t N, const uint8_t *H, orc_graph **out) {
    *out = NULL;
    if (M <= 0 || N <= 0) return ORC_ERR_ARG;
    int64_t E = 0;
    for (int64_t t = 0; t < (int64_t)M * N; t++) {
        if (H[t] > 1) return ORC_ERR_H;
        E += H[t];
    }
    int32_t *rows = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E > 0 ? E : 1));
    int64_t e = 0;
    for (int32_t i = 0; i < M; i++)
        for (int32_t j = 0; j < N; j++)
            if (H[(int64_t)i * N + j]) {
                rows[e] = i;
                cols[e] = j;
                e++;
            }
    int rc = orc_graph_create(M, N, E, rows, cols, out);
    free(rows);
    free(cols);
    return rc;
}

int64_t orc_graph_edges(const orc_graph *g) { return g->E; }

/* ------------------------------------------------------------------------- */
/* Hard decision and syndrome, eq. (slice) and eq. (1)-(2).                   */
/* ------------------------------------------------------------------------- */

static inline uint8_t slice_f32(float s, int flags) {
    return (flags & ORC_PAPER_SLICER) ? (uint8_t)(s > 0.0f) : (uint8_t)(s < 0.0f);
}
static inline uint8_t slice_f64(double s, int flags) {
    return (flags & ORC_PAPER_SLICER) ? (uint8_t)(s > 0.0) : (uint8_t)(s < 0.0);
}
static inline uint8_t slice_i32(int32_t s, int flags) {
    return (flags & ORC_PAPER_SLICER) ? (uint8_t)(s > 0) : (uint8_t)(s < 0);
}

/* z_i = XOR of b_j over j in N_i; returns the number of unsatisfied checks. */
int64_t orc_syndrome(const orc_graph *g, const uint8_t *b, uint8_t *z /* nullable */) {
    int64_t unsat = 0;
    for (int32_t i = 0; i < g->M; i++) {
        uint8_t x = 0;
        for (int64_t e = g->row_ptr[i]; e < g->row_ptr[i + 1]; e++) x ^= (uint8_t)(b[g->col_of[e]] & 1);
        if (z) z[i] = x;
        unsat += x;
    }
    return unsat;
}

/* ------------------------------------------------------------------------- */
/* Check-node update for one row, in the three arithmetics.                   */
/* lam[k] are the row's lambda values (k-th edge of N_i); eta[k] receives the */
/* new message to the k-th bit.                                               */
/* ------------------------------------------------------------------------- */

static void check_row_brute_f32(int64_t d, const float *lam, float *eta) {
    /* eq. (eta_update): minimum and sign product over all other neighbours */
    for (int64_t j = 0; j < d; j++) {
        float m = INFINITY;
        int neg = 0;
        for (int64_t k = 0; k < d; k++) {
            if (k == j) continue;
            float a = fabsf(lam[k]);
            if (a < m) m = a;
            if (lam[k] < 0.0f) neg ^= 1; /* sign(0) = +1 */
        }
        eta[j] = neg ? -m : m;
    }
}

static void check_row_twomin_f32(int64_t d, const float *lam, float *eta) {
    /* Observation 1: min0, its first location, and min1 (smallest elsewhere) */
    float min0 = INFINITY, min1 = INFINITY;
    int64_t loc = -1;
    int total_neg = 0;
    for (int64_t k = 0; k < d; k++) {
        float a = fabsf(lam[k]);
        if (a < min0) {
            min1 = min0;
            min0 = a;
            loc = k;
        } else if (a < min1) {
            min1 = a;
        }
        if (lam[k] < 0.0f) total_neg ^= 1; /* Observation 2: total sign product */
    }
    for (int64_t j = 0; j < d; j++) {
        int neg = total_neg ^ (lam[j] < 0.0f); /* extrinsic sign = total x own */
        float m = (j == loc) ? min1 : min0;
        eta[j] = neg ? -m : m;
    }
}

static void check_row_brute_f64(int64_t d, const double *lam, double *eta) {
    for (int64_t j = 0; j < d; j++) {
        double m = INFINITY;
        int neg = 0;
        for (int64_t k = 0; k < d; k++) {
            if (k == j) continue;
            double a = fabs(lam[k]);
            if (a < m) m = a;
            if (lam[k] < 0.0) neg ^= 1;
        }
        eta[j] = neg ? -m : m;
    }
}

static void check_row_twomin_f64(int64_t d, const double *lam, double *eta) {
    double min0 = INFINITY, min1 = INFINITY;
    int64_t loc = -1;
    int total_neg = 0;
    for (int64_t k = 0; k < d; k++) {
        double a = fabs(lam[k]);
        if (a < min0) {
            min1 = min0;
            min0 = a;
            loc = k;
        } else if (a < min1) {
            min1 = a;
        }
        if (lam[k] < 0.0) total_neg ^= 1;
    }
    for (int64_t j = 0; j < d; j++) {
        int neg = total_neg ^ (lam[j] < 0.0);
        double m = (j == loc) ? min1 : min0;
        eta[j] = neg ? -m : m;
    }
}

static void check_row_brute_i32(int64_t d, const int32_t *lam, int32_t *eta) {
    for (int64_t j = 0; j < d; j++) {
        int32_t m = INT32_MAX;
        int neg = 0;
        for (int64_t k = 0; k < d; k++) {
            if (k == j) continue;
            int32_t a = lam[k] < 0 ? -lam[k] : lam[k];
            if (a < m) m = a;
            if (lam[k] < 0) neg ^= 1;
        }
        eta[j] = neg ? -m : m;
    }
}

static void check_row_twomin_i32(int64_t d, const int32_t *lam, int32_t *eta) {
    int32_t min0 = INT32_MAX, min1 = INT32_MAX;
    int64_t loc = -1;
    int total_neg = 0;
    for (int64_t k = 0; k < d; k++) {
        int32_t a = lam[k] < 0 ? -lam[k] : lam[k];
        if (a < min0) {
            min1 = min0;
            min0 = a;
            loc = k;
        } else if (a < min1) {
            min1 = a;
        }
        if (lam[k] < 0) total_neg ^= 1;
    }
    for (int64_t j = 0; j < d; j++) {
        int neg = total_neg ^ (lam[j] < 0);
        int32_t m = (j == loc) ? min1 : min0;
        eta[j] = neg ? -m : m;
    }
}

/* Exposed for unit tests of the check update alone (one row). */
void orc_check_row_f32(int variant, int64_t d, const float *lam, float *eta) {
    if (variant == ORC_CHECK_BRUTE) check_row_brute_f32(d, lam, eta);
    else check_row_twomin_f32(d, lam, eta);
}
void orc_check_row_f64(int variant, int64_t d, const double *lam, double *eta) {
    if (variant == ORC_CHECK_BRUTE) check_row_brute_f64(d, lam, eta);
    else check_row_twomin_f64(d, lam, eta);
}
void orc_check_row_i32(int variant, int64_t d, const int32_t *lam, int32_t *eta) {
    if (variant == ORC_CHECK_BRUTE) check_row_brute_i32(d, lam, eta);
    else check_row_twomin_i32(d, lam, eta);
}

static inline int32_t sat16(int64_t v) {
    return v > ORC_SAT ? ORC_SAT : (v < -ORC_SAT ? -ORC_SAT : (int32_t)v);
}

/* Fixed-point input conversion (reading R7): LLR step 0.25, int8, saturating. */
int8_t orc_quantize_one(float x) {
    float t = 4.0f * x; /* exact scaling by a power of two */
    if (t != t) return 0;
    if (t > 127.0f) t = 127.0f;
    if (t < -127.0f) t = -127.0f;
    return (int8_t)lrintf(t); /* default rounding: to nearest, ties to even */
}
void orc_quantize(const float *x, int64_t n, int8_t *q) {
    for (int64_t t = 0; t < n; t++) q[t] = orc_quantize_one(x[t]);
}

/* ------------------------------------------------------------------------- */
/* One-frame decoders, Algorithm 1 (graph form).                              */
/* Outputs: b (N), *iters, *ok; optional soft (N) and per-iteration traces of */
/* eta (L x E) and s (L x N).                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int32_t L;
    int32_t early_stop;
    int32_t check_every;
    int32_t variant;
    int32_t flags;
} orc_opts;

/* The syndrome is tested after iteration k when early stop is on and k is a multiple
 * of check_every (k = 0 is the test before the first iteration). */
static inline int test_now(const orc_opts *o, int32_t k) {
    return o->early_stop && (k % (o->check_every > 0 ? o->check_every : 1) == 0);
}

typedef struct {
    double *lam, *tmp; /* max row degree */
} scratch_f64;

static int decode_frame_f32(const orc_graph *g, const orc_opts *o, const float *r, uint8_t *b,
                            int32_t *iters, uint8_t *ok, float *soft, float *eta_trace,
                            float *s_trace, float *eta, float *s, float *lam, float *tmp) {
    const int32_t M = g->M, N = g->N;
    const int64_t E = g->E;
    for (int32_t j = 0; j < N; j++) s[j] = r[j];
    for (int64_t e = 0; e < E; e++) eta[e] = 0.0f;
    for (int32_t j = 0; j < N; j++) b[j] = slice_f32(s[j], o->flags);
    int32_t k = 0;
    int done = test_now(o, 0) && orc_syndrome(g, b, NULL) == 0;
    while (!done && k < o->L) {
        /* check nodes: lambda_e = s_j - eta_e^prev, then eq. (eta_update) per row */
        for (int32_t i = 0; i < M; i++) {
            int64_t e0 = g->row_ptr[i], d = g->row_ptr[i + 1] - e0;
            for (int64_t t = 0; t < d; t++) lam[t] = s[g->col_of[e0 + t]] - eta[e0 + t];
            if (o->variant == ORC_CHECK_BRUTE) check_row_brute_f32(d, lam, tmp);
            else check_row_twomin_f32(d, lam, tmp);
            for (int64_t t = 0; t < d; t++) eta[e0 + t] = tmp[t];
        }
        /* bit nodes: eq. (lambda_j), r_j first, then ascending rows */
        for (int32_t j = 0; j < N; j++) {
            float acc = r[j];
            for (int64_t t = g->col_ptr[j]; t < g->col_ptr[j + 1]; t++) acc = acc + eta[g->edge_of[t]];
            s[j] = acc;
        }
        k++;
        if (eta_trace) memcpy(eta_trace + (int64_t)(k - 1) * E, eta, sizeof(float) * (size_t)E);
        if (s_trace) memcpy(s_trace + (int64_t)(k - 1) * N, s, sizeof(float) * (size_t)N);
        for (int32_t j = 0; j < N; j++) b[j] = slice_f32(s[j], o->flags);
        if (test_now(o, k) && orc_syndrome(g, b, NULL) == 0) done = 1;
    }
    *iters = k;
    *ok = (uint8_t)(orc_syndrome(g, b, NULL) == 0);
    if (soft) memcpy(soft, s, sizeof(float) * (size_t)N);
    return ORC_OK;
}

static int decode_frame_f64(const orc_graph *g, const orc_opts *o, const double *r, uint8_t *b,
                            int32_t *iters, uint8_t *ok, double *soft, double *eta, double *s,
                            double *lam, double *tmp) {
    const int32_t M = g->M, N = g->N;
    const int64_t E = g->E;
    for (int32_t j = 0; j < N; j++) s[j] = r[j];
    for (int64_t e = 0; e < E; e++) eta[e] = 0.0;
    for (int32_t j = 0; j < N; j++) b[j] = slice_f64(s[j], o->flags);
    int32_t k = 0;
    int done = test_now(o, 0) && orc_syndrome(g, b, NULL) == 0;
    while (!done && k < o->L) {
        for (int32_t i = 0; i < M; i++) {
            int64_t e0 = g->row_ptr[i], d = g->row_ptr[i + 1] - e0;
            for (int64_t t = 0; t < d; t++) lam[t] = s[g->col_of[e0 + t]] - eta[e0 + t];
            if (o->variant == ORC_CHECK_BRUTE) check_row_brute_f64(d, lam, tmp);
            else check_row_twomin_f64(d, lam, tmp);
            for (int64_t t = 0; t < d; t++) eta[e0 + t] = tmp[t];
        }
        for (int32_t j = 0; j < N; j++) {
            double acc = r[j];
            for (int64_t t = g->col_ptr[j]; t < g->col_ptr[j + 1]; t++) acc = acc + eta[g->edge_of[t]];
            s[j] = acc;
        }
        k++;
        for (int32_t j = 0; j < N; j++) b[j] = slice_f64(s[j], o->flags);
        if (test_now(o, k) && orc_syndrome(g, b, NULL) == 0) done = 1;
    }
    *iters = k;
    *ok = (uint8_t)(orc_syndrome(g, b, NULL) == 0);
    if (soft) memcpy(soft, s, sizeof(double) * (size_t)N);
    return ORC_OK;
}

static int decode_frame_fixed(const orc_graph *g, const orc_opts *o, const int8_t *q, uint8_t *b,
                              int32_t *iters, uint8_t *ok, int16_t *soft, int16_t *eta_trace,
                              int16_t *s_trace, int32_t *eta, int32_t *s, int32_t *lam,
                              int32_t *tmp) {
    const int32_t M = g->M, N = g->N;
    const int64_t E = g->E;
    for (int32_t j = 0; j < N; j++) s[j] = q[j];
    for (int64_t e = 0; e < E; e++) eta[e] = 0;
    for (int32_t j = 0; j < N; j++) b[j] = slice_i32(s[j], o->flags);
    int32_t k = 0;
    int done = test_now(o, 0) && orc_syndrome(g, b, NULL) == 0;
    while (!done && k < o->L) {
        for (int32_t i = 0; i < M; i++) {
            int64_t e0 = g->row_ptr[i], d = g->row_ptr[i + 1] - e0;
            for (int64_t t = 0; t < d; t++)
                lam[t] = sat16((int64_t)s[g->col_of[e0 + t]] - (int64_t)eta[e0 + t]);
            if (o->variant == ORC_CHECK_BRUTE) check_row_brute_i32(d, lam, tmp);
            else check_row_twomin_i32(d, lam, tmp);
            for (int64_t t = 0; t < d; t++) eta[e0 + t] = tmp[t];
        }
        for (int32_t j = 0; j < N; j++) {
            int64_t acc = q[j];
            for (int64_t t = g->col_ptr[j]; t < g->col_ptr[j + 1]; t++) acc += eta[g->edge_of[t]];
            s[j] = sat16(acc);
        }
        k++;
        if (eta_trace)
            for (int64_t e = 0; e < E; e++) eta_trace[(int64_t)(k - 1) * E + e] = (int16_t)eta[e];
        if (s_trace)
            for (int32_t j = 0; j < N; j++) s_trace[(int64_t)(k - 1) * N + j] = (int16_t)s[j];
        for (int32_t j = 0; j < N; j++) b[j] = slice_i32(s[j], o->flags);
        if (test_now(o, k) && orc_syndrome(g, b, NULL) == 0) done = 1;
    }
    *iters = k;
    *ok = (uint8_t)(orc_syndrome(g, b, NULL) == 0);
    if (soft)
        for (int32_t j = 0; j < N; j++) soft[j] = (int16_t)s[j];
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Batch drivers: frames are independent; split them over worker threads.    */
/* ------------------------------------------------------------------------- */

enum { KIND_F32 = 0, KIND_F64 = 1, KIND_FIXED = 2 };

typedef struct {
    const orc_graph *g;
    orc_opts o;
    int kind;
    const void *in; /* float [F][N], double [F][N] or int8 [F][N] */
    int64_t f0, f1;
    uint8_t *bits;
    int32_t *iters;
    uint8_t *ok;
    void *soft; /* nullable: float, double or int16 [F][N] */
    int rc;
} job_t;

static int64_t max_row_degree(const orc_graph *g) {
    int64_t d = 1;
    for (int32_t i = 0; i < g->M; i++)
        if (g->row_ptr[i + 1] - g->row_ptr[i] > d) d = g->row_ptr[i + 1] - g->row_ptr[i];
    return d;
}

static void *run_job(void *arg) {
    job_t *J = (job_t *)arg;
    const orc_graph *g = J->g;
    const int64_t N = g->N, E = g->E > 0 ? g->E : 1, D = max_row_degree(g);
    J->rc = ORC_OK;
    if (J->kind == KIND_F32) {
        float *eta = malloc(sizeof(float) * E), *s = malloc(sizeof(float) * N);
        float *lam = malloc(sizeof(float) * D), *tmp = malloc(sizeof(float) * D);
        if (!eta || !s || !lam || !tmp) J->rc = ORC_ERR_NOMEM;
        for (int64_t f = J->f0; f < J->f1 && J->rc == ORC_OK; f++)
            decode_frame_f32(g, &J->o, (const float *)J->in + f * N, J->bits + f * N, J->iters + f,
                             J->ok + f, J->soft ? (float *)J->soft + f * N : NULL, NULL, NULL, eta,
                             s, lam, tmp);
        free(eta); free(s); free(lam); free(tmp);
    } else if (J->kind == KIND_F64) {
        double *eta = malloc(sizeof(double) * E), *s = malloc(sizeof(double) * N);
        double *lam = malloc(sizeof(double) * D), *tmp = malloc(sizeof(double) * D);
        if (!eta || !s || !lam || !tmp) J->rc = ORC_ERR_NOMEM;
        for (int64_t f = J->f0; f < J->f1 && J->rc == ORC_OK; f++)
            decode_frame_f64(g, &J->o, (const double *)J->in + f * N, J->bits + f * N, J->iters + f,
                             J->ok + f, J->soft ? (double *)J->soft + f * N : NULL, eta, s, lam, tmp);
        free(eta); free(s); free(lam); free(tmp);
    } else {
        int32_t *eta = malloc(sizeof(int32_t) * E), *s = malloc(sizeof(int32_t) * N);
        int32_t *lam = malloc(sizeof(int32_t) * D), *tmp = malloc(sizeof(int32_t) * D);
        if (!eta || !s || !lam || !tmp) J->rc = ORC_ERR_NOMEM;
        for (int64_t f = J->f0; f < J->f1 && J->rc == ORC_OK; f++)
            decode_frame_fixed(g, &J->o, (const int8_t *)J->in + f * N, J->bits + f * N,
                               J->iters + f, J->ok + f, J->soft ? (int16_t *)J->soft + f * N : NULL,
                               NULL, NULL, eta, s, lam, tmp);
        free(eta); free(s); free(lam); free(tmp);
    }
    return NULL;
}

static int run_batch(const orc_graph *g, int kind, const void *in, int64_t F, int32_t L,
                     int32_t early_stop, int32_t check_every, int32_t variant, int32_t flags,
                     int32_t nthreads, uint8_t *bits, int32_t *iters, uint8_t *ok, void *soft) {
    if (!g || F < 0 || L < 0) return ORC_ERR_ARG;
    if (F == 0) return ORC_OK;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > F) nthreads = (int32_t)F;
    job_t *jobs = (job_t *)calloc((size_t)nthreads, sizeof(job_t));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    orc_opts o = {L, early_stop, check_every, variant, flags};
    for (int32_t t = 0; t < nthreads; t++) {
        job_t *J = &jobs[t];
        J->g = g;
        J->o = o;
        J->kind = kind;
        J->in = in;
        J->f0 = F * t / nthreads;
        J->f1 = F * (t + 1) / nthreads;
        J->bits = bits;
        J->iters = iters;
        J->ok = ok;
        J->soft = soft;
        if (nthreads == 1) run_job(J);
        else pthread_create(&th[t], NULL, run_job, J);
    }
    int rc = ORC_OK;
    for (int32_t t = 0; t < nthreads; t++) {
        if (nthreads > 1) pthread_join(th[t], NULL);
        if (jobs[t].rc != ORC_OK) rc = jobs[t].rc;
    }
    free(jobs);
    free(th);
    return rc;
}

int orc_decode_f32(const orc_graph *g, const float *r, int64_t F, int32_t L, int32_t early_stop,
                   int32_t check_every, int32_t variant, int32_t flags, int32_t nthreads,
                   uint8_t *bits, int32_t *iters, uint8_t *ok, float *soft) {
    return run_batch(g, KIND_F32, r, F, L, early_stop, check_every, variant, flags, nthreads, bits,
                     iters, ok, soft);
}

int orc_decode_f64(const orc_graph *g, const double *r, int64_t F, int32_t L, int32_t early_stop,
                   int32_t check_every, int32_t variant, int32_t flags, int32_t nthreads,
                   uint8_t *bits, int32_t *iters, uint8_t *ok, double *soft) {
    return run_batch(g, KIND_F64, r, F, L, early_stop, check_every, variant, flags, nthreads, bits,
                     iters, ok, soft);
}

int orc_decode_fixed(const orc_graph *g, const int8_t *q, int64_t F, int32_t L, int32_t early_stop,
                     int32_t check_every, int32_t variant, int32_t flags, int32_t nthreads,
                     uint8_t *bits, int32_t *iters, uint8_t *ok, int16_t *soft) {
    return run_batch(g, KIND_FIXED, q, F, L, early_stop, check_every, variant, flags, nthreads,
                     bits, iters, ok, soft);
}

/* Single frame with per-iteration traces of eta (L x E, edge order = row-major edges with
 * ascending columns) and s (L x N). Iterations not run leave their trace rows untouched. */
int orc_trace_f32(const orc_graph *g, const float *r, int32_t L, int32_t early_stop,
                  int32_t check_every, int32_t variant, int32_t flags, uint8_t *bits,
                  int32_t *iters, uint8_t *ok, float *eta_trace, float *s_trace) {
    const int64_t D = max_row_degree(g);
    float *eta = malloc(sizeof(float) * (size_t)(g->E > 0 ? g->E : 1));
    float *s = malloc(sizeof(float) * (size_t)g->N);
    float *lam = malloc(sizeof(float) * (size_t)D), *tmp = malloc(sizeof(float) * (size_t)D);
    orc_opts o = {L, early_stop, check_every, variant, flags};
    int rc = decode_frame_f32(g, &o, r, bits, iters, ok, NULL, eta_trace, s_trace, eta, s, lam, tmp);
    free(eta); free(s); free(lam); free(tmp);
    return rc;
}

int orc_trace_fixed(const orc_graph *g, const int8_t *q, int32_t L, int32_t early_stop,
                    int32_t check_every, int32_t variant, int32_t flags, uint8_t *bits,
                    int32_t *iters, uint8_t *ok, int16_t *eta_trace, int16_t *s_trace) {
    const int64_t D = max_row_degree(g);
    int32_t *eta = malloc(sizeof(int32_t) * (size_t)(g->E > 0 ? g->E : 1));
    int32_t *s = malloc(sizeof(int32_t) * (size_t)g->N);
    int32_t *lam = malloc(sizeof(int32_t) * (size_t)D), *tmp = malloc(sizeof(int32_t) * (size_t)D);
    orc_opts o = {L, early_stop, check_every, variant, flags};
    int rc = decode_frame_fixed(g, &o, q, bits, iters, ok, NULL, eta_trace, s_trace, eta, s, lam, tmp);
    free(eta); free(s); free(lam); free(tmp);
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Algorithm 2: the dense masked map-reduce form on m x n matrices (Section   */
/* III), one frame, FP32. lambda(i,j) = s(j) H(i,j) - eta(i,j); row reductions */
/* min0, min0Location, min1 over the support of row i and sgn over the whole  */
/* row with sign(0) = +1; eta(i,j) per eq. (etaCalculation) with min1 at the  */
/* location of the minimum (Observation 1); s(j) = r(j) + column sum of eta.  */
/* ------------------------------------------------------------------------- */

int orc_decode_dense_f32(int32_t m, int32_t n, const uint8_t *H, const float *r, int32_t L,
                         int32_t early_stop, int32_t flags, uint8_t *b, int32_t *iters,
                         uint8_t *ok, float *soft) {
    if (m <= 0 || n <= 0 || L < 0) return ORC_ERR_ARG;
    const int64_t mn = (int64_t)m * n;
    float *lam = calloc((size_t)mn, sizeof(float)), *eta = calloc((size_t)mn, sizeof(float));
    float *s = malloc(sizeof(float) * (size_t)n);
    float *min0 = malloc(sizeof(float) * (size_t)m), *min1 = malloc(sizeof(float) * (size_t)m);
    int32_t *loc = malloc(sizeof(int32_t) * (size_t)m);
    int8_t *sgn = malloc((size_t)m);
    int32_t *zi = malloc(sizeof(int32_t) * (size_t)m);
    if (!lam || !eta || !s || !min0 || !min1 || !loc || !sgn || !zi) return ORC_ERR_NOMEM;
#define DENSE_SYNDROME_ZERO(res)                                                  \
    do {                                                                          \
        int64_t nz_ = 0;                                                          \
        for (int32_t i = 0; i < m; i++) {                                         \
            int32_t acc_ = 0; /* integer product H b, then mod 2 */              \
            for (int32_t j = 0; j < n; j++) acc_ += H[(int64_t)i * n + j] * b[j]; \
            zi[i] = acc_ % 2;                                                     \
            nz_ += zi[i];                                                         \
        }                                                                         \
        (res) = (nz_ == 0);                                                       \
    } while (0)
    for (int32_t j = 0; j < n; j++) s[j] = r[j];
    for (int32_t j = 0; j < n; j++) b[j] = slice_f32(s[j], flags);
    int32_t k = 0;
    int done = 0, is_cw;
    if (early_stop) {
        DENSE_SYNDROME_ZERO(is_cw);
        done = is_cw;
    }
    while (!done && k < L) {
        /* fan-out (map): lambda(i,j) = s(j) H(i,j) - eta(i,j) */
        for (int32_t i = 0; i < m; i++)
            for (int32_t j = 0; j < n; j++) {
                int64_t t = (int64_t)i * n + j;
                lam[t] = s[j] * (float)H[t] - eta[t];
            }
        /* row reductions */
        for (int32_t i = 0; i < m; i++) {
            float a0 = INFINITY, a1 = INFINITY;
            int32_t l0 = -1;
            int neg = 0;
            for (int32_t j = 0; j < n; j++) {
                int64_t t = (int64_t)i * n + j;
                if (lam[t] < 0.0f) neg ^= 1; /* whole row; zeros count as +1 */
                if (!H[t]) continue;
                float a = fabsf(lam[t]);
                if (a < a0) { a1 = a0; a0 = a; l0 = j; }
                else if (a < a1) { a1 = a; }
            }
            min0[i] = a0; min1[i] = a1; loc[i] = l0; sgn[i] = (int8_t)(neg ? -1 : 1);
        }
        /* eta(i,j) = H(i,j) * sign(lambda(i,j)) * sgn(i) * (min1 at the location, else min0) */
        for (int32_t i = 0; i < m; i++)
            for (int32_t j = 0; j < n; j++) {
                int64_t t = (int64_t)i * n + j;
                if (!H[t]) { eta[t] = 0.0f; continue; }
                int neg = (sgn[i] < 0) ^ (lam[t] < 0.0f);
                float mag = (j == loc[i]) ? min1[i] : min0[i];
                eta[t] = neg ? -mag : mag;
            }
        /* column sums: s(j) = r(j) + sum_i eta(i,j), rows ascending */
        for (int32_t j = 0; j < n; j++) {
            float acc = r[j];
            for (int32_t i = 0; i < m; i++) acc = acc + eta[(int64_t)i * n + j]; /* eta = 0 off H */
            s[j] = acc;
        }
        k++;
        for (int32_t j = 0; j < n; j++) b[j] = slice_f32(s[j], flags);
        if (early_stop) {
            DENSE_SYNDROME_ZERO(is_cw);
            done = is_cw;
        }
    }
    DENSE_SYNDROME_ZERO(is_cw);
#undef DENSE_SYNDROME_ZERO
    *iters = k;
    *ok = (uint8_t)is_cw;
    if (soft) memcpy(soft, s, sizeof(float) * (size_t)n);
    free(lam); free(eta); free(s); free(min0); free(min1); free(loc); free(sgn); free(zi);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Normalised / offset Min-Sum with learned weights (an extension of eq.      */
/* (eta_update); not in the paper). Every check-to-bit magnitude m is replaced */
/* by max(alpha * m - beta, 0), computed as one fused multiply-add, with alpha */
/* and beta chosen by the iteration k (row min(k, n_w) - 1 of the tables) and */
/* by the class of the edge's bit (col_class[j] in [0, n_classes)). With      */
/* alpha = 1 and beta = 0 this is plain Min-Sum. FP32 and binary64.           */
/* ------------------------------------------------------------------------- */

typedef struct {
    const int32_t *col_class;
    int32_t n_classes, n_w;
    const float *alpha, *beta;   /* [n_w][n_classes] */
    const double *alpha64, *beta64;
} orc_weights;

static inline float weigh_f32(const orc_weights *w, int32_t k, int32_t j, float m) {
    if (!w || w->n_w <= 0) return m;
    int32_t row = (k < w->n_w ? k : w->n_w) - 1;
    int32_t c = w->col_class[j];
    float a = fmaf(w->alpha[row * w->n_classes + c], m, -w->beta[row * w->n_classes + c]);
    return a > 0.0f ? a : 0.0f;
}

static inline double weigh_f64(const orc_weights *w, int32_t k, int32_t j, double m) {
    if (!w || w->n_w <= 0) return m;
    int32_t row = (k < w->n_w ? k : w->n_w) - 1;
    int32_t c = w->col_class[j];
    double a = fma(w->alpha64[row * w->n_classes + c], m, -w->beta64[row * w->n_classes + c]);
    return a > 0.0 ? a : 0.0;
}

/* One frame; the check update through Observations 1 and 2, magnitudes weighted. */
static int decode_frame_w_f32(const orc_graph *g, const orc_opts *o, const orc_weights *w,
                              const float *r, uint8_t *b, int32_t *iters, uint8_t *ok, float *soft,
                              float *eta, float *s, float *lam) {
    const int32_t M = g->M, N = g->N;
    const int64_t E = g->E;
    for (int32_t j = 0; j < N; j++) s[j] = r[j];
    for (int64_t e = 0; e < E; e++) eta[e] = 0.0f;
    for (int32_t j = 0; j < N; j++) b[j] = slice_f32(s[j], o->flags);
    int32_t k = 0;
    int done = test_now(o, 0) && orc_syndrome(g, b, NULL) == 0;
    while (!done && k < o->L) {
        for (int32_t i = 0; i < M; i++) {
            int64_t e0 = g->row_ptr[i], d = g->row_ptr[i + 1] - e0;
            float min0 = INFINITY, min1 = INFINITY;
            int64_t loc = -1;
            int neg = 0;
            for (int64_t t = 0; t < d; t++) {
                lam[t] = s[g->col_of[e0 + t]] - eta[e0 + t];
                float a = fabsf(lam[t]);
                if (a < min0) { min1 = min0; min0 = a; loc = t; }
                else if (a < min1) { min1 = a; }
                if (lam[t] < 0.0f) neg ^= 1;
            }
            for (int64_t t = 0; t < d; t++) {
                float m = weigh_f32(w, k + 1, g->col_of[e0 + t], t == loc ? min1 : min0);
                eta[e0 + t] = (neg ^ (lam[t] < 0.0f)) ? -m : m;
            }
        }
        for (int32_t j = 0; j < N; j++) {
            float acc = r[j];
            for (int64_t t = g->col_ptr[j]; t < g->col_ptr[j + 1]; t++) acc = acc + eta[g->edge_of[t]];
            s[j] = acc;
        }
        k++;
        for (int32_t j = 0; j < N; j++) b[j] = slice_f32(s[j], o->flags);
        if (test_now(o, k) && orc_syndrome(g, b, NULL) == 0) done = 1;
    }
    *iters = k;
    *ok = (uint8_t)(orc_syndrome(g, b, NULL) == 0);
    if (soft) memcpy(soft, s, sizeof(float) * (size_t)N);
    return ORC_OK;
}

static int decode_frame_w_f64(const orc_graph *g, const orc_opts *o, const orc_weights *w,
                              const double *r, double *soft, double *eta, double *s, double *lam) {
    const int32_t M = g->M, N = g->N;
    for (int32_t j = 0; j < N; j++) s[j] = r[j];
    for (int64_t e = 0; e < g->E; e++) eta[e] = 0.0;
    for (int32_t k = 0; k < o->L; k++) {
        for (int32_t i = 0; i < M; i++) {
            int64_t e0 = g->row_ptr[i], d = g->row_ptr[i + 1] - e0;
            double min0 = INFINITY, min1 = INFINITY;
            int64_t loc = -1;
            int neg = 0;
            for (int64_t t = 0; t < d; t++) {
                lam[t] = s[g->col_of[e0 + t]] - eta[e0 + t];
                double a = fabs(lam[t]);
                if (a < min0) { min1 = min0; min0 = a; loc = t; }
                else if (a < min1) { min1 = a; }
                if (lam[t] < 0.0) neg ^= 1;
            }
            for (int64_t t = 0; t < d; t++) {
                double m = weigh_f64(w, k + 1, g->col_of[e0 + t], t == loc ? min1 : min0);
                eta[e0 + t] = (neg ^ (lam[t] < 0.0)) ? -m : m;
            }
        }
        for (int32_t j = 0; j < N; j++) {
            double acc = r[j];
            for (int64_t t = g->col_ptr[j]; t < g->col_ptr[j + 1]; t++) acc = acc + eta[g->edge_of[t]];
            s[j] = acc;
        }
    }
    memcpy(soft, s, sizeof(double) * (size_t)N);
    return ORC_OK;
}

/* Batch of FP32 frames with early stop options, like orc_decode_f32. */
int orc_decode_weighted_f32(const orc_graph *g, const float *r, int64_t F, int32_t L,
                            int32_t early_stop, int32_t check_every, int32_t flags,
                            const int32_t *col_class, int32_t n_classes, int32_t n_w,
                            const float *alpha, const float *beta, uint8_t *bits, int32_t *iters,
                            uint8_t *ok, float *soft) {
    if (!g || F < 0 || L < 0 || n_classes < 1 || n_w < 0) return ORC_ERR_ARG;
    for (int32_t j = 0; j < g->N; j++)
        if (col_class[j] < 0 || col_class[j] >= n_classes) return ORC_ERR_ARG;
    orc_opts o = {L, early_stop, check_every, ORC_CHECK_TWOMIN, flags};
    orc_weights w = {col_class, n_classes, n_w, alpha, beta, NULL, NULL};
    const int64_t D = max_row_degree(g);
    float *eta = malloc(sizeof(float) * (size_t)(g->E > 0 ? g->E : 1));
    float *s = malloc(sizeof(float) * (size_t)g->N), *lam = malloc(sizeof(float) * (size_t)D);
    for (int64_t f = 0; f < F; f++)
        decode_frame_w_f32(g, &o, &w, r + f * g->N, bits + f * g->N, iters + f, ok + f,
                           soft ? soft + f * g->N : NULL, eta, s, lam);
    free(eta); free(s); free(lam);
    return ORC_OK;
}

/* Batch of binary64 frames, exactly L iterations (no early stop): the posteriors only. */
int orc_decode_weighted_f64(const orc_graph *g, const double *r, int64_t F, int32_t L,
                            const int32_t *col_class, int32_t n_classes, int32_t n_w,
                            const double *alpha, const double *beta, double *soft) {
    if (!g || F < 0 || L < 0 || n_classes < 1 || n_w < 0) return ORC_ERR_ARG;
    orc_opts o = {L, 0, 1, ORC_CHECK_TWOMIN, 0};
    orc_weights w = {col_class, n_classes, n_w, NULL, NULL, alpha, beta};
    const int64_t D = max_row_degree(g);
    double *eta = malloc(sizeof(double) * (size_t)(g->E > 0 ? g->E : 1));
    double *s = malloc(sizeof(double) * (size_t)g->N), *lam = malloc(sizeof(double) * (size_t)D);
    for (int64_t f = 0; f < F; f++) decode_frame_w_f64(g, &o, &w, r + f * g->N, soft + f * g->N, eta, s, lam);
    free(eta); free(s); free(lam);
    return ORC_OK;
}
