/*
 * Cleora FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see cleora_oracle.h).
 *
 * Written from arXiv 2102.02302, Sec. 3.2 ("Embedding": M_ab = e_ab / deg(v_a), T0 ~ U(-1,1),
 * multiply then L2-normalise rows for I iterations) and Algorithm 1 with a single chunk.
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - node order: dense index = rank of the external id in ascending order;
 *   - an undirected self-loop contributes its weight once;
 *   - deg_a is the weighted out-degree sum_b e_ab, so every row of M sums to 1;
 *   - "constant L2 norm" is norm 1;
 *   - a row with deg_a = 0 (a directed sink) keeps its previous row, renormalised;
 *   - a row whose average is exactly zero is output as zeros;
 *   - weights must be finite and > 0.
 * The code is deliberately simple: qsort, sequential sums, one thread per block of rows.
 */
#include "cleora_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

struct oracle_graph {
    int64_t n, nnz;
    uint64_t* ids;     /* n, ascending */
    int64_t* rowptr;   /* n + 1 */
    int32_t* col;      /* nnz, ascending within a row */
    double* e;         /* nnz: e_ab */
    double* deg;       /* n: deg_a */
    int weighted;
    int has_val;
};

/* splitmix64 output function (Steele, Lea & Flood 2014; Vigna's splitmix64.c). */
static uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return (x > y) - (x < y);
}

typedef struct { int64_t row, col, edge; double w; } entry;

static int cmp_entry(const void* a, const void* b) {
    const entry* x = (const entry*)a;
    const entry* y = (const entry*)b;
    if (x->row != y->row) return (x->row > y->row) - (x->row < y->row);
    if (x->col != y->col) return (x->col > y->col) - (x->col < y->col);
    return (x->edge > y->edge) - (x->edge < y->edge);
}

static int64_t index_of(const uint64_t* ids, int64_t n, uint64_t id) {
    int64_t lo = 0, hi = n; /* first position with ids[pos] >= id */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (ids[mid] < id) lo = mid + 1; else hi = mid;
    }
    return lo;
}

void oracle_graph_free(oracle_graph* g) {
    if (!g) return;
    free(g->ids); free(g->rowptr); free(g->col); free(g->e); free(g->deg);
    free(g);
}

int oracle_build(const uint64_t* src, const uint64_t* dst, const float* w, int64_t num_edges,
                 int directed, oracle_graph** out) {
    if (!out || num_edges < 0 || (num_edges > 0 && (!src || !dst))) return -1;
    *out = NULL;
    for (int64_t k = 0; w && k < num_edges; ++k)
        if (!(isfinite(w[k]) && w[k] > 0.0f)) return -1;

    oracle_graph* g = (oracle_graph*)calloc(1, sizeof(oracle_graph));
    if (!g) return -2;
    g->weighted = (w != NULL);

    /* V: distinct ids, ascending. */
    uint64_t* all = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * num_edges + 1));
    if (!all) { oracle_graph_free(g); return -2; }
    for (int64_t k = 0; k < num_edges; ++k) { all[2 * k] = src[k]; all[2 * k + 1] = dst[k]; }
    qsort(all, (size_t)(2 * num_edges), sizeof(uint64_t), cmp_u64);
    int64_t n = 0;
    for (int64_t k = 0; k < 2 * num_edges; ++k)
        if (k == 0 || all[k] != all[k - 1]) all[n++] = all[k];
    if (n >= ((int64_t)1 << 31)) { free(all); oracle_graph_free(g); return -1; }
    g->n = n;
    g->ids = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(n + 1));
    if (!g->ids) { free(all); oracle_graph_free(g); return -2; }
    memcpy(g->ids, all, sizeof(uint64_t) * (size_t)n);
    free(all);

    /* Directed entries a->b with their edge number and weight. */
    entry* ent = (entry*)malloc(sizeof(entry) * (size_t)(2 * num_edges + 1));
    if (!ent) { oracle_graph_free(g); return -2; }
    int64_t m = 0;
    for (int64_t k = 0; k < num_edges; ++k) {
        int64_t a = index_of(g->ids, n, src[k]);
        int64_t b = index_of(g->ids, n, dst[k]);
        double wk = w ? (double)w[k] : 1.0;
        ent[m].row = a; ent[m].col = b; ent[m].edge = k; ent[m].w = wk; ++m;
        if (!directed && a != b) {
            ent[m].row = b; ent[m].col = a; ent[m].edge = k; ent[m].w = wk; ++m;
        }
    }
    qsort(ent, (size_t)m, sizeof(entry), cmp_entry);

    /* Merge duplicates: e_ab is the sum of the weights of all a->b edges, added in
     * ascending edge order. */
    int64_t nnz = 0;
    for (int64_t k = 0; k < m; ++k)
        if (k == 0 || ent[k].row != ent[k - 1].row || ent[k].col != ent[k - 1].col) ++nnz;
    g->nnz = nnz;
    g->rowptr = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    g->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz + 1));
    g->e = (double*)malloc(sizeof(double) * (size_t)(nnz + 1));
    g->deg = (double*)calloc((size_t)(n + 1), sizeof(double));
    if (!g->rowptr || !g->col || !g->e || !g->deg) { free(ent); oracle_graph_free(g); return -2; }
    int64_t p = -1;
    for (int64_t k = 0; k < m; ++k) {
        if (k == 0 || ent[k].row != ent[k - 1].row || ent[k].col != ent[k - 1].col) {
            ++p;
            g->col[p] = (int32_t)ent[k].col;
            g->e[p] = 0.0;
            g->rowptr[ent[k].row + 1] += 1;
        }
        g->e[p] += ent[k].w;
    }
    free(ent);
    for (int64_t a = 0; a < n; ++a) g->rowptr[a + 1] += g->rowptr[a];

    /* deg_a = sum_b e_ab in ascending b; the store needs values when any e_ab != 1. */
    g->has_val = g->weighted;
    for (int64_t a = 0; a < n; ++a) {
        double s = 0.0;
        for (int64_t k = g->rowptr[a]; k < g->rowptr[a + 1]; ++k) {
            s += g->e[k];
            if (g->e[k] != 1.0) g->has_val = 1;
        }
        g->deg[a] = s;
    }
    *out = g;
    return 0;
}

int64_t oracle_graph_n(const oracle_graph* g) { return g ? g->n : 0; }
int64_t oracle_graph_nnz(const oracle_graph* g) { return g ? g->nnz : 0; }
int oracle_graph_has_val(const oracle_graph* g) { return g ? g->has_val : 0; }

void oracle_graph_copy(const oracle_graph* g, uint64_t* ids, int64_t* rowptr, int32_t* col,
                       double* e, double* deg) {
    if (ids) memcpy(ids, g->ids, sizeof(uint64_t) * (size_t)g->n);
    if (rowptr) memcpy(rowptr, g->rowptr, sizeof(int64_t) * (size_t)(g->n + 1));
    if (col) memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
    if (e) memcpy(e, g->e, sizeof(double) * (size_t)g->nnz);
    if (deg) memcpy(deg, g->deg, sizeof(double) * (size_t)g->n);
}

void oracle_stored_values(const oracle_graph* g, float* val, float* inv_deg) {
    for (int64_t a = 0; a < g->n; ++a) {
        if (inv_deg) inv_deg[a] = g->deg[a] > 0.0 ? 1.0f / (float)g->deg[a] : 0.0f;
        if (val)
            for (int64_t k = g->rowptr[a]; k < g->rowptr[a + 1]; ++k)
                val[k] = (float)(g->e[k] / g->deg[a]);
    }
}

uint64_t oracle_mix(uint64_t z) { return mix(z); }

double oracle_init_value(uint64_t seed, uint64_t id, uint32_t j) {
    uint64_t h = mix(mix(mix(seed) ^ id) ^ (uint64_t)j);
    double u = (double)(h >> 40) * (1.0 / 16777216.0); /* in [0, 1) */
    return 2.0 * u - 1.0;
}

void oracle_init(const uint64_t* ids, int64_t n, int d, uint64_t seed, double* T0) {
    for (int64_t i = 0; i < n; ++i)
        for (int j = 0; j < d; ++j)
            T0[i * (int64_t)d + j] = oracle_init_value(seed, ids[i], (uint32_t)j);
}

/* One row of one iteration: y = sum_b M_ab T[b] (ascending b), then y / ||y||_2. */
static void step_row(const oracle_graph* g, int d, const double* T, int64_t a, double* y) {
    int64_t beg = g->rowptr[a], end = g->rowptr[a + 1];
    if (beg == end) {
        memcpy(y, T + a * (int64_t)d, sizeof(double) * (size_t)d);  /* sink keeps its row */
    } else {
        for (int j = 0; j < d; ++j) y[j] = 0.0;
        for (int64_t k = beg; k < end; ++k) {
            double mab = g->e[k] / g->deg[a];
            const double* tb = T + (int64_t)g->col[k] * d;
            for (int j = 0; j < d; ++j) y[j] += mab * tb[j];
        }
    }
    double ss = 0.0;
    for (int j = 0; j < d; ++j) ss += y[j] * y[j];
    double nrm = sqrt(ss);
    for (int j = 0; j < d; ++j) y[j] = nrm > 0.0 ? y[j] / nrm : 0.0;
}

typedef struct {
    const oracle_graph* g;
    int d;
    const double* Tin;
    double* Tout;
    const int64_t* rows;  /* NULL: rows are r0..r1-1 themselves */
    int64_t r0, r1;
} step_job;

static void* step_worker(void* arg) {
    step_job* jb = (step_job*)arg;
    for (int64_t r = jb->r0; r < jb->r1; ++r) {
        int64_t a = jb->rows ? jb->rows[r] : r;
        step_row(jb->g, jb->d, jb->Tin, a, jb->Tout + r * (int64_t)jb->d);
    }
    return NULL;
}

static int run_rows(const oracle_graph* g, int d, const double* Tin, double* Tout,
                    const int64_t* rows, int64_t count, int nthreads) {
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if ((int64_t)nthreads > count) nthreads = count > 0 ? (int)count : 1;
    pthread_t th[256];
    step_job jobs[256];
    for (int t = 0; t < nthreads; ++t) {
        jobs[t].g = g; jobs[t].d = d; jobs[t].Tin = Tin; jobs[t].Tout = Tout; jobs[t].rows = rows;
        jobs[t].r0 = count * t / nthreads;
        jobs[t].r1 = count * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; ++t)
        if (pthread_create(&th[t], NULL, step_worker, &jobs[t]) != 0) {
            for (int u = 1; u < t; ++u) pthread_join(th[u], NULL);
            return -2;
        }
    step_worker(&jobs[0]);
    for (int t = 1; t < nthreads; ++t) pthread_join(th[t], NULL);
    return 0;
}

int oracle_propagate(const oracle_graph* g, int d, const double* T_in, int iters,
                     double* T_out, int nthreads) {
    if (!g || d < 1 || iters < 0) return -1;
    size_t bytes = sizeof(double) * (size_t)g->n * (size_t)d;
    if (g->n == 0) return 0;
    double* a = (double*)malloc(bytes);
    double* b = (double*)malloc(bytes);
    if (!a || !b) { free(a); free(b); return -2; }
    memcpy(a, T_in, bytes);
    for (int it = 0; it < iters; ++it) {
        int rc = run_rows(g, d, a, b, NULL, g->n, nthreads);
        if (rc) { free(a); free(b); return rc; }
        double* t = a; a = b; b = t;
    }
    memcpy(T_out, a, bytes);
    free(a); free(b);
    return 0;
}

int oracle_step_rows(const oracle_graph* g, int d, const double* T_prev, const int64_t* rows,
                     int64_t nrows, double* out, int nthreads) {
    if (!g || d < 1 || nrows < 0) return -1;
    for (int64_t r = 0; r < nrows; ++r)
        if (rows[r] < 0 || rows[r] >= g->n) return -1;
    return run_rows(g, d, T_prev, out, rows, nrows, nthreads);
}

/* ---- one step over an external CSR (graphs too large to build here) ---------------------- */

typedef struct {
    const int64_t* rowptr;
    const int32_t* col;
    const double* e;
    int64_t n;
    int d;
    const float* T;
    const int64_t* rows;
    int64_t nrows;
    double* out;
    int64_t next; /* next row to hand out (atomic) */
    int bad;
} csr_job;

static void csr_row(const csr_job* jb, int64_t a, double* y) {
    const int d = jb->d;
    int64_t beg = jb->rowptr[a], end = jb->rowptr[a + 1];
    if (beg == end) {
        for (int j = 0; j < d; ++j) y[j] = (double)jb->T[a * (int64_t)d + j];
    } else {
        double deg = 0.0;
        for (int64_t k = beg; k < end; ++k) deg += jb->e ? jb->e[k] : 1.0;
        for (int j = 0; j < d; ++j) y[j] = 0.0;
        for (int64_t k = beg; k < end; ++k) {
            double mab = (jb->e ? jb->e[k] : 1.0) / deg;
            const float* tb = jb->T + (int64_t)jb->col[k] * d;
            for (int j = 0; j < d; ++j) y[j] += mab * (double)tb[j];
        }
    }
    double ss = 0.0;
    for (int j = 0; j < d; ++j) ss += y[j] * y[j];
    double nrm = sqrt(ss);
    for (int j = 0; j < d; ++j) y[j] = nrm > 0.0 ? y[j] / nrm : 0.0;
}

static void* csr_worker(void* arg) {
    csr_job* jb = (csr_job*)arg;
    for (;;) {
        int64_t r = __atomic_fetch_add(&jb->next, 1, __ATOMIC_RELAXED);
        if (r >= jb->nrows) break;
        csr_row(jb, jb->rows[r], jb->out + r * (int64_t)jb->d);
    }
    return NULL;
}

int oracle_step_csr_rows(const int64_t* rowptr, const int32_t* col, const double* e, int64_t n,
                         int d, const float* T_prev, const int64_t* rows, int64_t nrows,
                         double* out, int nthreads) {
    if (!rowptr || !T_prev || !rows || !out || d < 1 || n < 0 || nrows < 0) return -1;
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t a = rows[r];
        if (a < 0 || a >= n) return -1;
        for (int64_t k = rowptr[a]; k < rowptr[a + 1]; ++k)
            if (col[k] < 0 || col[k] >= n) return -1;
    }
    csr_job jb = {rowptr, col, e, n, d, T_prev, rows, nrows, out, 0, 0};
    if (nthreads <= 0) nthreads = (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 1;
    for (int t = 1; t < nthreads; ++t, ++started)
        if (pthread_create(&th[t], NULL, csr_worker, &jb) != 0) break;
    csr_worker(&jb);
    for (int t = 1; t < started; ++t) pthread_join(th[t], NULL);
    return 0;
}

/* ---- XXH64 (xxHash specification, 64-bit variant) ---------------------------------------- */

static const uint64_t XP1 = 0x9E3779B185EBCA87ULL, XP2 = 0xC2B2AE3D27D4EB4FULL,
                      XP3 = 0x165667B19E3779F9ULL, XP4 = 0x85EBCA77C2B2AE63ULL,
                      XP5 = 0x27D4EB2F165667C5ULL;

static uint64_t rotl64(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

/* little-endian reads, byte by byte (no alignment or host byte-order assumption) */
static uint64_t le64(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 7; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}
static uint64_t le32(const uint8_t* p) {
    uint64_t v = 0;
    for (int i = 3; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}

static uint64_t xround(uint64_t acc, uint64_t lane) {
    acc += lane * XP2;
    acc = rotl64(acc, 31);
    return acc * XP1;
}

static uint64_t xmerge(uint64_t acc, uint64_t v) {
    acc ^= xround(0, v);
    return acc * XP1 + XP4;
}

uint64_t oracle_xxh64(const uint8_t* p, int64_t len, uint64_t seed) {
    int64_t i = 0;
    uint64_t acc;
    if (len >= 32) {
        uint64_t a1 = seed + XP1 + XP2, a2 = seed + XP2, a3 = seed, a4 = seed - XP1;
        for (; i + 32 <= len; i += 32) {
            a1 = xround(a1, le64(p + i));
            a2 = xround(a2, le64(p + i + 8));
            a3 = xround(a3, le64(p + i + 16));
            a4 = xround(a4, le64(p + i + 24));
        }
        acc = rotl64(a1, 1) + rotl64(a2, 7) + rotl64(a3, 12) + rotl64(a4, 18);
        acc = xmerge(acc, a1);
        acc = xmerge(acc, a2);
        acc = xmerge(acc, a3);
        acc = xmerge(acc, a4);
    } else {
        acc = seed + XP5;
    }
    acc += (uint64_t)len;
    for (; i + 8 <= len; i += 8) {
        acc ^= xround(0, le64(p + i));
        acc = rotl64(acc, 27) * XP1 + XP4;
    }
    if (i + 4 <= len) {
        acc ^= le32(p + i) * XP1;
        acc = rotl64(acc, 23) * XP2 + XP3;
        i += 4;
    }
    for (; i < len; ++i) {
        acc ^= (uint64_t)p[i] * XP5;
        acc = rotl64(acc, 11) * XP1;
    }
    acc ^= acc >> 33;
    acc *= XP2;
    acc ^= acc >> 29;
    acc *= XP3;
    acc ^= acc >> 32;
    return acc;
}

void oracle_hash_strings(const uint8_t* bytes, const int64_t* offsets, int64_t count, uint64_t seed,
                         uint64_t* out) {
    for (int64_t k = 0; k < count; ++k)
        out[k] = oracle_xxh64(bytes + offsets[k], offsets[k + 1] - offsets[k], seed);
}
