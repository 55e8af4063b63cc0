/*
 * Cleora FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, obviously correct restatement of the Cleora embedding (arXiv 2102.02302,
 * Sec. 3.2 and Algorithm 1) used to check the CUDA library.  Only the tests, the package's
 * smoke entry and the bench's CPU-baseline leg may load it; the product path never does.
 * It shares no code, header or table with the CUDA library.
 *
 * Every function returns 0 on success, -1 for an invalid argument, -2 when out of memory.
 */
#ifndef CLEORA_ORACLE_H
#define CLEORA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oracle_graph oracle_graph;

/* Graph and transition matrix M = D^-1 A (Sec. 3.2, "Embedding"; Algorithm 1, M_q).
 * Nodes are the distinct ids among src and dst, indexed by rank in ascending id order.
 * e_ab sums the weights (1 when w == NULL) of the edges a->b; undirected edges count in
 * both directions (Sec. 4.5), a self-loop once.  deg_a = sum_b e_ab, M_ab = e_ab / deg_a. */
int oracle_build(const uint64_t* src, const uint64_t* dst, const float* w, int64_t num_edges,
                 int directed, oracle_graph** out);
void oracle_graph_free(oracle_graph* g);
int64_t oracle_graph_n(const oracle_graph* g);
int64_t oracle_graph_nnz(const oracle_graph* g);
/* 1 when the stored CSR needs per-entry values (weighted, or some multiplicity != 1). */
int oracle_graph_has_val(const oracle_graph* g);
/* Copies out any non-NULL array: ids[n], rowptr[n+1], col[nnz], e[nnz], deg[n]. */
void oracle_graph_copy(const oracle_graph* g, uint64_t* ids, int64_t* rowptr, int32_t* col,
                       double* e, double* deg);
/* The FP32 values a compact store keeps: val[k] = fp32(e_ab / deg_a) (FP64 division, one
 * rounding to FP32) and inv_deg[a] = 1.0f / fp32(deg_a) (FP32 division). */
void oracle_stored_values(const oracle_graph* g, float* val, float* inv_deg);

/* T0 ~ U(-1, 1) (Sec. 3.2; Algorithm 1 "Initialize"), made deterministic:
 * h = mix(mix(mix(seed) ^ id) ^ j), T0[i][j] = 2 * (h >> 40) * 2^-24 - 1. */
uint64_t oracle_mix(uint64_t z); /* the splitmix64 output function used by the hash */
double oracle_init_value(uint64_t seed, uint64_t id, uint32_t j);
void oracle_init(const uint64_t* ids, int64_t n, int d, uint64_t seed, double* T0);

/* I iterations of T_i = rownorm_L2(M T_{i-1}) (Algorithm 1, inner loop), FP64.
 * T_in and T_out are n x d row-major; they may alias. nthreads <= 0: all cores. */
int oracle_propagate(const oracle_graph* g, int d, const double* T_in, int iters,
                     double* T_out, int nthreads);
/* One iteration restricted to the listed rows: out[r] = rownorm(M T_prev)[rows[r]]. */
int oracle_step_rows(const oracle_graph* g, int d, const double* T_prev, const int64_t* rows,
                     int64_t nrows, double* out, int nthreads);
/* The same step for a graph given as a CSR (rowptr[n+1], col[nnz]; e[nnz] = e_ab, or NULL
 * when every e_ab is 1) and an FP32 T_prev (n x d), for graphs too large to build here:
 * out[r] = rownorm(sum_b (e_ab / deg_a) T_prev[b]) for a = rows[r], deg_a = sum_b e_ab in
 * ascending position, FP64 throughout; a row without entries keeps T_prev[a] renormalised.
 * Rows are handed to threads one at a time (long rows do not hold up a block of others). */
int oracle_step_csr_rows(const int64_t* rowptr, const int32_t* col, const double* e, int64_t n,
                         int d, const float* T_prev, const int64_t* rows, int64_t nrows,
                         double* out, int nthreads);

/* XXH64 of len bytes (the xxHash specification, 64-bit variant), the hash the paper uses to
 * turn entity identifiers into a small fixed-width format (Sec. 4.3).  oracle_hash_strings
 * hashes strings bytes[offsets[i] .. offsets[i+1]) for i < count. */
uint64_t oracle_xxh64(const uint8_t* p, int64_t len, uint64_t seed);
void oracle_hash_strings(const uint8_t* bytes, const int64_t* offsets, int64_t count, uint64_t seed,
                         uint64_t* out);

#ifdef __cplusplus
}
#endif
#endif
