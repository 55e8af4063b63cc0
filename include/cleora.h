/*
 * cleora.h -- C ABI of the GB300 (sm_103a) Cleora propagation library.
 *
 * Cleora (arXiv 2102.02302) embeds a graph by iterating T_i = rownorm_L2(M T_{i-1}) with the
 * random-walk transition matrix M = D^-1 A (Sec. 3.2, "Embedding"; Algorithm 1), starting
 * from T_0 ~ U(-1, 1).  This library builds M on the GPU from an edge list, fills T_0 and
 * runs the iterations with hand-written CUDA kernels.
 *
 * Conventions for every call:
 *   - The return value is a cleora_status (0 = CLEORA_OK).  No C++ exception crosses the
 *     ABI.  On failure, cleora_last_error(ctx) returns a one-line description; the context
 *     state is unchanged unless the call says otherwise.
 *   - Pointers are plain host or device addresses, as the matching *_on_device flag says.
 *     Device pointers must belong to the context's device.  The caller owns every array it
 *     passes; the library copies inputs during the call and never keeps a caller pointer.
 *   - The library owns the graph (CSR) and embedding buffers of a context and frees them
 *     on cleora_destroy or when a new graph is built.
 *   - Work is ordered on the context's stream.  A call that writes to host memory returns
 *     after the data is there.  A call that only touches device memory may return before
 *     the GPU is done; cleora_sync waits and reports errors the kernels raised.
 *   - State machine: create -> graph_build -> init -> propagate (repeatable).  Calls out of
 *     order return CLEORA_ERR_STATE.
 */
#ifndef CLEORA_H
#define CLEORA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cleora_ctx cleora_ctx;

typedef enum {
    CLEORA_OK = 0,
    CLEORA_ERR_INVALID_ARG = -1, /* a size, pointer, flag or weight is out of range      */
    CLEORA_ERR_OOM = -2,         /* device (or pinned host) memory ran out                 */
    CLEORA_ERR_CUDA = -3,        /* a CUDA runtime call failed                             */
    CLEORA_ERR_STATE = -4,       /* call out of order (e.g. propagate before init)         */
    CLEORA_ERR_TIMEOUT = -5,     /* a bounded wait ran out                                 */
    CLEORA_ERR_REJECTED = -6,    /* serving: the job can never fit the memory budget       */
    CLEORA_ERR_DEVICE = -7,      /* a kernel reported an inconsistency through its flag    */
    CLEORA_ERR_CANCELLED = -8    /* serving: the job was cancelled before it started       */
} cleora_status;

typedef enum { CLEORA_F32 = 0, CLEORA_BF16 = 1 } cleora_dtype;

/* ---------------------------------------------------------------------------------------
 * Context
 * ------------------------------------------------------------------------------------- */

/* Creates a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t the caller
 * owns (it must outlive the context), or NULL for a stream the context creates itself.
 * Device memory comes from a private stream-ordered pool that keeps freed blocks for
 * reuse; it is returned to the driver by cleora_destroy. */
int cleora_create(cleora_ctx** out, int device, void* cuda_stream);
void cleora_destroy(cleora_ctx* ctx);
const char* cleora_last_error(const cleora_ctx* ctx);
const char* cleora_status_string(int status);
/* Waits for the context's stream; returns CLEORA_ERR_DEVICE if a kernel raised its error
 * flag since the last check (the flag is then cleared). */
int cleora_sync(cleora_ctx* ctx);

/* ---------------------------------------------------------------------------------------
 * Graph build: node ids, CSR of M = D^-1 A (Sec. 3.2, "Embedding"; Algorithm 1, M_q)
 * ------------------------------------------------------------------------------------- */

/* Builds the transition matrix of the graph with edges src[k] -> dst[k], k < num_edges.
 *   - Nodes are the distinct uint64 ids among src and dst; node index = rank of the id in
 *     ascending order (so output rows follow ascending id).  At most 2^31 - 1 nodes.
 *   - e_ab = sum of the weights of the edges a->b (weights == NULL: every weight is 1).
 *     Undirected (directed == 0): each edge also counts as b->a (Sec. 4.5), except a
 *     self-loop, which counts once.  Duplicates merge, their weights added as FP64 in
 *     ascending edge order.
 *   - deg_a = sum_b e_ab (FP64, ascending b), so every row of M sums to 1.
 *   - Stored values: when the graph is weighted or some e_ab != 1, val[k] =
 *     fp32(e_ab / deg_a) (FP64 division, one rounding); always inv_deg[a] = 1.0f/fp32(deg_a).
 *   - Weights must be finite and > 0, else CLEORA_ERR_INVALID_ARG.
 *   - num_edges == 0 gives the empty graph (n = 0); init and propagate are then no-ops.
 * src/dst/weights are host arrays (inputs_on_device == 0) or device arrays (1).  The call
 * returns when the graph is built.  A previous graph and its embeddings are released. */
int cleora_graph_build(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst,
                       const float* weights, int64_t num_edges, int directed,
                       int inputs_on_device);
int cleora_num_nodes(const cleora_ctx* ctx, int64_t* n);
int cleora_num_entries(const cleora_ctx* ctx, int64_t* nnz);
/* has_val: 1 when per-entry values are stored; max_deg: largest row length. */
int cleora_graph_info(const cleora_ctx* ctx, int64_t* n, int64_t* nnz, int* has_val,
                      int64_t* max_row_len);
/* ids[n], ascending. */
int cleora_node_ids(cleora_ctx* ctx, uint64_t* out, int out_on_device);
/* Any output may be NULL.  rowptr[n+1] (int64), col[nnz] (int32, ascending in a row),
 * val[nnz] = M_ab as FP32 (the stored value, or inv_deg[a] when no values are stored),
 * inv_deg[n] (FP32), deg[n] (FP64). */
int cleora_get_csr(cleora_ctx* ctx, int64_t* rowptr, int32_t* col, float* val, float* inv_deg,
                   double* deg, int out_on_device);

/* ---------------------------------------------------------------------------------------
 * Embeddings (Sec. 3.2; Algorithm 1: initialise, then I times multiply and normalise)
 * ------------------------------------------------------------------------------------- */

/* Fills T_0 (n x d, row-major) in the storage type `storage`:
 *   h = mix(mix(mix(seed) ^ id_i) ^ j),  T_0[i][j] = 2 * (h >> 40) * 2^-24 - 1,
 * mix = the splitmix64 output function (add 0x9E3779B97F4A7C15, xor-shift 30, multiply
 * 0xBF58476D1CE4E5B9, xor-shift 27, multiply 0x94D049BB133111EB, xor-shift 31).  The value
 * is exact in FP32; BF16 storage keeps its round-to-nearest-even.  T_0 is not normalised.
 * d must be a multiple of 8 in [8, 1024]. */
int cleora_init(cleora_ctx* ctx, int d, uint64_t seed, cleora_dtype storage);

/* Runs `iters` (>= 0) iterations T_k = rownorm_L2(M T_{k-1}) from the current embeddings:
 *   y_a = sum_b M_ab T_{k-1}[b]  (FP32 accumulation whatever the storage type),
 *   T_k[a] = y_a / ||y_a||_2     (FP32 norm; BF16 storage rounds to nearest even).
 * A row with no entries (a directed sink) keeps T_{k-1}[a] / ||T_{k-1}[a]||; a row whose
 * y is exactly zero becomes zero.  Results are deterministic (no floating-point atomics),
 * and propagate(a) then propagate(b) equals propagate(a + b) bit for bit.
 * If out != NULL, T_k is also written there as FP32 n x d (host or device). */
int cleora_propagate(cleora_ctx* ctx, int iters, float* out, int out_on_device);
/* Iterations run since init / set_embeddings. */
int cleora_iteration(const cleora_ctx* ctx, int* k);
/* Copies the current embeddings (n x d) out, converted to `dtype`. */
int cleora_get_embeddings(cleora_ctx* ctx, void* out, cleora_dtype dtype, int out_on_device);
/* Replaces the current embeddings (resume from a checkpoint); converts from `dtype` to
 * the storage type given to init.  The iteration counter is reset to `iteration`. */
int cleora_set_embeddings(cleora_ctx* ctx, const void* in, cleora_dtype dtype,
                          int in_on_device, int iteration);

/* ---------------------------------------------------------------------------------------
 * Kernel schedule (autotuner hooks and counters)
 * ------------------------------------------------------------------------------------- */

typedef enum {
    CLEORA_OPT_VEC_BYTES = 0,    /* 16 or 8: bytes per gathered vector; 0 = automatic
                                    (16 when a row holds at least 32 such vectors, else 8) */
    CLEORA_OPT_ROW_MODE = 1,     /* 0 automatic, 1 = lane groups split one row's entries,
                                    2 = each lane group owns its own rows                 */
    CLEORA_OPT_SPLIT_LEN = 2,    /* rows longer than this are split across warps (>= 256)  */
    CLEORA_OPT_TASK_NNZ = 3,     /* entries per scheduled task (>= 64)                      */
    CLEORA_OPT_BLOCKS_PER_SM = 4, /* persistent CTAs per SM; 0 = occupancy limit           */
    CLEORA_OPT_HOT_BYTES = 5,    /* L2 bytes kept for the rows most entries point at:
                                    cleora_init moves the entries that point at them to the
                                    front of their rows (gathered with an evict_last
                                    policy, the rest evict_first) when T is larger than
                                    twice this; 0 = 72 MiB, 1 = off.  Only the summation
                                    order changes; cleora_get_csr still returns each row
                                    in ascending column order                              */
    CLEORA_OPT_ID_SLOTS = 6,     /* slots of the hash set that collects the distinct ids in
                                    cleora_graph_build; 0 = four times a HyperLogLog
                                    estimate of their number.  A set that fills up is
                                    rebuilt with 4 x num_edges slots, so any value gives the
                                    same graph                                             */
    CLEORA_OPT_STAGING = 7,      /* how gathered rows reach the sums: 0 or 1 = registers,
                                    2 = a shared-memory ring filled by one bulk copy per
                                    gathered row, 3 = the same ring filled by TMA tensor
                                    gathers of 4 rows (set before cleora_init, which builds the
                                    tensor maps) (rows of 32 x 8 or 32 x 16 bytes:
                                    FP32 d = 64 or 128, BF16 d = 128 or 256; other shapes use
                                    registers).  With the ring, rows keep ascending column
                                    order and hot entries are marked in a bitmap instead of
                                    moved to the front.  Results differ from the register
                                    path only in summation order                           */
    CLEORA_OPT_RING_STAGES = 8,  /* stages of the ring (windows of 32 entries): 2, 3 or 4;
                                    0 = 3                                                  */
    CLEORA_OPT_TEST_RING_WAIT = 9, /* test hook, 0 or 1: in the next ring launches, the first
                                    window of every warp waits for one row more than it
                                    copies.  Each ring wait is bounded (0.5 s): the wait runs
                                    out, the kernel raises its error flag (cleora_sync then
                                    returns CLEORA_ERR_DEVICE), waits again (bounded) and
                                    returns, leaving the context usable.  The results of
                                    that launch are not valid                              */
    CLEORA_OPT_CHUNK_BYTES = 10  /* device bytes one chunk of cleora_chunked_embed may use
                                    when the library picks the chunks; 0 = 80% of the free
                                    device memory at the call                              */
} cleora_option;
int cleora_set_option(cleora_ctx* ctx, cleora_option opt, int64_t value);
int cleora_get_option(const cleora_ctx* ctx, cleora_option opt, int64_t* value);
/* Number of this library's kernel launches on the context so far. */
int cleora_launch_count(const cleora_ctx* ctx, int64_t* launches);
/* Entries that the last cleora_init placed in the hot front part of their rows (see
 * CLEORA_OPT_HOT_BYTES); 0 when the rows are not partitioned.  ERR_STATE before a graph. */
int cleora_hot_entries(const cleora_ctx* ctx, int64_t* hot_entries);

/* ---------------------------------------------------------------------------------------
 * Inductivity and additivity (Sec. 1, "Additivity" / "Inductivity"; Sec. 3.2, end;
 * Algorithm 1, chunks and merge)
 * ------------------------------------------------------------------------------------- */

/* Rows for nodes added after the embedding (Sec. 1 "Inductivity"; Sec. 3.2: a new node's
 * embedding is the weighted average of its neighbours' representations, ideally those of
 * iteration I-1).  Edge k links new node new_ids[k] to existing node nbr_ids[k] with weight
 * weights[k] (NULL: 1).  With the builder's rules (duplicates merged, e_ub summed in FP64,
 * M_ub = e_ub / deg_u) each new node u gets rownorm(sum_b M_ub T[b]) over the context's
 * current embeddings T, computed by the propagation kernel; the context is not modified.
 * Edges to ids that are not nodes of the graph are dropped (*num_dropped counts them); a new
 * node with no kept edge gets no row.  Outputs: out_ids[*num_new] ascending and out
 * (*num_new x d FP32, out_rows capacity; NULL to skip).  Errors: CLEORA_ERR_STATE without
 * embeddings, CLEORA_ERR_INVALID_ARG for bad weights or too small an output. */
int cleora_inductive(cleora_ctx* ctx, const uint64_t* new_ids, const uint64_t* nbr_ids,
                     const float* weights, int64_t num_edges, int inputs_on_device,
                     uint64_t* out_ids, float* out, int64_t out_rows, int64_t* num_new,
                     int64_t* num_dropped, int out_on_device);

/* Algorithm 1 with Q = num_chunks edge chunks: edges chunk_offsets[q] .. chunk_offsets[q+1]-1
 * (host array of Q+1 offsets, chunk_offsets[0] = 0) form chunk q.  Each chunk is embedded on
 * its own (its own M_q and T_0 from the same id hash, `iters` iterations, `storage`) and
 * the results are merged: T_v = sum_q w_qv T^q_v with w_qv = occ_q(v) / sum_k occ_k(v), where
 * occ_q(v) counts the endpoints of chunk q's edges equal to v (the paper's node weight, read
 * as an occurrence share; a self-loop counts twice; counts are exact 64-bit integers and the
 * ratio is rounded once to FP32).  Q = 1 is the plain method.
 * num_chunks = 0: the library picks the chunks (the graph may be larger than device memory):
 * chunk_offsets[0] holds the number of edges E, and Q is the fewest chunks of equal size
 * (edges floor(E q / Q) .. floor(E (q+1) / Q) - 1) whose estimated device peak, next to
 * 28 bytes per node, fits CLEORA_OPT_CHUNK_BYTES (0: 80% of the free device memory).
 * Out of core: edges given in host memory are uploaded one chunk at a time; a first pass
 * over the chunks collects the node ids and occurrence counts, a second embeds each chunk and
 * adds its weighted rows straight into `out` -- device memory, or host memory that the call
 * maps into the device (pinned for the duration of the call when it is not already).  So the
 * device holds one chunk's graph and embeddings plus the ids and counts, never the whole edge
 * list or an n x d accumulator.  cleora_chunked_info reports Q and the device peak.
 * Outputs: out_ids[*num_nodes] (all nodes, ascending id) and out (FP32, out_rows capacity).
 * The context's graph and embeddings are replaced by the last chunk's. */
int cleora_chunked_embed(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst,
                         const float* weights, const int64_t* chunk_offsets, int num_chunks,
                         int directed, int d, int iters, uint64_t seed, cleora_dtype storage,
                         int inputs_on_device, uint64_t* out_ids, float* out, int64_t out_rows,
                         int64_t* num_nodes, int out_on_device);
/* Chunks of the last cleora_chunked_embed call and the high-water mark of the device memory
 * the library held during it (bytes, from the context's pool). */
int cleora_chunked_info(const cleora_ctx* ctx, int* chunks, int64_t* peak_device_bytes);

/* ---------------------------------------------------------------------------------------
 * Identifiers and hypergraphs (Sec. 4.3: identifiers hashed with xxhash into a small
 * fixed-width format; Sec. 3.2 "Hypergraph Expansion": clique and star expansion)
 * ------------------------------------------------------------------------------------- */

/* XXH64 (the xxHash specification, 64-bit variant, little-endian lanes) of every string
 * bytes[offsets[i] .. offsets[i+1]), i < count, with `seed`, into out[count]: the uint64 ids the
 * graph calls take.  offsets[0] must be 0.  bytes/offsets are host (inputs_on_device == 0) or
 * device arrays, out host or device; the call returns when out is written.  Distinct strings
 * can share a hash (about count^2 / 2^65 expected collisions), as in the paper's design. */
int cleora_hash_ids(cleora_ctx* ctx, const uint8_t* bytes, const int64_t* offsets, int64_t count,
                    uint64_t seed, uint64_t* out, int inputs_on_device, int out_on_device);

typedef enum { CLEORA_EXPAND_CLIQUE = 0, CLEORA_EXPAND_STAR = 1 } cleora_expansion;

/* Expands a hypergraph into undirected edges.  Hyperedge h (h < num_hyperedges) holds the ids
 * members[hoff[h] .. hoff[h+1]) (hoff[0] = 0, non-decreasing); repeated members count once, so
 * its distinct members in ascending id order u_0 < ... < u_{k-1} give
 *   CLEORA_EXPAND_CLIQUE: the edges (u_i, u_j), i < j, in lexicographic (i, j) order --
 *                         k(k-1)/2 edges (a hyperedge of one member gives none);
 *   CLEORA_EXPAND_STAR:   the edges (s_h, u_i), i = 0..k-1 -- k edges, s_h the hyperedge's star
 *                         node: star_ids[h], or when star_ids is NULL the splitmix64 output
 *                         function of h ^ 0x5354415253544152 (ids the caller should keep
 *                         apart from its members').
 * Hyperedges keep their order.  *num_edges gets the edge count; src_out / dst_out (capacity
 * edges each; NULL to only count) get the edges.  Inputs host or device (inputs_on_device),
 * outputs host or device (out_on_device).  CLEORA_ERR_INVALID_ARG when the edges do not fit. */
int cleora_expand_hypergraph(cleora_ctx* ctx, const uint64_t* members, const int64_t* hoff,
                             int64_t num_hyperedges, int mode, const uint64_t* star_ids,
                             int inputs_on_device, uint64_t* src_out, uint64_t* dst_out,
                             int64_t capacity, int64_t* num_edges, int out_on_device);
/* The same expansion kept on the device and built as the context's undirected graph, exactly
 * as cleora_graph_build would build the expanded edge list (unit weights). */
int cleora_hypergraph_build(cleora_ctx* ctx, const uint64_t* members, const int64_t* hoff,
                            int64_t num_hyperedges, int mode, const uint64_t* star_ids,
                            int inputs_on_device, int64_t* num_edges);

/* ---------------------------------------------------------------------------------------
 * Batched small graphs: many independent graphs in one persistent launch per iteration
 * step (Sec. 4.2-4.3: each relation pair gets its own M, trained independently; the paper
 * runs them in separate threads)
 * ------------------------------------------------------------------------------------- */

typedef struct {
    const uint64_t* src;      /* num_edges ids (host or device, as the batch flag says)     */
    const uint64_t* dst;
    const float* weights;     /* NULL: unit weights                                         */
    int64_t num_edges;        /* >= 0                                                       */
    int directed;
    int d;                    /* multiple of 8 in [8, 1024]                                 */
    int iters;                /* >= 0 iterations for this graph                             */
    uint64_t seed;            /* init seed (T_0 as in cleora_init)                          */
    cleora_dtype storage;     /* FP32 or BF16 embeddings                                    */
} cleora_graph_desc;

typedef struct cleora_batch cleora_batch;

/* Builds every graph exactly as cleora_graph_build would, packs them into one multi-graph
 * CSR (per-graph node, entry and embedding offsets), picks each graph's kernel schedule
 * (autotune != 0: the fastest of the candidate vector widths and row modes, timed per
 * (d, storage) class on a sample of its graphs; 0: the single-graph defaults) and captures
 * init + every iteration step + the FP32 output pass in one CUDA graph on `cuda_stream`
 * (NULL: a stream the batch creates).  Graph g's result equals, bit for bit, a single-graph
 * context given the same schedule options (cleora_batch_schedule reports them).
 * Errors: CLEORA_ERR_INVALID_ARG (a bad descriptor; *out stays NULL), CLEORA_ERR_OOM. */
int cleora_batch_create(cleora_batch** out, int device, void* cuda_stream,
                        const cleora_graph_desc* graphs, int count, int inputs_on_device,
                        int autotune);
void cleora_batch_destroy(cleora_batch* b);
const char* cleora_batch_last_error(const cleora_batch* b);
/* Totals: nodes, CSR entries, FP32 output elements (sum of n_g * d_g), largest iters. */
int cleora_batch_totals(const cleora_batch* b, int64_t* nodes, int64_t* nnz,
                        int64_t* out_elems, int* max_iters);
/* Graph g: its node count, entries, and the element offset of its n_g x d_g FP32 rows in
 * the packed output. */
int cleora_batch_graph_info(const cleora_batch* b, int g, int64_t* n, int64_t* nnz,
                            int64_t* out_offset);
/* Schedule chosen for graph g: gather bytes, row mode, split length, task size. */
int cleora_batch_schedule(const cleora_batch* b, int g, int64_t* vec_bytes, int64_t* row_mode,
                          int64_t* split_len, int64_t* task_nnz);
/* ids[n_g] of graph g, ascending. */
int cleora_batch_node_ids(cleora_batch* b, int g, uint64_t* out, int out_on_device);
/* Replays the captured graph: T_0, iters_g iterations of every graph, then all results
 * packed as FP32 into out[out_elems] (host or device).  Returns when `out` is written. */
int cleora_batch_run(cleora_batch* b, float* out, int out_on_device);
/* Kernel launches of the last run (the captured graph's kernel nodes). */
int cleora_batch_launches(const cleora_batch* b, int64_t* launches);

/* ---------------------------------------------------------------------------------------
 * Serving: a continuous-batching request loop for embedding jobs of different sizes
 * (the whole method -- build, init, I iterations -- per job; Sec. 4.5's linear memory model
 * is what admission budgets against)
 * ------------------------------------------------------------------------------------- */

typedef struct cleora_server cleora_server;

typedef struct {
    int device;
    int64_t hbm_budget_bytes;  /* device bytes the running jobs may hold together;
                                  0: 80% of the free memory at creation                   */
    int max_slots;             /* jobs resident and running at once (one stream each); 0: 4 */
    int queue_capacity;        /* waiting jobs accepted; 0: unbounded                       */
    int inject_alloc_failure_every; /* test hook: every k-th admitted job gets a failing
                                       allocation (reported as CLEORA_ERR_OOM); 0: off      */
    int short_slots;           /* further slots (0..64) that take short jobs only, from a
                                  reserve of their own: min(2 GiB per slot, 1/8 of the
                                  budget), set aside from the budget; 0: none               */
    double short_job_seconds;  /* a job is short when its estimated service time is at most
                                  this; short jobs run on a high-priority stream in any
                                  slot; 0: 0.02 s                                          */
} cleora_server_config;

typedef struct {
    const uint64_t* src;   /* host arrays; they must stay valid until the job is done       */
    const uint64_t* dst;
    const float* weights;  /* NULL: unit weights                                            */
    int64_t num_edges;
    int directed;
    int d;                 /* multiple of 8 in [8, 1024]                                    */
    int iters;             /* >= 0                                                          */
    uint64_t seed;
    cleora_dtype storage;
    float* out;            /* host, out_rows x d FP32 (rows in ascending id order); NULL:
                              the result is computed and dropped                            */
    int64_t out_rows;      /* capacity of out in rows (must be >= the node count)           */
    int64_t nodes_hint;    /* node count if known (tightens the memory estimate); 0: <= 2E */
} cleora_job;

typedef struct {
    int status;            /* the job's own status: CLEORA_OK or the error it ended with    */
    int slot;              /* slot that ran it (-1 if it never ran)                         */
    int64_t n, nnz;
    int64_t bytes_reserved;/* the admission estimate it was charged                         */
    double t_submit, t_admit, t_done;  /* seconds on the server's monotonic clock           */
    double t_built, t_inited;  /* when its graph build and its init returned (0 if not reached) */
} cleora_result;

/* Starts the server: max_slots worker threads, each with its own context and stream, on
 * `device`.  Admission: a waiting job starts when a slot is free and its estimated peak
 * device bytes (cleora_serve_estimate) fit in the budget next to the running jobs.  Among
 * the jobs that fit, the one with the earliest virtual finish time starts first: arrival time
 * plus an estimated service time (a cost model of its host transfers, graph build and
 * gathered bytes), so short jobs go ahead of long ones while a job is only passed by jobs
 * that arrived within its own service estimate after it.  A job passed over 8 times because
 * it did not fit stops later jobs from passing it.  A short_slots slot takes the earliest short
 * job that fits its reserve.  Jobs on different slots overlap on the GPU.  The slots allocate
 * from one device memory pool that keeps what finished jobs freed for the next ones (it is
 * returned to the driver when an allocation would otherwise fail, and at destroy), so the
 * budget bounds what running jobs hold.  cleora_serve_stats reports the general budget and
 * the short reserve together. */
int cleora_serve_create(cleora_server** out, const cleora_server_config* cfg);
/* Queues a job; *job_id identifies it.  CLEORA_ERR_REJECTED: its estimate exceeds the whole
 * budget, or the queue is full.  CLEORA_ERR_INVALID_ARG: a malformed job. */
int cleora_serve_submit(cleora_server* s, const cleora_job* job, uint64_t* job_id);
/* Waits up to timeout_ms (< 0: no limit) for the job; on success fills *result and forgets
 * the job.  CLEORA_ERR_TIMEOUT: not done yet (poll again).  CLEORA_ERR_INVALID_ARG: unknown
 * id (or already collected). */
int cleora_serve_poll(cleora_server* s, uint64_t job_id, int timeout_ms, cleora_result* result);
/* Waits up to timeout_ms (< 0: no limit) for the next finished job not yet collected, in
 * completion order; fills *job_id and *result and forgets the job.  CLEORA_ERR_TIMEOUT: none
 * finished in time. */
int cleora_serve_next(cleora_server* s, int timeout_ms, uint64_t* job_id, cleora_result* result);
/* Cancels a job that has not started (its result status becomes CLEORA_ERR_CANCELLED);
 * CLEORA_ERR_STATE if it is already running or done. */
int cleora_serve_cancel(cleora_server* s, uint64_t job_id);
/* Estimated peak device bytes of a job (graph build, then CSR + two embedding buffers). */
int64_t cleora_serve_estimate(const cleora_job* job);
/* Seconds on the server's clock (the clock of cleora_result's timestamps). */
double cleora_serve_now(const cleora_server* s);
int cleora_serve_stats(const cleora_server* s, int* queued, int* running, int64_t* bytes_reserved,
                       int64_t* completed, int64_t* budget);
/* Stops accepting jobs, cancels waiting ones, waits for running ones, frees everything. */
void cleora_serve_destroy(cleora_server* s);

/* ---------------------------------------------------------------------------------------
 * Allocation-free propagation step (this entry point has no counterpart in the paper)
 * ------------------------------------------------------------------------------------- */

/* One iteration T_out = rownorm_L2(M T_in) that never allocates device memory: no
 * cudaMalloc/cudaFree, no pool, no library routine that allocates.  It is meant for callers
 * that may not let this library take device memory on its own: a framework whose
 * allocator owns all of HBM and hands out fixed budgets, a latency-critical loop that
 * cannot afford cudaMalloc/cudaFree (which can synchronise the device), or a job that must
 * not fail with out-of-memory halfway.
 *
 * Inputs, all device pointers owned by the caller: the CSR of M (rowptr[n+1] int64,
 * col[nnz] int32, and val[nnz] FP32 M_ab, or val == NULL for unit weights, where rows are
 * summed and the normalisation removes the common 1/deg factor), T_in (n x d, storage type)
 * and the output T_out (n x d, same type).  The CSR must be well formed: rowptr[0] = 0,
 * non-decreasing, rowptr[n] = nnz (entries past nnz are not read; a row reaching past it is
 * wrong).  Alignment: T_in and T_out on 16-byte boundaries (the kernel moves 16-byte
 * vectors), rowptr on 8, col and val on 4; T_in and T_out must not overlap.  A call that
 * breaks either rule returns CLEORA_ERR_INVALID_ARG before launching anything.  Results agree with
 * cleora_propagate within the parity tolerances (1e-5 FP32, 2e-2 BF16); the summation order
 * can differ because rows longer than split_len are split differently.
 *
 * Scratch: one file-scope device array of 8,618,240 bytes (cleora_noalloc_limits reports
 * it), held by every GPU that loads the library until the process exits.  It carries the
 * work counter, the table of split rows and up to min(16384, 8 MiB / (4 d)) FP32 partial
 * sums of split rows.  split_len (0 = the smallest allowed, at least 256) must be at least
 * ceil(2 * nnz / that chunk limit), else the call returns CLEORA_ERR_INVALID_ARG before
 * launching anything; d must be a multiple of 8 in [8, 1024].
 *
 * Every call shares the array and keeps the previous call's contents (the counters are
 * cleared at the start of each call), so calls that overlap on the GPU -- on different
 * streams, or from different host threads -- race and give wrong results.  Work is queued
 * on `cuda_stream` (NULL: the legacy default stream) on the current device; the call returns
 * without waiting.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and caches it; make that first call
 * before any stream capture.  Out-of-range column indices are skipped, not reported. */
int cleora_propagate_noalloc(const int64_t* rowptr, const int32_t* col, const float* val,
                             int64_t n, int64_t nnz, const void* T_in, void* T_out, int d,
                             cleora_dtype storage, int64_t split_len, void* cuda_stream);
/* Scratch size in bytes and the largest number of split-row chunks for dimension d. */
int cleora_noalloc_limits(int d, int64_t* scratch_bytes, int64_t* max_split_chunks);

#ifdef __cplusplus
}
#endif
#endif /* CLEORA_H */
