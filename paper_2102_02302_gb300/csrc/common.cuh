// Internal declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>

#include "cleora.h"

namespace cleora {

// A scheduled unit of propagation work (16 bytes).
//   normal task : rows [a, b) processed whole;              c = -1, k = 0
//   split chunk : entries [c * len, (c+1) * len) of row a;  b = split-row index, k = chunks
struct Task {
    int32_t a, b, c, k;
};

// Work list of one graph for one schedule (split length and task size).
struct Plan {
    bool valid = false;
    int64_t split_len = 0, task_nnz = 0;
    int64_t ntasks = 0;        // split chunks first, then normal tasks
    int64_t nsplit_rows = 0;   // rows split across warps
    int64_t nsplit_chunks = 0; // = number of partial-sum slots
    Task* tasks = nullptr;
    int64_t* split_base = nullptr;  // per split row: its first partial slot
    int32_t* split_count = nullptr; // per split row: arrival counter, reset by the last warp
    unsigned long long* counter = nullptr;  // dynamic task counter (zeroed per launch)
    float* partials = nullptr;      // nsplit_chunks x d FP32 partial sums
    int64_t partials_d = 0;
};

struct Graph {
    bool built = false;
    int64_t n = 0, nnz = 0, max_row_len = 0;
    bool has_val = false;
    bool directed = false;
    // Rows partitioned hot-first (entries pointing at the hottest rows of T first, each part in
    // ascending column order): hot_cnt != NULL, for this row size and hot-row budget.
    int64_t part_row_bytes = 0;
    int64_t part_budget = 0;
    int32_t* hot_cnt = nullptr;  // n: hot entries at the front of each row
    int64_t hot_entries = 0;     // their total
    // Shared-memory ring kernel: rows keep ascending order and a bitmap marks the entries that
    // point at hot rows (bit k & 31 of word k >> 5); hot_bits != NULL instead of hot_cnt.
    uint32_t* hot_bits = nullptr;
    uint64_t* ids = nullptr;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;      // nnz, only when has_val
    float* inv_deg = nullptr;  // n
    double* deg = nullptr;     // n
};

// Kernel shape for one (d, storage) pair.
struct Shape {
    int vec = 16;   // bytes per gathered vector
    int G = 32;     // lanes that cover one row of T
    int cpl = 1;    // vectors per lane per row
    int mode = 1;   // 1: lane groups split a row's entries, 2: each group owns rows
    int chunks = 0; // vectors per row
};

enum { OPT_COUNT = 11 };

constexpr int64_t DEFAULT_SPLIT_LEN = 8192;  // rows longer than this are split across warps
constexpr int64_t DEFAULT_TASK_NNZ = 4096;   // entries per row-run task
constexpr int64_t DEFAULT_HOT_BYTES = (int64_t)72 << 20;  // L2 share kept for hot rows
constexpr size_t HOST_STAGE_BYTES = (size_t)128 << 10;     // pinned staging for small copies

}  // namespace cleora

struct cleora_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaMemPool_t pool = nullptr;
    bool own_pool = true;  // false: a pool shared with other contexts (serving slots)
    int num_sms = 0;
    std::string err;

    cleora::Graph g;
    cleora::Plan plan;

    bool inited = false;
    int d = 0;
    cleora_dtype dtype = CLEORA_F32;
    void* T[2] = {nullptr, nullptr};
    int cur = 0;
    int iteration = 0;

    int64_t opt[cleora::OPT_COUNT] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    CUtensorMap tmap[2];            // ring with 4-row tensor gathers: maps over T[0], T[1]
    bool tmap_ready = false;
    int chunks_used = 0;            // cleora_chunked_embed: chunks of the last call
    int64_t chunk_peak_bytes = 0;   // ... and the pool's high-water mark during it
    int* err_flag = nullptr;  // device int, raised by kernels
    unsigned char* host_stage = nullptr;      // pinned and mapped, cleora::HOST_STAGE_BYTES
    unsigned char* host_stage_dev = nullptr;  // ... its device address (small read-backs)
    int64_t launches = 0;
    int64_t inject_alloc_fail = -1;  // test hook: >= 0 counts down, the allocation at 0 fails
};

namespace cleora {

// ---- error plumbing ------------------------------------------------------------------
int fail(cleora_ctx* ctx, int status, const char* fmt, ...);
int cuda_fail(cleora_ctx* ctx, cudaError_t e, const char* what, const char* file, int line);

#define CL_CUDA(ctx, call)                                                          \
    do {                                                                            \
        cudaError_t e_ = (call);                                                    \
        if (e_ != cudaSuccess) return ::cleora::cuda_fail(ctx, e_, #call, __FILE__, __LINE__); \
    } while (0)

#define CL_LAUNCHED(ctx)                                                            \
    do {                                                                            \
        (ctx)->launches += 1;                                                       \
        cudaError_t e_ = cudaGetLastError();                                        \
        if (e_ != cudaSuccess) return ::cleora::cuda_fail(ctx, e_, "kernel launch", __FILE__, __LINE__); \
    } while (0)

// Small copies between host and device.  A copy to or from pageable host memory is staged
// by the driver and waits behind large copies that other streams have in flight: on a GB300 an
// 8-byte pageable read-back waited up to 90 ms behind a 16 GiB device-to-host copy on another
// stream, against 0.015 ms through pinned memory or a kernel.  A pinned copy still needs a copy
// engine, which concurrent serving jobs can keep busy with large downloads, and a kernel needs
// a free CTA slot, which other streams' persistent kernels can hold.  So a read-back between a
// context's own kernels (the graph build's counts and flags) is a kernel that writes the bytes
// into the context's mapped pinned staging buffer (`by_kernel`), and one after a download (the
// error flag at a synchronize) is a copy into the same buffer; either is followed by a
// synchronize of `s`, as a pageable copy would be.  Small values go to the device as kernel
// arguments.
cudaError_t read_back(cleora_ctx* ctx, void* host, const void* dev, size_t bytes, cudaStream_t s,
                      bool by_kernel = true);
cudaError_t put_bytes(cleora_ctx* ctx, void* dev, const void* host, size_t bytes, cudaStream_t s);  // bytes <= 32

#define CL_TRY(x)                      \
    do {                               \
        int s_ = (x);                  \
        if (s_ != CLEORA_OK) return s_; \
    } while (0)

// ---- stream-ordered device memory from the context's pool ----------------------------
int dalloc_bytes(cleora_ctx* ctx, void** p, size_t bytes);
// A context on `device`; with `shared_pool` its allocations come from that pool, which the
// caller owns and destroys after the context.
int ctx_create(cleora_ctx** out, int device, void* cuda_stream, cudaMemPool_t shared_pool);
template <class T>
inline int dalloc(cleora_ctx* ctx, T** p, size_t count) {
    return dalloc_bytes(ctx, reinterpret_cast<void**>(p), count * sizeof(T));
}
void dfree(cleora_ctx* ctx, void* p);
template <class T>
inline void dfree_null(cleora_ctx* ctx, T*& p) {
    dfree(ctx, p);
    p = nullptr;
}

// splitmix64 output function (Steele, Lea & Flood 2014), used by the T_0 hash.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// T_0 value of element j of a row whose prefix is mix(mix(seed) ^ id): 2 (h >> 40) 2^-24 - 1,
// with every step exact in FP32.
__device__ __forceinline__ float init_value(uint64_t prefix, uint32_t j) {
    const uint64_t h = mix64(prefix ^ (uint64_t)j);
    return (float)(uint32_t)(h >> 40) * 0x1p-23f - 1.0f;
}

inline unsigned grid_for(int64_t items, int threads, int num_sms) {
    int64_t b = (items + threads - 1) / threads;
    int64_t cap = (int64_t)num_sms * 32;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

// Makes a device current for the duration of a call, then restores the caller's device.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) { ok = false; return; }
        if (prev != dev && cudaSetDevice(dev) != cudaSuccess) ok = false;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---- parts implemented in the other translation units --------------------------------
int graph_build_impl(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst,
                     const float* w, int64_t E, int directed);
void graph_release(cleora_ctx* ctx);
// CSR of M from entry keys (row << bits | col; `invalid` marks dropped entries) and optional
// FP32 weights (vbuf_a/vbuf_b NULL: unit).  Sorts stably, merges duplicates, fills g's col,
// rowptr, deg, inv_deg, val, nnz, max_row_len and has_val.  The key buffers (kbuf_words
// words each) and weight buffers are consumed as scratch.
int csr_from_entries(cleora_ctx* ctx, uint64_t* kbuf_a, uint64_t* kbuf_b, float* vbuf_a, float* vbuf_b,
                     int64_t m, int64_t kbuf_words, int64_t n, int bits, uint64_t invalid, Graph& g);
// The same for an undirected graph from one (lo, hi) key per edge (lo <= hi, E < 2^31).
int csr_undirected(cleora_ctx* ctx, uint64_t* kbuf_a, uint64_t* kbuf_b, float* vbuf_a, float* vbuf_b, int64_t E,
                   int64_t kbuf_words, int64_t n, int bits, Graph& g);
int check_weights(cleora_ctx* ctx, const float* w, int64_t E);  // finite and > 0
int bit_width_of(int64_t v);
int sort_unique_ids(cleora_ctx* ctx, const uint64_t* keys, int64_t count, uint64_t** ids_out, int64_t* n_out);
int rank_ids(cleora_ctx* ctx, const uint64_t* ids, int64_t n, const uint64_t* x, int64_t count,
             int32_t* rank_out);  // rank of each x among ids, -1 when absent
int csr_values_out(cleora_ctx* ctx, float* val_dev);  // M_ab per entry as FP32
int values_out_sorted(cleora_ctx* ctx, float* val_dev);  // weighted values, ascending column order

void ctx_release_all(cleora_ctx* ctx);  // graph, plan and embeddings of a context

int init_impl(cleora_ctx* ctx, uint64_t seed);
int convert_impl(cleora_ctx* ctx, const void* src, cleora_dtype sdt, void* dst, cleora_dtype ddt,
                 int64_t count);

Shape choose_shape(const cleora_ctx* ctx, int d, cleora_dtype dt);
Shape shape_for(int d, cleora_dtype dt, int64_t vec_opt, int64_t mode_opt);
int plan_build(cleora_ctx* ctx, int64_t split_len, int64_t task_nnz);
void plan_release(cleora_ctx* ctx);
int plan_ensure(cleora_ctx* ctx);
int propagate_step(cleora_ctx* ctx, const void* Tin, void* Tout);
// Shapes the shared-memory ring kernel covers: a full warp, one vector per lane, rows of
// 32 x 8 or 32 x 16 bytes.
inline bool ring_shape(const Shape& sh) { return sh.G == 32 && sh.cpl == 1 && sh.chunks == 32; }
bool use_ring(const cleora_ctx* ctx);          // the current (d, storage, options) runs the ring
int ring_tensor_maps(cleora_ctx* ctx);         // tensor maps over T for the 4-row gathers (init)
constexpr int DEFAULT_RING_STAGES = 3;
int hot_partition(cleora_ctx* ctx);            // partition rows hot-first (after init)
int hot_restore(cleora_ctx* ctx);              // back to ascending column order
int col_out(cleora_ctx* ctx, int32_t* col_dev); // column indices in ascending order per row

}  // namespace cleora
