// Graph build on the GPU: node ids and the CSR of M = D^-1 A
// (arXiv 2102.02302, Sec. 3.2 "Embedding": M_ab = e_ab / deg(v_a), e_ab the number of
// edges a->b or the sum of their weights; Sec. 4.5: undirected edges count both ways).
//
// Steps (all on the context's stream; sort, unique and compaction use CUB):
//   1. ids   = sort-unique(src ++ dst)                 (node index = rank of the id)
//   2. entry keys (a << bits) | b, one per edge (two for an undirected non-loop edge,
//      interleaved 2e, 2e+1 so that a stable sort keeps duplicates in edge order)
//   3. stable radix sort of the keys (weights carried along when weighted)
//   4. runs of equal keys -> col, e_ab (count, or FP64 sum in edge order)
//   5. rowptr from the sorted rows; deg_a = FP64 sum of e_ab in ascending col
//   6. val = fp32(e_ab / deg_a) when needed; inv_deg = 1.0f / fp32(deg_a)
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>
#include <thrust/iterator/counting_iterator.h>

#include "common.cuh"

namespace cleora {
namespace {

__global__ void k_check_weights(const float* w, int64_t E, int* bad) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        float x = w[i];
        if (!(isfinite(x) && x > 0.0f)) atomicOr(bad, 1);
    }
}

constexpr int SAMPLE = 64;  // ids per segment of the two-level lookup

// Every SAMPLE-th id: a small table that stays in L2 and narrows each search to one segment.
__global__ void k_sample_ids(const uint64_t* ids, int64_t n, uint64_t* sample, int64_t ns) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns;
         i += (int64_t)gridDim.x * blockDim.x)
        sample[i] = ids[i * SAMPLE];
}

// Rank of x among the sorted ids (x is one of them): search the sample, then its segment.
__device__ __forceinline__ int64_t rank_of(const uint64_t* ids, int64_t n, const uint64_t* sample,
                                           int64_t ns, uint64_t x) {
    int64_t lo = 0, hi = ns;  // last sample entry <= x
    while (hi - lo > 1) {
        const int64_t mid = (lo + hi) >> 1;
        if (sample[mid] <= x) lo = mid; else hi = mid;
    }
    int64_t a = lo * SAMPLE, b = min(n, a + SAMPLE);  // first position with ids[pos] >= x
    while (a < b) {
        const int64_t mid = (a + b) >> 1;
        if (ids[mid] < x) a = mid + 1; else b = mid;
    }
    return a;
}

__global__ void k_entries(const uint64_t* src, const uint64_t* dst, const float* w, int64_t E,
                          int directed, const uint64_t* ids, int64_t n, const uint64_t* sample,
                          int64_t ns, int bits, uint64_t invalid, uint64_t* keys, float* vals) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t a = (uint64_t)rank_of(ids, n, sample, ns, src[e]);
        const uint64_t b = (uint64_t)rank_of(ids, n, sample, ns, dst[e]);
        if (directed) {
            keys[e] = (a << bits) | b;
            if (vals) vals[e] = w[e];
        } else {
            keys[2 * e] = (a << bits) | b;
            keys[2 * e + 1] = (a == b) ? invalid : ((b << bits) | a);
            if (vals) {
                vals[2 * e] = w[e];
                vals[2 * e + 1] = w[e];
            }
        }
    }
}

__global__ void k_heads(const uint64_t* keys, int64_t m, uint64_t invalid, uint8_t* head) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[i];
        head[i] = (k != invalid && (i == 0 || keys[i - 1] != k)) ? 1 : 0;
    }
}

// Number of valid (non-sentinel) keys: the sentinel sorts last.
__global__ void k_count_valid(const uint64_t* keys, int64_t m, uint64_t invalid, int64_t* out) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (keys[mid] < invalid) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

// Per unique entry k: column, row, and e_ab (count or FP64 weight sum in edge order).
__global__ void k_runs(const uint64_t* keys, const float* vals, const int64_t* start, int64_t nnz,
                       const int64_t* m_valid, int bits, int32_t* col, int32_t* row, double* e,
                       int* not_unit) {
    const uint64_t mask = (1ull << bits) - 1ull;
    const int64_t mv = *m_valid;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t s = start[k];
        const int64_t t = (k + 1 < nnz) ? start[k + 1] : mv;
        const uint64_t key = keys[s];
        col[k] = (int32_t)(key & mask);
        row[k] = (int32_t)(key >> bits);
        double acc;
        if (vals) {
            acc = 0.0;
            for (int64_t i = s; i < t; ++i) acc = __dadd_rn(acc, (double)vals[i]);
        } else {
            acc = (double)(t - s);
            if (t - s != 1) atomicOr(not_unit, 1);
        }
        e[k] = acc;
    }
}

__global__ void k_rowptr(const int32_t* row, int64_t nnz, int64_t n, int64_t* rowptr) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k <= nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t rp = (k == 0) ? -1 : (int64_t)row[k - 1];
        const int64_t rc = (k == nnz) ? n : (int64_t)row[k];
        for (int64_t r = rp + 1; r <= rc; ++r) rowptr[r] = k;
    }
}

// Unweighted graphs: every e_ab is an integer count, so the row sum is exact in any order;
// one warp per row (integer accumulation) keeps hub rows from becoming stragglers.
__global__ void k_degree_int(const int64_t* rowptr, const double* e, int64_t n, double* deg,
                             float* inv_deg, unsigned long long* max_len) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x / 32);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32; r < n; r += warps) {
        const int64_t b = rowptr[r], t = rowptr[r + 1];
        long long acc = 0;
        for (int64_t k = b + lane; k < t; k += 32) acc += (long long)e[k];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            const double s = (double)acc;
            deg[r] = s;
            inv_deg[r] = s > 0.0 ? __fdiv_rn(1.0f, __double2float_rn(s)) : 0.0f;
            atomicMax(max_len, (unsigned long long)(t - b));
        }
    }
}

// Weighted graphs: deg_a is the FP64 sum of e_ab in ascending column order, one thread per
// row (the order is part of the bit-exact definition of the stored values).
__global__ void k_degree(const int64_t* rowptr, const double* e, int64_t n, double* deg,
                         float* inv_deg, unsigned long long* max_len) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[r], t = rowptr[r + 1];
        double s = 0.0;
        for (int64_t k = b; k < t; ++k) s = __dadd_rn(s, e[k]);
        deg[r] = s;
        inv_deg[r] = s > 0.0 ? __fdiv_rn(1.0f, __double2float_rn(s)) : 0.0f;
        atomicMax(max_len, (unsigned long long)(t - b));
    }
}

__global__ void k_values(const int32_t* row, const double* e, const double* deg, int64_t nnz,
                         float* val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        val[k] = __double2float_rn(__ddiv_rn(e[k], deg[row[k]]));
}

__global__ void k_broadcast_inv(const int64_t* rowptr, const float* inv_deg, int64_t n, float* val) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) val[k] = inv_deg[r];
}

int bit_width(int64_t v) {
    int b = 0;
    while (v > 0) {
        ++b;
        v >>= 1;
    }
    return b;
}

// Scoped device allocation from the context pool.
template <class T>
struct DBuf {
    cleora_ctx* ctx;
    T* p = nullptr;
    explicit DBuf(cleora_ctx* c) : ctx(c) {}
    ~DBuf() { dfree(ctx, p); }
    int alloc(size_t count) { return dalloc(ctx, &p, count ? count : 1); }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
};

}  // namespace

void graph_release(cleora_ctx* ctx) {
    Graph& g = ctx->g;
    dfree_null(ctx, g.ids);
    dfree_null(ctx, g.rowptr);
    dfree_null(ctx, g.col);
    dfree_null(ctx, g.val);
    dfree_null(ctx, g.inv_deg);
    dfree_null(ctx, g.deg);
    dfree_null(ctx, g.hot_cnt);
    g = Graph();
}

int graph_build_impl(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst, const float* w,
                     int64_t E, int directed) {
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    Graph& g = ctx->g;

    DBuf<int64_t> scal(ctx);  // device scalars: [0] count, [1] flag, [2] max_len, [3] m_valid
    CL_TRY(scal.alloc(4));
    CL_CUDA(ctx, cudaMemsetAsync(scal.p, 0, 4 * sizeof(int64_t), s));
    int* d_flag = reinterpret_cast<int*>(scal.p + 1);

    if (w) {
        k_check_weights<<<grid_for(E, 256, sms), 256, 0, s>>>(w, E, d_flag);
        CL_LAUNCHED(ctx);
        int bad = 0;
        CL_CUDA(ctx, cudaMemcpyAsync(&bad, d_flag, sizeof(int), cudaMemcpyDeviceToHost, s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        if (bad) return fail(ctx, CLEORA_ERR_INVALID_ARG, "weights must be finite and > 0");
    }

    const int64_t m = directed ? E : 2 * E;  // entries before dedup
    DBuf<uint64_t> ka(ctx), kb(ctx);
    CL_TRY(ka.alloc((size_t)(2 * E)));
    CL_TRY(kb.alloc((size_t)(2 * E)));

    // 1. ids = sort-unique(src ++ dst)
    CL_CUDA(ctx, cudaMemcpyAsync(ka.p, src, E * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    CL_CUDA(ctx, cudaMemcpyAsync(ka.p + E, dst, E * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    {
        cub::DoubleBuffer<uint64_t> db(ka.p, kb.p);
        size_t tb = 0;
        CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(nullptr, tb, db, 2 * E, 0, 64, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb));
        CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(tmp.p, tb, db, 2 * E, 0, 64, s));
        uint64_t* sorted = db.Current();
        uint64_t* other = db.Alternate();
        size_t tu = 0;
        CL_CUDA(ctx, cub::DeviceSelect::Unique(nullptr, tu, sorted, other, scal.p, 2 * E, s));
        DBuf<unsigned char> tmp2(ctx);
        CL_TRY(tmp2.alloc(tu));
        CL_CUDA(ctx, cub::DeviceSelect::Unique(tmp2.p, tu, sorted, other, scal.p, 2 * E, s));
        int64_t n = 0;
        CL_CUDA(ctx, cudaMemcpyAsync(&n, scal.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        if (n >= ((int64_t)1 << 31))
            return fail(ctx, CLEORA_ERR_INVALID_ARG, "graph has %lld nodes; the limit is 2^31-1",
                        (long long)n);
        g.n = n;
        CL_TRY(dalloc(ctx, &g.ids, (size_t)n));
        CL_CUDA(ctx, cudaMemcpyAsync(g.ids, other, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    }
    const int64_t n = g.n;

    // 2. entry keys (and weights)
    const int bits = bit_width(n);  // n < 2^bits, so the all-ones key is never a real entry
    const uint64_t invalid = (bits * 2 >= 64) ? ~0ull : ((1ull << (2 * bits)) - 1ull);
    DBuf<float> va(ctx), vb(ctx);
    if (w) {
        CL_TRY(va.alloc((size_t)m));
        CL_TRY(vb.alloc((size_t)m));
    }
    const int64_t ns = (n + SAMPLE - 1) / SAMPLE;
    DBuf<uint64_t> sample(ctx);
    CL_TRY(sample.alloc((size_t)ns));
    k_sample_ids<<<grid_for(ns, 256, sms), 256, 0, s>>>(g.ids, n, sample.p, ns);
    CL_LAUNCHED(ctx);
    k_entries<<<grid_for(E, 256, sms), 256, 0, s>>>(src, dst, w, E, directed, g.ids, n, sample.p, ns,
                                                   bits, invalid, ka.p, w ? va.p : nullptr);
    CL_LAUNCHED(ctx);

    g.directed = directed != 0;
    return csr_from_entries(ctx, ka.p, kb.p, w ? va.p : nullptr, w ? vb.p : nullptr, m, 2 * E, n, bits,
                            invalid, g);
}

int csr_from_entries(cleora_ctx* ctx, uint64_t* kbuf_a, uint64_t* kbuf_b, float* vbuf_a, float* vbuf_b,
                     int64_t m, int64_t kbuf_words, int64_t n, int bits, uint64_t invalid, Graph& g) {
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    const bool weighted = vbuf_a != nullptr;
    DBuf<int64_t> scal(ctx);  // device scalars: [0] count, [1] flag, [2] max_len, [3] m_valid
    CL_TRY(scal.alloc(4));
    CL_CUDA(ctx, cudaMemsetAsync(scal.p, 0, 4 * sizeof(int64_t), s));
    int* d_flag = reinterpret_cast<int*>(scal.p + 1);

    // stable sort by (row, col)
    uint64_t* keys = nullptr;
    float* vals = nullptr;
    {
        cub::DoubleBuffer<uint64_t> dk(kbuf_a, kbuf_b);
        size_t tb = 0;
        DBuf<unsigned char> tmp(ctx);
        if (weighted) {
            cub::DoubleBuffer<float> dv(vbuf_a, vbuf_b);
            CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(nullptr, tb, dk, dv, m, 0, 2 * bits, s));
            CL_TRY(tmp.alloc(tb));
            CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(tmp.p, tb, dk, dv, m, 0, 2 * bits, s));
            vals = dv.Current();
        } else {
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(nullptr, tb, dk, m, 0, 2 * bits, s));
            CL_TRY(tmp.alloc(tb));
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(tmp.p, tb, dk, m, 0, 2 * bits, s));
        }
        keys = dk.Current();
    }
    uint64_t* spare = (keys == kbuf_a) ? kbuf_b : kbuf_a;  // free after the sort: reused below

    // runs of equal keys: head flags (m bytes) and run starts (m int64) share the spare key
    // buffer when it is large enough
    uint8_t* head = reinterpret_cast<uint8_t*>(spare);
    int64_t* start = reinterpret_cast<int64_t*>(spare) + (m + 7) / 8;
    DBuf<int64_t> starts_buf(ctx);
    if ((m + 7) / 8 + m > kbuf_words) {
        CL_TRY(starts_buf.alloc((size_t)m));
        start = starts_buf.p;
    }
    k_heads<<<grid_for(m, 256, sms), 256, 0, s>>>(keys, m, invalid, head);
    CL_LAUNCHED(ctx);
    k_count_valid<<<1, 1, 0, s>>>(keys, m, invalid, scal.p + 3);
    CL_LAUNCHED(ctx);
    {
        size_t tb = 0;
        thrust::counting_iterator<int64_t> it(0);
        CL_CUDA(ctx, cub::DeviceSelect::Flagged(nullptr, tb, it, head, start, scal.p, m, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb));
        CL_CUDA(ctx, cub::DeviceSelect::Flagged(tmp.p, tb, it, head, start, scal.p, m, s));
    }
    int64_t nnz = 0;
    CL_CUDA(ctx, cudaMemcpyAsync(&nnz, scal.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    g.nnz = nnz;

    DBuf<int32_t> rows(ctx);
    DBuf<double> e(ctx);
    CL_TRY(rows.alloc((size_t)nnz));
    CL_TRY(e.alloc((size_t)nnz));
    CL_TRY(dalloc(ctx, &g.col, (size_t)(nnz ? nnz : 1)));
    k_runs<<<grid_for(nnz, 256, sms), 256, 0, s>>>(keys, vals, start, nnz, scal.p + 3, bits, g.col,
                                                   rows.p, e.p, d_flag);
    CL_LAUNCHED(ctx);

    // rowptr, degrees
    CL_TRY(dalloc(ctx, &g.rowptr, (size_t)(n + 1)));
    k_rowptr<<<grid_for(nnz + 1, 256, sms), 256, 0, s>>>(rows.p, nnz, n, g.rowptr);
    CL_LAUNCHED(ctx);
    CL_TRY(dalloc(ctx, &g.deg, (size_t)(n ? n : 1)));
    CL_TRY(dalloc(ctx, &g.inv_deg, (size_t)(n ? n : 1)));
    if (weighted)
        k_degree<<<grid_for(n, 256, sms), 256, 0, s>>>(g.rowptr, e.p, n, g.deg, g.inv_deg,
                                                       reinterpret_cast<unsigned long long*>(scal.p + 2));
    else
        k_degree_int<<<grid_for(n * 32, 256, sms), 256, 0, s>>>(g.rowptr, e.p, n, g.deg, g.inv_deg,
                                                                reinterpret_cast<unsigned long long*>(scal.p + 2));
    CL_LAUNCHED(ctx);

    int64_t hv[3] = {0, 0, 0};
    CL_CUDA(ctx, cudaMemcpyAsync(hv, scal.p, 3 * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    const int not_unit = (int)(hv[1] & 0xffffffff);
    g.max_row_len = hv[2];
    g.has_val = weighted || not_unit;

    // stored values
    if (g.has_val) {
        CL_TRY(dalloc(ctx, &g.val, (size_t)(nnz ? nnz : 1)));
        k_values<<<grid_for(nnz, 256, sms), 256, 0, s>>>(rows.p, e.p, g.deg, nnz, g.val);
        CL_LAUNCHED(ctx);
    }
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    g.built = true;
    return CLEORA_OK;
}

namespace {
__global__ void k_rank(const uint64_t* ids, int64_t n, const uint64_t* sample, int64_t ns, const uint64_t* x,
                       int64_t count, int32_t* out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t v = x[i];
        int32_t r = -1;
        if (n > 0 && v >= sample[0]) {
            const int64_t p = rank_of(ids, n, sample, ns, v);
            if (p < n && ids[p] == v) r = (int32_t)p;
        }
        out[i] = r;
    }
}
}  // namespace

int bit_width_of(int64_t v) { return bit_width(v); }

// Sorted distinct values of keys[count] into a new pool allocation *ids_out (*n_out of them).
int sort_unique_ids(cleora_ctx* ctx, const uint64_t* keys, int64_t count, uint64_t** ids_out, int64_t* n_out) {
    cudaStream_t s = ctx->stream;
    *ids_out = nullptr;
    *n_out = 0;
    DBuf<uint64_t> a(ctx), b(ctx);
    DBuf<int64_t> num(ctx);
    CL_TRY(a.alloc((size_t)count));
    CL_TRY(b.alloc((size_t)count));
    CL_TRY(num.alloc(1));
    if (count > 0)
        CL_CUDA(ctx, cudaMemcpyAsync(a.p, keys, count * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
    CL_CUDA(ctx, cudaMemsetAsync(num.p, 0, sizeof(int64_t), s));
    if (count > 0) {
        cub::DoubleBuffer<uint64_t> db(a.p, b.p);
        size_t tb = 0, tu = 0;
        CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(nullptr, tb, db, count, 0, 64, s));
        CL_CUDA(ctx, cub::DeviceSelect::Unique(nullptr, tu, db.Current(), db.Alternate(), num.p, count, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb > tu ? tb : tu));
        CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(tmp.p, tb, db, count, 0, 64, s));
        CL_CUDA(ctx, cub::DeviceSelect::Unique(tmp.p, tu, db.Current(), db.Alternate(), num.p, count, s));
        int64_t n = 0;
        CL_CUDA(ctx, cudaMemcpyAsync(&n, num.p, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        CL_TRY(dalloc(ctx, ids_out, (size_t)(n ? n : 1)));
        CL_CUDA(ctx, cudaMemcpyAsync(*ids_out, db.Alternate(), n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        *n_out = n;
    } else {
        CL_TRY(dalloc(ctx, ids_out, 1));
    }
    return CLEORA_OK;
}

int check_weights(cleora_ctx* ctx, const float* w, int64_t E) {
    if (!w || E == 0) return CLEORA_OK;
    DBuf<int> flag(ctx);
    CL_TRY(flag.alloc(1));
    CL_CUDA(ctx, cudaMemsetAsync(flag.p, 0, sizeof(int), ctx->stream));
    k_check_weights<<<grid_for(E, 256, ctx->num_sms), 256, 0, ctx->stream>>>(w, E, flag.p);
    CL_LAUNCHED(ctx);
    int bad = 0;
    CL_CUDA(ctx, cudaMemcpyAsync(&bad, flag.p, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (bad) return fail(ctx, CLEORA_ERR_INVALID_ARG, "weights must be finite and > 0");
    return CLEORA_OK;
}

int rank_ids(cleora_ctx* ctx, const uint64_t* ids, int64_t n, const uint64_t* x, int64_t count,
             int32_t* rank_out) {
    if (count == 0) return CLEORA_OK;
    const int64_t ns = n > 0 ? (n + SAMPLE - 1) / SAMPLE : 1;
    DBuf<uint64_t> sample(ctx);
    CL_TRY(sample.alloc((size_t)ns));
    if (n > 0) {
        k_sample_ids<<<grid_for(ns, 256, ctx->num_sms), 256, 0, ctx->stream>>>(ids, n, sample.p, ns);
        CL_LAUNCHED(ctx);
    }
    k_rank<<<grid_for(count, 256, ctx->num_sms), 256, 0, ctx->stream>>>(ids, n, sample.p, ns, x, count, rank_out);
    CL_LAUNCHED(ctx);
    return CLEORA_OK;
}

int csr_values_out(cleora_ctx* ctx, float* val_dev) {
    Graph& g = ctx->g;
    if (g.nnz == 0) return CLEORA_OK;
    if (g.has_val) {
        if (g.hot_cnt) return values_out_sorted(ctx, val_dev);
        CL_CUDA(ctx, cudaMemcpyAsync(val_dev, g.val, g.nnz * sizeof(float), cudaMemcpyDeviceToDevice,
                                     ctx->stream));
        return CLEORA_OK;
    }
    k_broadcast_inv<<<grid_for(g.n, 256, ctx->num_sms), 256, 0, ctx->stream>>>(g.rowptr, g.inv_deg,
                                                                             g.n, val_dev);
    CL_LAUNCHED(ctx);
    return CLEORA_OK;
}

}  // namespace cleora
