// The two operations the paper derives from weighted averaging (arXiv 2102.02302, Sec. 1,
// "Additivity" and "Inductivity"; Sec. 3.2, end; Algorithm 1, chunks q = 1..Q and the final
// merge):
//
//  * cleora_inductive: rows for nodes added after the embedding.  Each new node u gets
//    rownorm(sum_b M_ub T[b]) over its edges to existing nodes, with M_ub = e_ub / deg_u --
//    one more multiply-and-normalise step restricted to the new rows, run on the context's
//    current embeddings (the paper advises those of iteration I-1).  The new rows' CSR is
//    built with the graph builder's own rules and multiplied by the same row kernel.
//
//  * cleora_chunked_embed: Algorithm 1 with Q edge chunks.  Chunk q is embedded on its own
//    (its own M_q, T_0 from the same id hash, I iterations) and the results are merged as
//    T_v = sum_q w_qv T^q_v with w_qv = occ_q(v) / sum_k occ_k(v), occ_q(v) the number of
//    endpoint occurrences of v in chunk q's edges (a self-loop counts twice).  Chunks are
//    merged in order, so the result is deterministic.
#include <algorithm>
#include <vector>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_reduce.cuh>
#include <cub/device/device_run_length_encode.cuh>
#include <cub/device/device_select.cuh>

#include "propagate_kernels.cuh"

namespace cleora {
namespace ext {
namespace {

constexpr int ROWS_PER_TASK = 32;

// Rows [0, nrows) of a CSR whose rows all have entries, as tasks of 32 rows.
template <typename ST, int VEC, int CPL, int G, bool HV>
__global__ void __launch_bounds__(256) k_rows(prop::Args a, int64_t nrows, unsigned long long* counter) {
    using K = prop::Kern<ST, VEC, CPL, G, HV>;
    const int lane = threadIdx.x & 31;
    const int g = lane / G, lg = lane % G;
    const int64_t ntasks = (nrows + ROWS_PER_TASK - 1) / ROWS_PER_TASK;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(counter, 1ull);
        t = __shfl_sync(prop::FULL, t, 0);
        if ((int64_t)t >= ntasks) break;
        const int64_t rb = (int64_t)t * ROWS_PER_TASK;
        K::rows_coop(a, rb, min(nrows, rb + ROWS_PER_TASK), lane, g, lg);
        __syncwarp();
    }
}

template <typename ST, int VEC, bool HV>
cudaError_t launch_rows(const Shape& sh, const prop::Args& a, int64_t nrows, unsigned long long* counter,
                        int sms, cudaStream_t s) {
    auto go = [&](auto kern) -> cudaError_t {
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0);
        if (e != cudaSuccess) return e;
        kern<<<(bps < 1 ? 1 : bps) * sms, 256, 0, s>>>(a, nrows, counter);
        return cudaGetLastError();
    };
    if (sh.cpl == 1) {
        switch (sh.G) {
            case 1: return go(k_rows<ST, VEC, 1, 1, HV>);
            case 2: return go(k_rows<ST, VEC, 1, 2, HV>);
            case 4: return go(k_rows<ST, VEC, 1, 4, HV>);
            case 8: return go(k_rows<ST, VEC, 1, 8, HV>);
            case 16: return go(k_rows<ST, VEC, 1, 16, HV>);
            case 32: return go(k_rows<ST, VEC, 1, 32, HV>);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sh.cpl) {
        case 2: return go(k_rows<ST, VEC, 2, 32, HV>);
        case 4: return go(k_rows<ST, VEC, 4, 32, HV>);
        case 8: return go(k_rows<ST, VEC, 8, 32, HV>);
        default: return cudaErrorInvalidValue;
    }
}

__global__ void k_valid_flags(const int32_t* rank, int64_t E, uint8_t* flag) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x)
        flag[i] = rank[i] >= 0 ? 1 : 0;
}

__global__ void k_new_entries(const int32_t* urank, const int32_t* nrank, const float* w, int64_t E, int bits,
                              uint64_t invalid, uint64_t* keys, float* vals) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool ok = nrank[i] >= 0 && urank[i] >= 0;
        keys[i] = ok ? (((uint64_t)urank[i] << bits) | (uint64_t)nrank[i]) : invalid;
        if (vals) vals[i] = w[i];
    }
}

// Endpoint occurrences of the chunk's edges, per node index of `ids` (exact integer counts).
__global__ void k_occ(const int32_t* rs, const int32_t* rd, int64_t E, unsigned long long* occ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (rs[i] >= 0) atomicAdd(occ + rs[i], 1ull);
        if (rd[i] >= 0) atomicAdd(occ + rd[i], 1ull);
    }
}

// acc[v] += w_qv T_q[i] for every node i of the chunk (v its index in the union), with
// w_qv = occ_q(i) / occ(v) from the exact counts (FP64 ratio rounded once to FP32).  acc is
// the caller's output: device memory or mapped host memory.
template <typename ST>
__global__ void k_merge(const ST* Tq, int64_t nq, int d, const int32_t* vidx, const unsigned long long* occ_q,
                        const unsigned long long* occ_all, float* acc) {
    const int64_t total = nq * (int64_t)d;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / d;
        const int j = (int)(k - i * d);
        const int32_t v = vidx[i];
        const float wq = (float)((double)occ_q[i] / (double)occ_all[v]);
        float x;
        if constexpr (sizeof(ST) == 4) x = Tq[k];
        else x = __bfloat162float(Tq[k]);
        acc[(int64_t)v * d + j] = fmaf(wq, x, acc[(int64_t)v * d + j]);
    }
}

__global__ void k_zero(float* p, int64_t count) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        p[k] = 0.f;
}

__global__ void k_concat_u32to64(const uint32_t* c, int64_t n, unsigned long long* out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = c[k];
}

size_t es_of(cleora_dtype t) { return t == CLEORA_F32 ? 4 : 2; }

int to_device(cleora_ctx* ctx, const void* p, size_t bytes, int on_device, void** dev, bool* owned) {
    *owned = false;
    *dev = const_cast<void*>(p);
    if (on_device || !p || bytes == 0) return CLEORA_OK;
    CL_TRY(dalloc_bytes(ctx, dev, bytes));
    *owned = true;
    CL_CUDA(ctx, cudaMemcpyAsync(*dev, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return CLEORA_OK;
}

int copy_back(cleora_ctx* ctx, void* out, const void* dev, size_t bytes, int out_on_device) {
    if (bytes == 0) return CLEORA_OK;
    CL_CUDA(ctx, cudaMemcpyAsync(out, dev, bytes, out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CLEORA_OK;
}

void release_sub(cleora_ctx* ctx, Graph& g) {
    dfree_null(ctx, g.rowptr);
    dfree_null(ctx, g.col);
    dfree_null(ctx, g.val);
    dfree_null(ctx, g.deg);
    dfree_null(ctx, g.inv_deg);
    dfree_null(ctx, g.ids);
}

}  // namespace
}  // namespace ext
}  // namespace cleora

using namespace cleora;
using namespace cleora::ext;

extern "C" {

int cleora_inductive(cleora_ctx* ctx, const uint64_t* new_ids, const uint64_t* nbr_ids, const float* weights,
                     int64_t num_edges, int inputs_on_device, uint64_t* out_ids, float* out, int64_t out_rows,
                     int64_t* num_new, int64_t* num_dropped, int out_on_device) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!ctx->inited) return fail(ctx, CLEORA_ERR_STATE, "inductive rows need embeddings (init first)");
    if (num_edges < 0 || (num_edges > 0 && (!new_ids || !nbr_ids)) || out_rows < 0)
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "bad inductive arguments");
    if (num_new) *num_new = 0;
    if (num_dropped) *num_dropped = 0;
    if (num_edges == 0) return CLEORA_OK;
    const int64_t E = num_edges;
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    void *d_new = nullptr, *d_nbr = nullptr, *d_w = nullptr;
    bool o1 = false, o2 = false, o3 = false;
    int32_t *nrank = nullptr, *urank = nullptr;
    uint8_t* flag = nullptr;
    uint64_t *kept = nullptr, *U = nullptr, *ka = nullptr, *kb = nullptr;
    float *va = nullptr, *vb = nullptr;
    int64_t* scal = nullptr;
    unsigned long long* counter = nullptr;
    void* Tsub = nullptr;
    Graph sub;
    int rc = CLEORA_OK;
    int64_t m_new = 0;
    do {
        if ((rc = to_device(ctx, new_ids, E * 8, inputs_on_device, &d_new, &o1))) break;
        if ((rc = to_device(ctx, nbr_ids, E * 8, inputs_on_device, &d_nbr, &o2))) break;
        if ((rc = to_device(ctx, weights, E * 4, inputs_on_device, &d_w, &o3))) break;
        if ((rc = check_weights(ctx, static_cast<const float*>(d_w), E))) break;
        // neighbours among the existing nodes; edges to unknown nodes are dropped
        if ((rc = dalloc(ctx, &nrank, (size_t)E))) break;
        if ((rc = rank_ids(ctx, ctx->g.ids, ctx->g.n, static_cast<const uint64_t*>(d_nbr), E, nrank))) break;
        // new nodes: distinct new ids over the kept edges, ascending
        if ((rc = dalloc(ctx, &flag, (size_t)E))) break;
        if ((rc = dalloc(ctx, &kept, (size_t)E))) break;
        if ((rc = dalloc(ctx, &scal, 1))) break;
        k_valid_flags<<<grid_for(E, 256, sms), 256, 0, s>>>(nrank, E, flag);
        ctx->launches++;
        {
            size_t tb = 0;
            cudaError_t e = cub::DeviceSelect::Flagged(nullptr, tb, static_cast<const uint64_t*>(d_new), flag, kept,
                                                       scal, E, s);
            void* tmp = nullptr;
            if (e == cudaSuccess && (rc = dalloc_bytes(ctx, &tmp, tb)) == CLEORA_OK)
                e = cub::DeviceSelect::Flagged(tmp, tb, static_cast<const uint64_t*>(d_new), flag, kept, scal, E, s);
            dfree(ctx, tmp);
            if (rc) break;
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "select", __FILE__, __LINE__); break; }
        }
        int64_t nkept = 0;
        cudaError_t e = read_back(ctx, &nkept, scal, 8, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "inductive", __FILE__, __LINE__); break; }
        if (num_dropped) *num_dropped = E - nkept;
        if ((rc = sort_unique_ids(ctx, kept, nkept, &U, &m_new))) break;
        if (num_new) *num_new = m_new;
        if (m_new == 0) break;
        if (out && out_rows < m_new) {
            rc = fail(ctx, CLEORA_ERR_INVALID_ARG, "out has %lld rows, %lld new nodes", (long long)out_rows,
                      (long long)m_new);
            break;
        }
        if ((rc = dalloc(ctx, &urank, (size_t)E))) break;
        if ((rc = rank_ids(ctx, U, m_new, static_cast<const uint64_t*>(d_new), E, urank))) break;
        // CSR of the new rows against the existing columns (the builder's rules)
        const int bits = bit_width_of(std::max<int64_t>(m_new, ctx->g.n));
        const uint64_t invalid = (bits * 2 >= 64) ? ~0ull : ((1ull << (2 * bits)) - 1ull);
        if ((rc = dalloc(ctx, &ka, (size_t)E))) break;
        if ((rc = dalloc(ctx, &kb, (size_t)E))) break;
        if (d_w) {
            if ((rc = dalloc(ctx, &va, (size_t)E))) break;
            if ((rc = dalloc(ctx, &vb, (size_t)E))) break;
        }
        k_new_entries<<<grid_for(E, 256, sms), 256, 0, s>>>(urank, nrank, static_cast<const float*>(d_w), E, bits,
                                                           invalid, ka, va);
        ctx->launches++;
        if ((rc = csr_from_entries(ctx, ka, kb, va, vb, E, E, m_new, bits, invalid, sub))) break;
        // one multiply-and-normalise step of the new rows on the current embeddings
        const size_t es = es_of(ctx->dtype);
        if ((rc = dalloc_bytes(ctx, &Tsub, (size_t)m_new * ctx->d * es))) break;
        if ((rc = dalloc(ctx, &counter, 1))) break;
        e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "inductive", __FILE__, __LINE__); break; }
        const Shape sh = shape_for(ctx->d, ctx->dtype, 16, 1);
        prop::Args a;
        a.rowptr = sub.rowptr;
        a.col = sub.col;
        a.val = sub.val;
        a.Tin = static_cast<const unsigned char*>(ctx->T[ctx->cur]);
        a.Tout = static_cast<unsigned char*>(Tsub);
        a.n = ctx->g.n;
        a.nnz = sub.nnz;
        a.row_bytes = (int64_t)ctx->d * es;
        a.chunks = sh.chunks;
        a.d = ctx->d;
        a.split_len = 0;
        a.tasks = nullptr;
        a.ntasks = 0;
        a.counter = nullptr;
        a.split_base = nullptr;
        a.split_count = nullptr;
        a.partials = nullptr;
        a.err = ctx->err_flag;
        const bool hv = sub.has_val;
        if (ctx->dtype == CLEORA_F32)
            e = hv ? launch_rows<float, 16, true>(sh, a, m_new, counter, sms, s)
                   : launch_rows<float, 16, false>(sh, a, m_new, counter, sms, s);
        else
            e = hv ? launch_rows<__nv_bfloat16, 16, true>(sh, a, m_new, counter, sms, s)
                   : launch_rows<__nv_bfloat16, 16, false>(sh, a, m_new, counter, sms, s);
        ctx->launches++;
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "inductive launch", __FILE__, __LINE__); break; }
        // results: FP32 rows and their ids
        if (out) {
            const int64_t count = m_new * (int64_t)ctx->d;
            if (out_on_device) {
                rc = convert_impl(ctx, Tsub, ctx->dtype, out, CLEORA_F32, count);
            } else {
                float* tmp = nullptr;
                if ((rc = dalloc(ctx, &tmp, (size_t)count))) break;
                rc = convert_impl(ctx, Tsub, ctx->dtype, tmp, CLEORA_F32, count);
                if (rc == CLEORA_OK) rc = copy_back(ctx, out, tmp, count * 4, 0);
                dfree(ctx, tmp);
            }
            if (rc) break;
        }
        if (out_ids && (rc = copy_back(ctx, out_ids, U, m_new * 8, out_on_device))) break;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "inductive", __FILE__, __LINE__);
    } while (0);
    if (o1) dfree(ctx, d_new);
    if (o2) dfree(ctx, d_nbr);
    if (o3) dfree(ctx, d_w);
    dfree(ctx, nrank);
    dfree(ctx, urank);
    dfree(ctx, flag);
    dfree(ctx, kept);
    dfree(ctx, U);
    dfree(ctx, ka);
    dfree(ctx, kb);
    dfree(ctx, va);
    dfree(ctx, vb);
    dfree(ctx, scal);
    dfree(ctx, counter);
    dfree(ctx, Tsub);
    release_sub(ctx, sub);
    return rc;
}

int cleora_chunked_embed(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst, const float* weights,
                         const int64_t* chunk_offsets, int num_chunks, int directed, int d, int iters, uint64_t seed,
                         cleora_dtype storage, int inputs_on_device, uint64_t* out_ids, float* out,
                         int64_t out_rows, int64_t* num_nodes, int out_on_device) {
    using namespace ext;
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (num_chunks < 0 || (num_chunks > 0 && (!chunk_offsets || chunk_offsets[0] != 0)) || d < 8 || d > 1024 ||
        d % 8 || iters < 0 || (storage != CLEORA_F32 && storage != CLEORA_BF16) || out_rows < 0)
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "bad chunked-embedding arguments");
    for (int q = 0; q < num_chunks; ++q)
        if (chunk_offsets[q + 1] < chunk_offsets[q]) return fail(ctx, CLEORA_ERR_INVALID_ARG, "chunk offsets decrease");
    if (num_chunks == 0 && !chunk_offsets && src == nullptr && dst == nullptr)
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "no edges");
    if (num_nodes) *num_nodes = 0;
    ctx->chunks_used = 0;
    ctx->chunk_peak_bytes = 0;
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    // the number of edges: given by the offsets, or (automatic chunks) by chunk_offsets[0] = E
    // passed as the only element
    const int64_t E = num_chunks > 0 ? chunk_offsets[num_chunks] : (chunk_offsets ? chunk_offsets[0] : 0);
    if (E < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "negative edge count");
    if (E > 0 && (!src || !dst)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null edge array");
    // device bytes a chunk may use
    int64_t cap = ctx->opt[CLEORA_OPT_CHUNK_BYTES];
    if (cap == 0) {
        size_t fr = 0, tot = 0;
        CL_CUDA(ctx, cudaMemGetInfo(&fr, &tot));
        cap = (int64_t)(0.8 * (double)fr);
    }
    {  // reset the pool's high-water mark: the call reports its own device peak
        unsigned long long zero = 0;
        cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    // a chunk's peak: the serving estimate of its build and embedding, taken for FP32 storage
    // (BF16 needs no more; the estimate's BF16 term is for result staging, which chunks skip)
    auto chunk_estimate = [&](int64_t Eq) -> int64_t {
        cleora_job j{};
        j.num_edges = Eq;
        j.directed = directed;
        j.d = d;
        j.storage = CLEORA_F32;
        j.weights = weights;
        return cleora_serve_estimate(&j);
    };
    const size_t ew = weights ? 4 : 0;
    // chunk staging: device pointers of edges [b, b + Eq) (uploaded when the inputs are on the host)
    void *bs = nullptr, *bd = nullptr, *bw = nullptr;
    int64_t bcap = 0;
    auto stage = [&](int64_t b, int64_t Eq, const uint64_t** qs, const uint64_t** qd, const float** qw) -> int {
        if (inputs_on_device) {
            *qs = src + b;
            *qd = dst + b;
            *qw = weights ? weights + b : nullptr;
            return CLEORA_OK;
        }
        if (Eq > bcap) {
            dfree_null(ctx, bs);
            dfree_null(ctx, bd);
            dfree_null(ctx, bw);
            bcap = 0;
            CL_TRY(dalloc_bytes(ctx, &bs, (size_t)Eq * 8));
            CL_TRY(dalloc_bytes(ctx, &bd, (size_t)Eq * 8));
            if (weights) CL_TRY(dalloc_bytes(ctx, &bw, (size_t)Eq * 4));
            bcap = Eq;
        }
        CL_CUDA(ctx, cudaMemcpyAsync(bs, src + b, Eq * 8, cudaMemcpyHostToDevice, s));
        CL_CUDA(ctx, cudaMemcpyAsync(bd, dst + b, Eq * 8, cudaMemcpyHostToDevice, s));
        if (weights) CL_CUDA(ctx, cudaMemcpyAsync(bw, weights + b, Eq * ew, cudaMemcpyHostToDevice, s));
        *qs = static_cast<const uint64_t*>(bs);
        *qd = static_cast<const uint64_t*>(bd);
        *qw = static_cast<const float*>(bw);
        return CLEORA_OK;
    };
    uint64_t* V = nullptr;               // distinct ids of all chunks, ascending
    unsigned long long* occ_all = nullptr;  // their endpoint occurrences (exact)
    int64_t nV = 0;
    uint64_t *ends = nullptr, *ends2 = nullptr, *ku = nullptr, *mk = nullptr, *mk2 = nullptr;
    uint32_t* cu = nullptr;
    unsigned long long *mv = nullptr, *mv2 = nullptr, *occ_q = nullptr;
    int64_t* scal = nullptr;
    int32_t *rs = nullptr, *rd = nullptr, *vidx = nullptr;
    void* tmp = nullptr;
    float* acc = nullptr;
    bool registered = false;
    int rc = CLEORA_OK;
    std::vector<int64_t> offs;
    auto cub_tmp = [&](size_t bytes) -> int {  // temporary storage for one CUB call
        dfree_null(ctx, tmp);
        return dalloc_bytes(ctx, &tmp, bytes ? bytes : 1);
    };
    do {
        if ((rc = dalloc(ctx, &scal, 1))) break;
        // ---- pass 1: the node set and occurrence counts, chunk by chunk -------------------
        // (automatic chunks: pieces of cap / 160 edges, about 70 bytes per edge plus the node arrays)
        std::vector<int64_t> offs1;
        if (num_chunks > 0) {
            offs1.assign(chunk_offsets, chunk_offsets + num_chunks + 1);
        } else {
            const int64_t Eq1 = std::max<int64_t>(1, cap / 160);
            for (int64_t b = 0; b < E; b += Eq1) offs1.push_back(b);
            offs1.push_back(E);
        }
        for (size_t q = 0; q + 1 < offs1.size() && rc == CLEORA_OK; ++q) {
            const int64_t b = offs1[q], Eq = offs1[q + 1] - b;
            if (Eq == 0) continue;
            const uint64_t *qs, *qd;
            const float* qw;
            if ((rc = stage(b, Eq, &qs, &qd, &qw))) break;
            if ((rc = check_weights(ctx, qw, Eq))) break;
            const int64_t m = 2 * Eq;
            if ((rc = dalloc(ctx, &ends, (size_t)m))) break;
            if ((rc = dalloc(ctx, &ends2, (size_t)m))) break;
            cudaError_t e = cudaMemcpyAsync(ends, qs, Eq * 8, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(ends + Eq, qd, Eq * 8, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            size_t tb = 0;
            cub::DoubleBuffer<uint64_t> keys(ends, ends2);
            e = cub::DeviceRadixSort::SortKeys(nullptr, tb, keys, m, 0, 64, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess) e = cub::DeviceRadixSort::SortKeys(tmp, tb, keys, m, 0, 64, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            uint64_t* sorted = keys.Current();
            uint64_t* spare = keys.Alternate();
            // run-length encode: unique ids into `spare`, counts into cu
            if ((rc = dalloc(ctx, &cu, (size_t)m))) break;
            tb = 0;
            e = cub::DeviceRunLengthEncode::Encode(nullptr, tb, sorted, spare, cu, scal, m, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess) e = cub::DeviceRunLengthEncode::Encode(tmp, tb, sorted, spare, cu, scal, m, s);
            int64_t nu = 0;
            if (e == cudaSuccess) e = read_back(ctx, &nu, scal, 8, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            ctx->launches += 2;
            // merge (V, occ_all) with (spare, cu): concatenate, sort by id, add equal ids' counts
            const int64_t mm = nV + nu;
            if ((rc = dalloc(ctx, &mk, (size_t)mm))) break;
            if ((rc = dalloc(ctx, &mk2, (size_t)mm))) break;
            if ((rc = dalloc(ctx, &mv, (size_t)mm))) break;
            if ((rc = dalloc(ctx, &mv2, (size_t)mm))) break;
            if (nV) e = cudaMemcpyAsync(mk, V, nV * 8, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && nV) e = cudaMemcpyAsync(mv, occ_all, nV * 8, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(mk + nV, spare, nu * 8, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            k_concat_u32to64<<<grid_for(nu, 256, sms), 256, 0, s>>>(cu, nu, mv + nV);
            ctx->launches++;
            dfree_null(ctx, ends);
            dfree_null(ctx, ends2);
            dfree_null(ctx, cu);
            cub::DoubleBuffer<uint64_t> k2(mk, mk2);
            cub::DoubleBuffer<unsigned long long> v2(mv, mv2);
            tb = 0;
            e = cub::DeviceRadixSort::SortPairs(nullptr, tb, k2, v2, mm, 0, 64, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess) e = cub::DeviceRadixSort::SortPairs(tmp, tb, k2, v2, mm, 0, 64, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            dfree_null(ctx, V);
            dfree_null(ctx, occ_all);
            if ((rc = dalloc(ctx, &V, (size_t)mm))) break;
            if ((rc = dalloc(ctx, &occ_all, (size_t)mm))) break;
            tb = 0;
            e = cub::DeviceReduce::ReduceByKey(nullptr, tb, k2.Current(), V, v2.Current(), occ_all, scal,
                                               cuda::std::plus<unsigned long long>(), mm, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess)
                e = cub::DeviceReduce::ReduceByKey(tmp, tb, k2.Current(), V, v2.Current(), occ_all, scal,
                                                   cuda::std::plus<unsigned long long>(), mm, s);
            if (e == cudaSuccess) e = read_back(ctx, &nV, scal, 8, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk ids", __FILE__, __LINE__); break; }
            ctx->launches += 2;
            dfree_null(ctx, mk);
            dfree_null(ctx, mk2);
            dfree_null(ctx, mv);
            dfree_null(ctx, mv2);
            dfree_null(ctx, tmp);
        }
        if (rc) break;
        dfree_null(ctx, bs);  // pass 2 stages its own chunk sizes
        dfree_null(ctx, bd);
        dfree_null(ctx, bw);
        bcap = 0;
        if (nV >= ((int64_t)1 << 31)) { rc = fail(ctx, CLEORA_ERR_INVALID_ARG, "more than 2^31 - 1 nodes"); break; }
        if (num_nodes) *num_nodes = nV;
        if (out && out_rows < nV) {
            rc = fail(ctx, CLEORA_ERR_INVALID_ARG, "out has %lld rows, the graph %lld nodes", (long long)out_rows,
                      (long long)nV);
            break;
        }
        if (nV == 0) break;
        // ---- the chunks of Algorithm 1 -------------------------------------------------------
        if (num_chunks > 0) {
            offs.assign(chunk_offsets, chunk_offsets + num_chunks + 1);
        } else {  // fewest equal chunks whose estimated peak, next to the node arrays, fits the cap
            const int64_t fixed = nV * (8 + 8 + 4 + 8);  // V, occ_all, and a chunk's vidx, occ_q
            int64_t Q = 1;
            while (Q < E && chunk_estimate((E + Q - 1) / Q) + fixed + (inputs_on_device ? 0 : ((E + Q - 1) / Q) * (16 + (int64_t)ew)) > cap)
                Q = Q * 2 > E ? E : Q * 2;
            int64_t lo = std::max<int64_t>(1, Q / 2), hi = Q;  // smallest Q in (Q/2, Q] that fits
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                const int64_t Em = (E + mid - 1) / mid;
                if (chunk_estimate(Em) + fixed + (inputs_on_device ? 0 : Em * (16 + (int64_t)ew)) <= cap) hi = mid;
                else lo = mid + 1;
            }
            Q = hi;
            if (Q > (int64_t)1 << 20) { rc = fail(ctx, CLEORA_ERR_OOM, "the chunk cap is too small for this graph"); break; }
            offs.resize(Q + 1);
            for (int64_t q = 0; q <= Q; ++q) offs[q] = (int64_t)((__int128)E * q / Q);
        }
        ctx->chunks_used = (int)(offs.size() - 1);
        // accumulator: the caller's output (device, or host memory mapped into the device)
        if (out) {
            if (out_on_device) {
                acc = out;
            } else {
                void* mapped = nullptr;
                cudaPointerAttributes pa;
                if (cudaPointerGetAttributes(&pa, out) == cudaSuccess && pa.type == cudaMemoryTypeHost)
                    mapped = pa.devicePointer;
                cudaGetLastError();
                if (!mapped) {
                    cudaError_t e = cudaHostRegister(out, (size_t)nV * d * 4, cudaHostRegisterMapped);
                    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&mapped, out, 0);
                    if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "map output", __FILE__, __LINE__); break; }
                    registered = true;
                }
                acc = static_cast<float*>(mapped);
            }
            k_zero<<<grid_for(nV * (int64_t)d, 256, sms), 256, 0, s>>>(acc, nV * (int64_t)d);
            ctx->launches++;
        }
        // ---- pass 2: embed each chunk, merge its weighted rows into the output -------------
        for (size_t q = 0; q + 1 < offs.size() && rc == CLEORA_OK; ++q) {
            const int64_t b = offs[q], Eq = offs[q + 1] - b;
            if (Eq == 0) continue;
            const uint64_t *qs, *qd;
            const float* qw;
            if ((rc = stage(b, Eq, &qs, &qd, &qw))) break;
            if ((rc = cleora_graph_build(ctx, qs, qd, qw, Eq, directed, 1))) break;
            if ((rc = cleora_init(ctx, d, seed, storage))) break;
            if ((rc = cleora_propagate(ctx, iters, nullptr, 1))) break;
            if (!acc) continue;
            const int64_t nq = ctx->g.n;
            if ((rc = dalloc(ctx, &rs, (size_t)Eq))) break;
            if ((rc = dalloc(ctx, &rd, (size_t)Eq))) break;
            if ((rc = dalloc(ctx, &occ_q, (size_t)nq))) break;
            if ((rc = dalloc(ctx, &vidx, (size_t)nq))) break;
            cudaError_t e = cudaMemsetAsync(occ_q, 0, nq * 8, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__); break; }
            if ((rc = rank_ids(ctx, ctx->g.ids, nq, qs, Eq, rs))) break;
            if ((rc = rank_ids(ctx, ctx->g.ids, nq, qd, Eq, rd))) break;
            k_occ<<<grid_for(Eq, 256, sms), 256, 0, s>>>(rs, rd, Eq, occ_q);
            if ((rc = rank_ids(ctx, V, nV, ctx->g.ids, nq, vidx))) break;
            if (storage == CLEORA_F32)
                k_merge<float><<<grid_for(nq * (int64_t)d, 256, sms), 256, 0, s>>>(
                    static_cast<const float*>(ctx->T[ctx->cur]), nq, d, vidx, occ_q, occ_all, acc);
            else
                k_merge<__nv_bfloat16><<<grid_for(nq * (int64_t)d, 256, sms), 256, 0, s>>>(
                    static_cast<const __nv_bfloat16*>(ctx->T[ctx->cur]), nq, d, vidx, occ_q, occ_all, acc);
            ctx->launches += 2;
            e = cudaGetLastError();
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk merge", __FILE__, __LINE__); break; }
            dfree_null(ctx, rs);
            dfree_null(ctx, rd);
            dfree_null(ctx, occ_q);
            dfree_null(ctx, vidx);
        }
        if (rc) break;
        if (out_ids && (rc = copy_back(ctx, out_ids, V, nV * 8, out_on_device))) break;
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__);
    } while (0);
    cudaStreamSynchronize(s);
    if (registered) cudaHostUnregister(out);
    dfree(ctx, bs);
    dfree(ctx, bd);
    dfree(ctx, bw);
    dfree(ctx, V);
    dfree(ctx, occ_all);
    dfree(ctx, ends);
    dfree(ctx, ends2);
    dfree(ctx, ku);
    dfree(ctx, mk);
    dfree(ctx, mk2);
    dfree(ctx, mv);
    dfree(ctx, mv2);
    dfree(ctx, cu);
    dfree(ctx, occ_q);
    dfree(ctx, scal);
    dfree(ctx, rs);
    dfree(ctx, rd);
    dfree(ctx, vidx);
    dfree(ctx, tmp);
    {
        unsigned long long high = 0;
        if (cudaMemPoolGetAttribute(ctx->pool, cudaMemPoolAttrUsedMemHigh, &high) == cudaSuccess)
            ctx->chunk_peak_bytes = (int64_t)high;
        cudaGetLastError();
    }
    return rc;
}

int cleora_chunked_info(const cleora_ctx* ctx, int* chunks, int64_t* peak_device_bytes) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    if (chunks) *chunks = ctx->chunks_used;
    if (peak_device_bytes) *peak_device_bytes = ctx->chunk_peak_bytes;
    return CLEORA_OK;
}

}  // extern "C"
