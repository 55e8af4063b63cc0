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

// Endpoint occurrences of the chunk's edges, per node index of `ids`.
__global__ void k_occ(const int32_t* rs, const int32_t* rd, int64_t E, float* occ) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < E;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (rs[i] >= 0) atomicAdd(occ + rs[i], 1.0f);
        if (rd[i] >= 0) atomicAdd(occ + rd[i], 1.0f);
    }
}

// acc[v] += occ_q(i) / occ(v) * T_q[i] for every node i of the chunk (v its union index).
template <typename ST>
__global__ void k_merge(const ST* Tq, int64_t nq, int d, const int32_t* vidx, const float* occ_q,
                        const float* occ_all, float* acc) {
    const int64_t total = nq * (int64_t)d;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = k / d;
        const int j = (int)(k - i * d);
        const int32_t v = vidx[i];
        const float wq = __fdiv_rn(occ_q[i], occ_all[v]);
        float x;
        if constexpr (sizeof(ST) == 4) x = Tq[k];
        else x = __bfloat162float(Tq[k]);
        acc[(int64_t)v * d + j] = fmaf(wq, x, acc[(int64_t)v * d + j]);
    }
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
        cudaError_t e = cudaMemcpyAsync(&nkept, scal, 8, cudaMemcpyDeviceToHost, s);
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
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (num_chunks < 1 || !chunk_offsets || chunk_offsets[0] != 0 || d < 8 || d > 1024 || d % 8 || iters < 0 ||
        (storage != CLEORA_F32 && storage != CLEORA_BF16) || out_rows < 0)
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "bad chunked-embedding arguments");
    for (int q = 0; q < num_chunks; ++q)
        if (chunk_offsets[q + 1] < chunk_offsets[q]) return fail(ctx, CLEORA_ERR_INVALID_ARG, "chunk offsets decrease");
    const int64_t E = chunk_offsets[num_chunks];
    if (E > 0 && (!src || !dst)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null edge array");
    if (num_nodes) *num_nodes = 0;
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    void *d_src = nullptr, *d_dst = nullptr, *d_w = nullptr;
    bool o1 = false, o2 = false, o3 = false;
    uint64_t *ends = nullptr, *ids_u = nullptr;
    int32_t *rs = nullptr, *rd = nullptr, *vidx = nullptr;
    float *occ_all = nullptr, *occ_q = nullptr, *acc = nullptr;
    int64_t n_u = 0;
    int rc = CLEORA_OK;
    do {
        if ((rc = to_device(ctx, src, E * 8, inputs_on_device, &d_src, &o1))) break;
        if ((rc = to_device(ctx, dst, E * 8, inputs_on_device, &d_dst, &o2))) break;
        if ((rc = to_device(ctx, weights, E * 4, inputs_on_device, &d_w, &o3))) break;
        if ((rc = check_weights(ctx, static_cast<const float*>(d_w), E))) break;
        // V = union of all chunks' nodes, ascending id
        if ((rc = dalloc(ctx, &ends, (size_t)(2 * E)))) break;
        cudaError_t e = cudaSuccess;
        if (E) e = cudaMemcpyAsync(ends, d_src, E * 8, cudaMemcpyDeviceToDevice, s);
        if (E && e == cudaSuccess) e = cudaMemcpyAsync(ends + E, d_dst, E * 8, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__); break; }
        if ((rc = sort_unique_ids(ctx, ends, 2 * E, &ids_u, &n_u))) break;
        if (num_nodes) *num_nodes = n_u;
        if (out && out_rows < n_u) {
            rc = fail(ctx, CLEORA_ERR_INVALID_ARG, "out has %lld rows, the graph %lld nodes", (long long)out_rows,
                      (long long)n_u);
            break;
        }
        if (n_u == 0) break;
        // occurrences of every node over all chunks
        if ((rc = dalloc(ctx, &rs, (size_t)E))) break;
        if ((rc = dalloc(ctx, &rd, (size_t)E))) break;
        if ((rc = dalloc(ctx, &occ_all, (size_t)n_u))) break;
        if ((rc = dalloc(ctx, &acc, (size_t)n_u * d))) break;
        e = cudaMemsetAsync(occ_all, 0, n_u * 4, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(acc, 0, n_u * (size_t)d * 4, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__); break; }
        if ((rc = rank_ids(ctx, ids_u, n_u, static_cast<const uint64_t*>(d_src), E, rs))) break;
        if ((rc = rank_ids(ctx, ids_u, n_u, static_cast<const uint64_t*>(d_dst), E, rd))) break;
        k_occ<<<grid_for(E, 256, sms), 256, 0, s>>>(rs, rd, E, occ_all);
        ctx->launches++;
        // chunk by chunk: embed, then add w_qv * T^q_v
        for (int q = 0; q < num_chunks && rc == CLEORA_OK; ++q) {
            const int64_t b = chunk_offsets[q], Eq = chunk_offsets[q + 1] - b;
            if (Eq == 0) continue;
            const uint64_t* qs = static_cast<const uint64_t*>(d_src) + b;
            const uint64_t* qd = static_cast<const uint64_t*>(d_dst) + b;
            const float* qw = d_w ? static_cast<const float*>(d_w) + b : nullptr;
            if ((rc = cleora_graph_build(ctx, qs, qd, qw, Eq, directed, 1))) break;
            if ((rc = cleora_init(ctx, d, seed, storage))) break;
            if ((rc = cleora_propagate(ctx, iters, nullptr, 1))) break;
            const int64_t nq = ctx->g.n;
            if ((rc = dalloc(ctx, &occ_q, (size_t)nq))) break;
            if ((rc = dalloc(ctx, &vidx, (size_t)nq))) break;
            e = cudaMemsetAsync(occ_q, 0, nq * 4, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__); break; }
            if ((rc = rank_ids(ctx, ctx->g.ids, nq, qs, Eq, rs))) break;
            if ((rc = rank_ids(ctx, ctx->g.ids, nq, qd, Eq, rd))) break;
            k_occ<<<grid_for(Eq, 256, sms), 256, 0, s>>>(rs, rd, Eq, occ_q);
            if ((rc = rank_ids(ctx, ids_u, n_u, ctx->g.ids, nq, vidx))) break;
            if (storage == CLEORA_F32)
                k_merge<float><<<grid_for(nq * (int64_t)d, 256, sms), 256, 0, s>>>(
                    static_cast<const float*>(ctx->T[ctx->cur]), nq, d, vidx, occ_q, occ_all, acc);
            else
                k_merge<__nv_bfloat16><<<grid_for(nq * (int64_t)d, 256, sms), 256, 0, s>>>(
                    static_cast<const __nv_bfloat16*>(ctx->T[ctx->cur]), nq, d, vidx, occ_q, occ_all, acc);
            ctx->launches += 2;
            e = cudaGetLastError();
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "chunk merge", __FILE__, __LINE__); break; }
            dfree_null(ctx, occ_q);
            dfree_null(ctx, vidx);
        }
        if (rc) break;
        if (out && (rc = copy_back(ctx, out, acc, n_u * (size_t)d * 4, out_on_device))) break;
        if (out_ids && (rc = copy_back(ctx, out_ids, ids_u, n_u * 8, out_on_device))) break;
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "chunked", __FILE__, __LINE__);
    } while (0);
    if (o1) dfree(ctx, d_src);
    if (o2) dfree(ctx, d_dst);
    if (o3) dfree(ctx, d_w);
    dfree(ctx, ends);
    dfree(ctx, ids_u);
    dfree(ctx, rs);
    dfree(ctx, rd);
    dfree(ctx, vidx);
    dfree(ctx, occ_all);
    dfree(ctx, occ_q);
    dfree(ctx, acc);
    return rc;
}

}  // extern "C"
