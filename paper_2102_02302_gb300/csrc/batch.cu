// Host side of the batched path (include/cleora.h, cleora_batch_*): build, pack, autotune,
// capture, replay.
//
// Every graph is built by the single-graph builder and planned by the single-graph planner
// on its own (local) CSR, so its rows are summed in exactly the order a single-graph context
// with the same schedule uses.  Packing concatenates ids, rowptr (shifted to global entry
// positions), col and values; embeddings of all graphs share two ping-pong buffers.  Graphs
// are ordered by iteration count (descending) so the tasks still active at step s are a
// prefix of each family's task list.  The captured CUDA graph holds: counter reset, T_0 of
// every graph, one persistent launch per family per step, and the FP32 output pass.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <tuple>
#include <vector>

#include "batch_kernels.cuh"

namespace cleora {
namespace batch {

struct OneGraph {
    int64_t n = 0, nnz = 0;
    bool has_val = false;
    uint64_t* ids = nullptr;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;
    Task* tasks = nullptr;
    int64_t ntasks = 0, nsplit_rows = 0, nsplit_chunks = 0;
    int64_t* split_base = nullptr;
    int64_t split_len = DEFAULT_SPLIT_LEN, task_nnz = DEFAULT_TASK_NNZ;
    int d = 0, iters = 0;
    uint64_t seed = 0;
    cleora_dtype dtype = CLEORA_F32;
    Shape shape;
};

struct Family {
    int dtype = 0, vec = 16, cpl = 1, G = 32, mode = 1, hv = 0;
    BTask* tasks = nullptr;
    int64_t ntasks = 0;
    std::vector<int64_t> nt_step;  // nt_step[s]: tasks of graphs with iters >= s
};

struct Packed {
    int count = 0, max_iters = 0;
    int64_t total_n = 0, total_nnz = 0, total_out = 0, T_bytes = 0;
    std::vector<GDesc> hgd;
    std::vector<int> slot_of;  // input graph -> packed slot
    GDesc* gd = nullptr;
    uint64_t* ids = nullptr;
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    float* val = nullptr;
    unsigned char* TA = nullptr;
    unsigned char* TB = nullptr;
    float* partials = nullptr;
    int64_t* split_base = nullptr;
    int32_t* split_count = nullptr;
    float* out = nullptr;
    int64_t* vec_prefix = nullptr;
    int64_t* outv_prefix = nullptr;
    std::vector<Family> fams;
    unsigned long long* counters = nullptr;
};

__global__ void k_shift(int64_t* dst, const int64_t* src, int64_t count, int64_t add) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i] + add;
}

__global__ void k_wrap_tasks(BTask* dst, const Task* src, int64_t count, int g) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        BTask b;
        b.t = src[i];
        b.g = g;
        b.pad = 0;
        dst[i] = b;
    }
}

// Graph holding element x of a prefix table (prefix[count] = total).
__device__ __forceinline__ int find_graph(const int64_t* prefix, int count, int64_t x) {
    int lo = 0, hi = count;  // last g with prefix[g] <= x
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (prefix[mid] <= x) lo = mid; else hi = mid;
    }
    return lo;
}

// Both passes below walk tiles of consecutive 16-byte vectors (coalesced), finding the graph
// of a thread's first vector in the tile by binary search and then stepping forward.
constexpr int64_t TILE_VECS = 4096;

inline unsigned tile_grid(int64_t total, int sms) {
    const int64_t tiles = (total + TILE_VECS - 1) / TILE_VECS;
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>(tiles, (int64_t)sms * 16));
}

// T_0 of every graph (16-byte vectors), same values as the single-graph init.
__global__ void k_batch_init(const GDesc* gd, int count, const int64_t* vec_prefix,
                             const uint64_t* ids, unsigned char* TA) {
    const int64_t total = vec_prefix[count];
    for (int64_t t0 = blockIdx.x * TILE_VECS; t0 < total; t0 += (int64_t)gridDim.x * TILE_VECS) {
        const int64_t t1 = min(total, t0 + TILE_VECS);
        if (t0 + threadIdx.x >= t1) continue;
        int g = find_graph(vec_prefix, count, t0 + threadIdx.x);
        for (int64_t v = t0 + threadIdx.x; v < t1; v += blockDim.x) {
            while (vec_prefix[g + 1] <= v) ++g;
            const GDesc& G = gd[g];
            const int64_t lv = v - vec_prefix[g];
            const int vpr = G.row_bytes / 16;
            const int64_t i = lv / vpr;
            const int64_t jv = lv - i * vpr;
            const uint64_t p = mix64(G.mseed ^ ids[G.node_off + i]);
            uint4* dst = reinterpret_cast<uint4*>(TA + G.T_off) + lv;
            if (G.dtype == CLEORA_F32) {
                const uint32_t j = (uint32_t)jv * 4u;
                *dst = make_uint4(__float_as_uint(init_value(p, j)), __float_as_uint(init_value(p, j + 1)),
                                  __float_as_uint(init_value(p, j + 2)), __float_as_uint(init_value(p, j + 3)));
            } else {
                const uint32_t j = (uint32_t)jv * 8u;
                uint32_t w[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    __nv_bfloat162 h = __floats2bfloat162_rn(init_value(p, j + 2 * k), init_value(p, j + 2 * k + 1));
                    w[k] = *reinterpret_cast<uint32_t*>(&h);
                }
                *dst = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
    }
}

// Every graph's final iterate as FP32 into the packed output (4 elements per unit).
__global__ void k_batch_out(const GDesc* gd, int count, const int64_t* outv_prefix,
                            const unsigned char* TA, const unsigned char* TB, float* out) {
    const int64_t total = outv_prefix[count];
    for (int64_t t0 = blockIdx.x * TILE_VECS; t0 < total; t0 += (int64_t)gridDim.x * TILE_VECS) {
        const int64_t t1 = min(total, t0 + TILE_VECS);
        if (t0 + threadIdx.x >= t1) continue;
        int g = find_graph(outv_prefix, count, t0 + threadIdx.x);
        for (int64_t u = t0 + threadIdx.x; u < t1; u += blockDim.x) {
            while (outv_prefix[g + 1] <= u) ++g;
            const GDesc& G = gd[g];
            const int64_t e = (u - outv_prefix[g]) * 4;
            const unsigned char* src = ((G.iters & 1) ? TB : TA) + G.T_off;
            float4 o;
            if (G.dtype == CLEORA_F32) {
                o = __ldcs(reinterpret_cast<const float4*>(src + e * 4));
            } else {
                const uint2 w = __ldcs(reinterpret_cast<const uint2*>(src + e * 2));
                o.x = __uint_as_float(w.x << 16);
                o.y = __uint_as_float(w.x & 0xffff0000u);
                o.z = __uint_as_float(w.y << 16);
                o.w = __uint_as_float(w.y & 0xffff0000u);
            }
            __stcs(reinterpret_cast<float4*>(out + G.out_off + e), o);
        }
    }
}

int variant_for(const Shape& sh, bool hv) { return variant_of(sh.G, sh.mode, hv); }

cudaError_t launch_family(const Family& f, const BatchArgs& ba, int sms, cudaStream_t s) {
    if (f.dtype == CLEORA_F32)
        return f.vec == 16 ? launch_batch_f32_v16(f.cpl, f.G, f.mode, ba, sms, s, nullptr)
                           : launch_batch_f32_v8(f.cpl, f.G, f.mode, ba, sms, s, nullptr);
    return f.vec == 16 ? launch_batch_bf16_v16(f.cpl, f.G, f.mode, ba, sms, s, nullptr)
                       : launch_batch_bf16_v8(f.cpl, f.G, f.mode, ba, sms, s, nullptr);
}

}  // namespace batch
}  // namespace cleora

struct cleora_batch {
    cleora_ctx* ctx = nullptr;  // internal context: device, stream, memory pool
    std::string err;
    std::vector<cleora::batch::OneGraph> graphs;
    cleora::batch::Packed pk;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_run = 0;
    std::vector<cudaStream_t> fstreams;  // one stream per kernel family
    std::vector<cudaEvent_t> fevents;    // ... and its join event
    cudaEvent_t fork = nullptr;
};

namespace cleora {
namespace batch {
namespace {

int bfail(cleora_batch* b, int st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    b->err = buf;
    return st;
}

// Status from the internal context, with its message copied to the batch.
int from_ctx(cleora_batch* b, int st) {
    if (st != CLEORA_OK) b->err = b->ctx->err;
    return st;
}

void free_graph_arrays(cleora_ctx* c, OneGraph& og) {
    dfree_null(c, og.ids);
    dfree_null(c, og.rowptr);
    dfree_null(c, og.col);
    dfree_null(c, og.val);
    dfree_null(c, og.tasks);
    dfree_null(c, og.split_base);
}

int build_one(cleora_batch* b, const cleora_graph_desc& gd, int on_dev, OneGraph& og) {
    cleora_ctx* c = b->ctx;
    og.d = gd.d;
    og.iters = gd.iters;
    og.seed = gd.seed;
    og.dtype = gd.storage;
    og.shape = shape_for(gd.d, gd.storage, 0, 1);
    if (gd.num_edges == 0) return CLEORA_OK;
    const uint64_t* s = gd.src;
    const uint64_t* t = gd.dst;
    const float* w = gd.weights;
    void *ds = nullptr, *dt = nullptr, *dw = nullptr;
    int rc = CLEORA_OK;
    if (!on_dev) {
        const size_t eb = (size_t)gd.num_edges * 8;
        rc = dalloc_bytes(c, &ds, eb);
        if (!rc) rc = dalloc_bytes(c, &dt, eb);
        if (!rc && w) rc = dalloc_bytes(c, &dw, (size_t)gd.num_edges * 4);
        cudaError_t e = cudaSuccess;
        if (!rc) e = cudaMemcpyAsync(ds, gd.src, eb, cudaMemcpyHostToDevice, c->stream);
        if (!rc && e == cudaSuccess) e = cudaMemcpyAsync(dt, gd.dst, eb, cudaMemcpyHostToDevice, c->stream);
        if (!rc && e == cudaSuccess && w)
            e = cudaMemcpyAsync(dw, w, (size_t)gd.num_edges * 4, cudaMemcpyHostToDevice, c->stream);
        if (!rc && e != cudaSuccess) rc = cuda_fail(c, e, "edge upload", __FILE__, __LINE__);
        s = static_cast<const uint64_t*>(ds);
        t = static_cast<const uint64_t*>(dt);
        w = static_cast<const float*>(dw);
    }
    if (!rc) rc = graph_build_impl(c, s, t, w, gd.num_edges, gd.directed ? 1 : 0);
    if (!rc) rc = plan_build(c, og.split_len, og.task_nnz);
    dfree(c, ds);
    dfree(c, dt);
    dfree(c, dw);
    if (rc) {
        plan_release(c);
        graph_release(c);
        return from_ctx(b, rc);
    }
    Graph& g = c->g;
    og.n = g.n;
    og.nnz = g.nnz;
    og.has_val = g.has_val;
    og.ids = g.ids;
    og.rowptr = g.rowptr;
    og.col = g.col;
    og.val = g.val;
    dfree(c, g.inv_deg);
    dfree(c, g.deg);
    g = Graph();
    Plan& p = c->plan;
    og.tasks = p.tasks;
    og.ntasks = p.ntasks;
    og.nsplit_rows = p.nsplit_rows;
    og.nsplit_chunks = p.nsplit_chunks;
    og.split_base = p.split_base;
    dfree(c, p.split_count);
    dfree(c, p.counter);
    dfree(c, p.partials);
    p = Plan();
    return CLEORA_OK;
}

void release_packed(cleora_ctx* c, Packed& pk) {
    dfree(c, pk.gd);
    dfree(c, pk.ids);
    dfree(c, pk.rowptr);
    dfree(c, pk.col);
    dfree(c, pk.val);
    dfree(c, pk.TA);
    dfree(c, pk.TB);
    dfree(c, pk.partials);
    dfree(c, pk.split_base);
    dfree(c, pk.split_count);
    dfree(c, pk.out);
    dfree(c, pk.vec_prefix);
    dfree(c, pk.outv_prefix);
    dfree(c, pk.counters);
    for (Family& f : pk.fams) dfree(c, f.tasks);
    pk = Packed();
}

// Packs the listed graphs (indices into b->graphs) with their current shapes.
int pack(cleora_batch* b, const std::vector<int>& which, Packed& pk) {
    cleora_ctx* c = b->ctx;
    cudaStream_t s = c->stream;
    const int sms = c->num_sms;
    std::vector<int> order(which);
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return b->graphs[x].iters > b->graphs[y].iters; });
    pk = Packed();
    pk.count = (int)order.size();
    pk.slot_of.assign(b->graphs.size(), -1);
    std::map<std::tuple<int, int, int, int, int, int>, int> fam_index;
    std::vector<int64_t> vecp(pk.count + 1, 0), outp(pk.count + 1, 0);
    int64_t split_off = 0, partial_off = 0;
    for (int k = 0; k < pk.count; ++k) {
        const OneGraph& og = b->graphs[order[k]];
        pk.slot_of[order[k]] = k;
        const int es = og.dtype == CLEORA_F32 ? 4 : 2;
        auto key = std::make_tuple((int)og.dtype, og.shape.vec, og.shape.cpl, og.shape.G, og.shape.mode,
                                   og.has_val ? 1 : 0);
        auto it = fam_index.find(key);
        int fam;
        if (it == fam_index.end()) {
            fam = (int)pk.fams.size();
            fam_index[key] = fam;
            Family f;
            f.dtype = og.dtype;
            f.vec = og.shape.vec;
            f.cpl = og.shape.cpl;
            f.G = og.shape.G;
            f.mode = og.shape.mode;
            f.hv = og.has_val ? 1 : 0;
            pk.fams.push_back(f);
        } else {
            fam = it->second;
        }
        GDesc G;
        memset(&G, 0, sizeof(G));
        G.node_off = pk.total_n;
        G.n = og.n;
        G.T_off = pk.T_bytes;
        G.out_off = pk.total_out;
        G.split_off = split_off;
        G.partial_off = partial_off;
        G.split_len = og.split_len;
        G.mseed = mix64(og.seed);
        G.d = og.d;
        G.row_bytes = og.d * es;
        G.chunks = og.shape.chunks;
        G.iters = og.iters;
        G.variant = variant_for(og.shape, og.has_val);
        G.dtype = og.dtype;
        G.family = fam;
        pk.hgd.push_back(G);
        pk.total_n += og.n;
        pk.total_nnz += og.nnz;
        pk.total_out += og.n * og.d;
        pk.T_bytes += og.n * og.d * es;
        split_off += og.nsplit_rows;
        partial_off += og.nsplit_chunks * og.d;
        pk.max_iters = std::max(pk.max_iters, og.iters);
        vecp[k + 1] = vecp[k] + og.n * og.d * es / 16;
        outp[k + 1] = outp[k] + og.n * og.d / 4;
        pk.fams[fam].ntasks += og.ntasks;
    }
    int rc = CLEORA_OK;
#define PK(x) do { if ((rc = (x)) != CLEORA_OK) { release_packed(c, pk); return from_ctx(b, rc); } } while (0)
#define PKC(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) { rc = cuda_fail(c, e_, #x, __FILE__, __LINE__); release_packed(c, pk); return from_ctx(b, rc); } } while (0)
    PK(dalloc(c, &pk.gd, (size_t)std::max(pk.count, 1)));
    PK(dalloc(c, &pk.ids, (size_t)std::max<int64_t>(pk.total_n, 1)));
    PK(dalloc(c, &pk.rowptr, (size_t)(pk.total_n + 1)));
    PK(dalloc(c, &pk.col, (size_t)std::max<int64_t>(pk.total_nnz, 1)));
    PK(dalloc(c, &pk.val, (size_t)std::max<int64_t>(pk.total_nnz, 1)));
    PK(dalloc_bytes(c, reinterpret_cast<void**>(&pk.TA), (size_t)std::max<int64_t>(pk.T_bytes, 16)));
    PK(dalloc_bytes(c, reinterpret_cast<void**>(&pk.TB), (size_t)std::max<int64_t>(pk.T_bytes, 16)));
    PK(dalloc(c, &pk.partials, (size_t)std::max<int64_t>(partial_off, 1)));
    PK(dalloc(c, &pk.split_base, (size_t)std::max<int64_t>(split_off, 1)));
    PK(dalloc(c, &pk.split_count, (size_t)std::max<int64_t>(split_off, 1)));
    PK(dalloc(c, &pk.out, (size_t)std::max<int64_t>(pk.total_out, 4)));
    PK(dalloc(c, &pk.vec_prefix, (size_t)(pk.count + 1)));
    PK(dalloc(c, &pk.outv_prefix, (size_t)(pk.count + 1)));
    PK(dalloc(c, &pk.counters, pk.fams.size() * (size_t)(pk.max_iters + 1) + 1));
    for (Family& f : pk.fams) PK(dalloc(c, &f.tasks, (size_t)std::max<int64_t>(f.ntasks, 1)));
    PKC(cudaMemsetAsync(pk.split_count, 0, sizeof(int32_t) * std::max<int64_t>(split_off, 1), s));
    PKC(cudaMemsetAsync(pk.rowptr, 0, sizeof(int64_t), s));
    std::vector<int64_t> fam_fill(pk.fams.size(), 0);
    int64_t nnz_off = 0;
    for (int k = 0; k < pk.count; ++k) {
        const OneGraph& og = b->graphs[order[k]];
        const GDesc& G = pk.hgd[k];
        if (og.n > 0) {
            PKC(cudaMemcpyAsync(pk.ids + G.node_off, og.ids, og.n * 8, cudaMemcpyDeviceToDevice, s));
            k_shift<<<grid_for(og.n + 1, 256, sms), 256, 0, s>>>(pk.rowptr + G.node_off, og.rowptr, og.n + 1, nnz_off);
            PKC(cudaGetLastError());
            if (og.nnz) PKC(cudaMemcpyAsync(pk.col + nnz_off, og.col, og.nnz * 4, cudaMemcpyDeviceToDevice, s));
            if (og.nnz && og.has_val)
                PKC(cudaMemcpyAsync(pk.val + nnz_off, og.val, og.nnz * 4, cudaMemcpyDeviceToDevice, s));
            if (og.nsplit_rows)
                PKC(cudaMemcpyAsync(pk.split_base + G.split_off, og.split_base, og.nsplit_rows * 8,
                                    cudaMemcpyDeviceToDevice, s));
            if (og.ntasks) {
                Family& f = pk.fams[G.family];
                k_wrap_tasks<<<grid_for(og.ntasks, 256, sms), 256, 0, s>>>(f.tasks + fam_fill[G.family], og.tasks,
                                                                          og.ntasks, k);
                PKC(cudaGetLastError());
                fam_fill[G.family] += og.ntasks;
            }
        }
        nnz_off += og.nnz;
    }
    // tasks still active at step s: slots are sorted by iters, so count per family
    for (Family& f : pk.fams) f.nt_step.assign(pk.max_iters + 1, 0);
    for (int k = 0; k < pk.count; ++k) {
        const OneGraph& og = b->graphs[order[k]];
        for (int st = 1; st <= og.iters; ++st) pk.fams[pk.hgd[k].family].nt_step[st] += og.ntasks;
    }
    PKC(cudaMemcpyAsync(pk.gd, pk.hgd.data(), sizeof(GDesc) * pk.count, cudaMemcpyHostToDevice, s));
    PKC(cudaMemcpyAsync(pk.vec_prefix, vecp.data(), 8 * vecp.size(), cudaMemcpyHostToDevice, s));
    PKC(cudaMemcpyAsync(pk.outv_prefix, outp.data(), 8 * outp.size(), cudaMemcpyHostToDevice, s));
    PKC(cudaStreamSynchronize(s));  // host vectors above must outlive the copies
#undef PK
#undef PKC
    return CLEORA_OK;
}

// Enqueues counter reset, init (optional), steps [s0, s1], output (optional).
int enqueue(cleora_batch* b, Packed& pk, bool init, int s0, int s1, bool out, int64_t* launches) {
    cleora_ctx* c = b->ctx;
    cudaStream_t s = c->stream;
    const int sms = c->num_sms;
    int64_t nl = 0;
    cudaError_t e = cudaMemsetAsync(pk.counters, 0,
                                    sizeof(unsigned long long) * (pk.fams.size() * (pk.max_iters + 1) + 1), s);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "counter reset", __FILE__, __LINE__));
    if (init && pk.T_bytes > 0) {
        k_batch_init<<<tile_grid(pk.T_bytes / 16, sms), 256, 0, s>>>(pk.gd, pk.count, pk.vec_prefix, pk.ids, pk.TA);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "batch init", __FILE__, __LINE__));
    }
    // Families are independent (disjoint graphs, own counters): each runs its steps on its own
    // stream, forked from and joined back to the batch stream, so small families overlap.
    if ((int)b->fstreams.size() < (int)pk.fams.size()) {
        while ((int)b->fstreams.size() < (int)pk.fams.size()) {
            cudaStream_t fs = nullptr;
            cudaEvent_t ev = nullptr;
            if ((e = cudaStreamCreateWithFlags(&fs, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return from_ctx(b, cuda_fail(c, e, "family stream", __FILE__, __LINE__));
            b->fstreams.push_back(fs);
            b->fevents.push_back(ev);
        }
    }
    if (b->fork == nullptr && (e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
        return from_ctx(b, cuda_fail(c, e, "fork event", __FILE__, __LINE__));
    if ((e = cudaEventRecord(b->fork, s)) != cudaSuccess)
        return from_ctx(b, cuda_fail(c, e, "fork", __FILE__, __LINE__));
    for (size_t f = 0; f < pk.fams.size(); ++f)
        if ((e = cudaStreamWaitEvent(b->fstreams[f], b->fork, 0)) != cudaSuccess)
            return from_ctx(b, cuda_fail(c, e, "fork", __FILE__, __LINE__));
    for (int st = s0; st <= s1; ++st) {
        for (size_t f = 0; f < pk.fams.size(); ++f) {
            const Family& fam = pk.fams[f];
            if (fam.nt_step[st] == 0) continue;
            BatchArgs ba;
            ba.gd = pk.gd;
            ba.tasks = fam.tasks;
            ba.ntasks = fam.nt_step[st];
            ba.counter = pk.counters + f * (pk.max_iters + 1) + st;
            ba.rowptr = pk.rowptr;
            ba.col = pk.col;
            ba.val = pk.val;
            ba.TA = pk.TA;
            ba.TB = pk.TB;
            ba.total_nnz = pk.total_nnz;
            ba.split_base = pk.split_base;
            ba.split_count = pk.split_count;
            ba.partials = pk.partials;
            ba.err = c->err_flag;
            ba.step = st;
            ba.hv = fam.hv;
            ++nl;
            if ((e = launch_family(fam, ba, sms, b->fstreams[f])) != cudaSuccess)
                return from_ctx(b, cuda_fail(c, e, "batch step", __FILE__, __LINE__));
        }
    }
    for (size_t f = 0; f < pk.fams.size(); ++f) {  // join
        if ((e = cudaEventRecord(b->fevents[f], b->fstreams[f])) != cudaSuccess ||
            (e = cudaStreamWaitEvent(s, b->fevents[f], 0)) != cudaSuccess)
            return from_ctx(b, cuda_fail(c, e, "join", __FILE__, __LINE__));
    }
    if (out && pk.total_out > 0) {
        k_batch_out<<<tile_grid(pk.total_out / 4, sms), 256, 0, s>>>(pk.gd, pk.count, pk.outv_prefix, pk.TA,
                                                                         pk.TB, pk.out);
        ++nl;
        if ((e = cudaGetLastError()) != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "batch output", __FILE__, __LINE__));
    }
    if (launches) *launches = nl;
    c->launches += nl;
    return CLEORA_OK;
}

// Candidate schedules of a (d, storage) class: 16/8-byte gathers x row modes.
std::vector<Shape> candidates(int d, cleora_dtype dt) {
    std::vector<Shape> out;
    for (int vec : {16, 8})
        for (int mode : {1, 2}) {
            Shape sh = shape_for(d, dt, vec, mode);
            bool dup = false;
            for (const Shape& o : out)
                dup |= (o.vec == sh.vec && o.G == sh.G && o.cpl == sh.cpl && o.mode == sh.mode);
            if (!dup) out.push_back(sh);
        }
    return out;
}

// Times one step of a sample of each class under every candidate; keeps the fastest.
int autotune(cleora_batch* b) {
    cleora_ctx* c = b->ctx;
    std::map<std::pair<int, int>, std::vector<int>> classes;
    for (int i = 0; i < (int)b->graphs.size(); ++i) {
        const OneGraph& og = b->graphs[i];
        if (og.iters >= 1 && og.nnz > 0) classes[{(int)og.dtype, og.d}].push_back(i);
    }
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, CLEORA_ERR_CUDA, "event creation failed");
    int rc = CLEORA_OK;
    for (auto& kv : classes) {
        const int dt = kv.first.first, d = kv.first.second;
        std::vector<int>& members = kv.second;
        std::vector<Shape> cands = candidates(d, (cleora_dtype)dt);
        if (cands.size() < 2) continue;
        // sample: graphs spread over the class's sizes holding up to 200M entries -- the whole
        // class when it is smaller -- so that its embeddings, like the batch's, outgrow L2 and
        // the candidates are timed in the memory regime they will run in
        std::vector<int> byn(members);
        std::sort(byn.begin(), byn.end(), [&](int x, int y) { return b->graphs[x].nnz < b->graphs[y].nnz; });
        std::vector<int> sample;
        int64_t class_nnz = 0;
        for (int i : byn) class_nnz += b->graphs[i].nnz;
        const int64_t cap = 200000000;
        const int want = class_nnz <= cap ? (int)byn.size()
                                          : std::max<int>(1, (int)((double)byn.size() * cap / class_nnz));
        int64_t nnz_sum = 0;
        for (int k = 0; k < want; ++k) {
            const int idx = byn[(size_t)k * byn.size() / want];
            if (nnz_sum > cap && !sample.empty()) break;
            sample.push_back(idx);
            nnz_sum += b->graphs[idx].nnz;
        }
        float best = 1e30f;
        Shape best_sh = cands[0];
        for (const Shape& sh : cands) {
            for (int i : sample) b->graphs[i].shape = sh;
            Packed mini;
            if ((rc = pack(b, sample, mini)) != CLEORA_OK) break;
            float ms = 0.f;
            rc = enqueue(b, mini, true, 1, 1, false, nullptr);  // warm-up
            for (int rep = 0; rep < 5 && rc == CLEORA_OK; ++rep) {
                cudaEventRecord(e0, c->stream);
                rc = enqueue(b, mini, false, 1, 1, false, nullptr);
                cudaEventRecord(e1, c->stream);
                cudaEventSynchronize(e1);
                float t = 0.f;
                cudaEventElapsedTime(&t, e0, e1);
                ms += t;
            }
            release_packed(c, mini);
            if (rc != CLEORA_OK) break;
            if (ms < best) {
                best = ms;
                best_sh = sh;
            }
        }
        if (rc != CLEORA_OK) break;
        for (int i : members) b->graphs[i].shape = best_sh;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(c->stream);
    return rc;
}

int capture(cleora_batch* b) {
    cleora_ctx* c = b->ctx;
    cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "begin capture", __FILE__, __LINE__));
    int rc = enqueue(b, b->pk, true, 1, b->pk.max_iters, true, &b->launches_per_run);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(c->stream, &g);
    if (rc != CLEORA_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "end capture", __FILE__, __LINE__));
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, g, 0);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "graph instantiate", __FILE__, __LINE__));
    return CLEORA_OK;
}

}  // namespace
}  // namespace batch
}  // namespace cleora

using namespace cleora;
using namespace cleora::batch;

extern "C" {

void cleora_batch_destroy(cleora_batch* b) {
    if (!b) return;
    if (b->ctx) {
        DeviceGuard guard(b->ctx->device);
        cudaStreamSynchronize(b->ctx->stream);
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        for (cudaStream_t fs : b->fstreams) cudaStreamDestroy(fs);
        for (cudaEvent_t ev : b->fevents) cudaEventDestroy(ev);
        if (b->fork) cudaEventDestroy(b->fork);
        for (OneGraph& og : b->graphs) free_graph_arrays(b->ctx, og);
        release_packed(b->ctx, b->pk);
        cleora_destroy(b->ctx);
    }
    delete b;
}

const char* cleora_batch_last_error(const cleora_batch* b) { return b ? b->err.c_str() : "null batch"; }

int cleora_batch_create(cleora_batch** out, int device, void* cuda_stream, const cleora_graph_desc* graphs,
                        int count, int inputs_on_device, int autotune_flag) {
    if (!out || count < 0 || (count > 0 && !graphs)) return CLEORA_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; ++i) {
        const cleora_graph_desc& g = graphs[i];
        if (g.num_edges < 0 || (g.num_edges > 0 && (!g.src || !g.dst)) || g.d < 8 || g.d > 1024 ||
            g.d % 8 || g.iters < 0 || (g.storage != CLEORA_F32 && g.storage != CLEORA_BF16))
            return CLEORA_ERR_INVALID_ARG;
    }
    cleora_batch* b = new (std::nothrow) cleora_batch();
    if (!b) return CLEORA_ERR_OOM;
    int rc = cleora_create(&b->ctx, device, cuda_stream);
    if (rc != CLEORA_OK) {
        delete b;
        return rc;
    }
    DeviceGuard guard(device);
    b->graphs.resize(count);
    for (int i = 0; i < count && rc == CLEORA_OK; ++i) rc = build_one(b, graphs[i], inputs_on_device, b->graphs[i]);
    if (rc == CLEORA_OK && autotune_flag) rc = autotune(b);
    if (rc == CLEORA_OK) {
        std::vector<int> all(count);
        for (int i = 0; i < count; ++i) all[i] = i;
        rc = pack(b, all, b->pk);
    }
    if (rc == CLEORA_OK) {
        for (OneGraph& og : b->graphs) free_graph_arrays(b->ctx, og);
        cudaError_t e = cudaStreamSynchronize(b->ctx->stream);
        if (e != cudaSuccess) rc = from_ctx(b, cuda_fail(b->ctx, e, "pack", __FILE__, __LINE__));
    }
    if (rc == CLEORA_OK) rc = capture(b);
    if (rc != CLEORA_OK) {
        // keep the message for the caller through the status only: the batch is destroyed
        cleora_batch_destroy(b);
        return rc;
    }
    *out = b;
    return CLEORA_OK;
}

int cleora_batch_totals(const cleora_batch* b, int64_t* nodes, int64_t* nnz, int64_t* out_elems, int* max_iters) {
    if (!b) return CLEORA_ERR_INVALID_ARG;
    if (nodes) *nodes = b->pk.total_n;
    if (nnz) *nnz = b->pk.total_nnz;
    if (out_elems) *out_elems = b->pk.total_out;
    if (max_iters) *max_iters = b->pk.max_iters;
    return CLEORA_OK;
}

int cleora_batch_graph_info(const cleora_batch* b, int g, int64_t* n, int64_t* nnz, int64_t* out_offset) {
    if (!b || g < 0 || g >= (int)b->graphs.size()) return CLEORA_ERR_INVALID_ARG;
    const int k = b->pk.slot_of[g];
    if (n) *n = b->graphs[g].n;
    if (nnz) *nnz = b->graphs[g].nnz;
    if (out_offset) *out_offset = b->pk.hgd[k].out_off;
    return CLEORA_OK;
}

int cleora_batch_schedule(const cleora_batch* b, int g, int64_t* vec_bytes, int64_t* row_mode, int64_t* split_len,
                          int64_t* task_nnz) {
    if (!b || g < 0 || g >= (int)b->graphs.size()) return CLEORA_ERR_INVALID_ARG;
    const OneGraph& og = b->graphs[g];
    if (vec_bytes) *vec_bytes = og.shape.vec;
    if (row_mode) *row_mode = og.shape.mode;
    if (split_len) *split_len = og.split_len;
    if (task_nnz) *task_nnz = og.task_nnz;
    return CLEORA_OK;
}

int cleora_batch_node_ids(cleora_batch* b, int g, uint64_t* out, int out_on_device) {
    if (!b || g < 0 || g >= (int)b->graphs.size()) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(b->ctx->device);
    const int64_t n = b->graphs[g].n;
    if (n == 0) return CLEORA_OK;
    if (!out) return bfail(b, CLEORA_ERR_INVALID_ARG, "null output");
    const GDesc& G = b->pk.hgd[b->pk.slot_of[g]];
    cudaError_t e = cudaMemcpyAsync(out, b->pk.ids + G.node_off, n * 8,
                                    out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->ctx->stream);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(b->ctx, e, "node ids", __FILE__, __LINE__));
    return CLEORA_OK;
}

int cleora_batch_run(cleora_batch* b, float* out, int out_on_device) {
    if (!b) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(b->ctx->device);
    cleora_ctx* c = b->ctx;
    cudaError_t e = cudaGraphLaunch(b->exec, c->stream);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "graph launch", __FILE__, __LINE__));
    c->launches += b->launches_per_run;
    if (out && b->pk.total_out > 0) {
        e = cudaMemcpyAsync(out, b->pk.out, b->pk.total_out * 4,
                            out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "output copy", __FILE__, __LINE__));
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return from_ctx(b, cuda_fail(c, e, "batch run", __FILE__, __LINE__));
    int flag = 0;
    e = read_back(c, &flag, c->err_flag, sizeof(int), c->stream);
    if (e == cudaSuccess && flag) {
        cudaMemset(c->err_flag, 0, sizeof(int));
        return bfail(b, CLEORA_ERR_DEVICE, "a kernel reported an inconsistency (flag %d)", flag);
    }
    return CLEORA_OK;
}

int cleora_batch_launches(const cleora_batch* b, int64_t* launches) {
    if (!b || !launches) return CLEORA_ERR_INVALID_ARG;
    *launches = b->launches_per_run;
    return CLEORA_OK;
}

}  // extern "C"
