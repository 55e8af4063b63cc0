// Identifier hashing and hypergraph expansion on the GPU (arXiv 2102.02302, Sec. 4.3: entity
// identifiers are hashed with xxhash into a small fixed-width format; Sec. 3.2 "Hypergraph
// Expansion": clique and star expansion break hyperedges into pairwise edges).
//
//  * cleora_hash_ids: XXH64 (xxHash specification, 64-bit variant) of every string, a thread
//    per string, bytes read one at a time (any alignment, little-endian lanes).
//  * cleora_expand_hypergraph / cleora_hypergraph_build: each hyperedge's members are sorted
//    (segmented radix sort), repeated members dropped, and the distinct members u_0 < ... <
//    u_{k-1} (ascending id) give the clique edges (u_i, u_j), i < j, in lexicographic order
//    (k(k-1)/2 per hyperedge), or the star edges (s_h, u_i) (k per hyperedge) with s_h the
//    hyperedge's star node.  Hyperedges keep their order, so the edge list is fully determined.
#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_reduce.cuh>
#include <cub/device/device_segmented_sort.cuh>
#include <cub/device/device_select.cuh>

#include "common.cuh"

namespace cleora {
namespace hyper {
namespace {

constexpr uint64_t P1 = 0x9E3779B185EBCA87ull, P2 = 0xC2B2AE3D27D4EB4Full, P3 = 0x165667B19E3779F9ull,
                   P4 = 0x85EBCA77C2B2AE63ull, P5 = 0x27D4EB2F165667C5ull;
constexpr uint64_t STAR_KEY = 0x5354415253544152ull;  // "STARSTAR"

__device__ __forceinline__ uint64_t rotl(uint64_t x, int r) { return (x << r) | (x >> (64 - r)); }

__device__ __forceinline__ uint64_t load_le(const uint8_t* p, int bytes) {
    uint64_t v = 0;
    for (int i = bytes - 1; i >= 0; --i) v = (v << 8) | p[i];
    return v;
}

__device__ __forceinline__ uint64_t lane_round(uint64_t acc, uint64_t lane) {
    return rotl(acc + lane * P2, 31) * P1;
}

__device__ uint64_t xxh64(const uint8_t* p, int64_t len, uint64_t seed) {
    int64_t i = 0;
    uint64_t h;
    if (len >= 32) {
        uint64_t v1 = seed + P1 + P2, v2 = seed + P2, v3 = seed, v4 = seed - P1;
        while (i + 32 <= len) {
            v1 = lane_round(v1, load_le(p + i, 8));
            v2 = lane_round(v2, load_le(p + i + 8, 8));
            v3 = lane_round(v3, load_le(p + i + 16, 8));
            v4 = lane_round(v4, load_le(p + i + 24, 8));
            i += 32;
        }
        h = rotl(v1, 1) + rotl(v2, 7) + rotl(v3, 12) + rotl(v4, 18);
        const uint64_t vs[4] = {v1, v2, v3, v4};
#pragma unroll
        for (int k = 0; k < 4; ++k) h = (h ^ lane_round(0, vs[k])) * P1 + P4;
    } else {
        h = seed + P5;
    }
    h += (uint64_t)len;
    while (i + 8 <= len) {
        h = rotl(h ^ lane_round(0, load_le(p + i, 8)), 27) * P1 + P4;
        i += 8;
    }
    if (i + 4 <= len) {
        h = rotl(h ^ (load_le(p + i, 4) * P1), 23) * P2 + P3;
        i += 4;
    }
    while (i < len) {
        h = rotl(h ^ ((uint64_t)p[i] * P5), 11) * P1;
        ++i;
    }
    h = (h ^ (h >> 33)) * P2;
    h = (h ^ (h >> 29)) * P3;
    return h ^ (h >> 32);
}

__global__ void k_hash(const uint8_t* bytes, const int64_t* offsets, int64_t count, uint64_t seed, uint64_t* out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x)
        out[k] = xxh64(bytes + offsets[k], offsets[k + 1] - offsets[k], seed);
}

// First position of every non-empty hyperedge.
__global__ void k_starts(const int64_t* hoff, int64_t H, uint8_t* start) {
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H;
         h += (int64_t)gridDim.x * blockDim.x)
        if (hoff[h] < hoff[h + 1]) start[hoff[h]] = 1;
}

// 1 for the first occurrence of a member in its (sorted) hyperedge.
__global__ void k_distinct(const uint64_t* sorted, const uint8_t* start, int64_t M, uint8_t* flag, int64_t* flag64) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < M;
         i += (int64_t)gridDim.x * blockDim.x) {
        const bool f = start[i] || sorted[i] != sorted[i - 1];
        flag[i] = f ? 1 : 0;
        flag64[i] = f ? 1 : 0;
    }
}

__global__ void k_edge_counts(const int64_t* kd, int64_t H, int star, int64_t* cnt) {
    for (int64_t h = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; h < H;
         h += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = kd[h];
        cnt[h] = star ? k : k * (k - 1) / 2;
    }
}

// Hyperedge holding distinct-member position q: the last h with uoff[h] <= q.
__device__ __forceinline__ int64_t owner(const int64_t* uoff, int64_t H, int64_t q) {
    int64_t lo = 0, hi = H - 1;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (uoff[mid] <= q) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void k_clique(const uint64_t* U, int64_t Mu, const int64_t* uoff, const int64_t* kd, const int64_t* eoff,
                         int64_t H, uint64_t* src, uint64_t* dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Mu;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = owner(uoff, H, q);
        const int64_t i = q - uoff[h], k = kd[h];
        int64_t e = eoff[h] + i * (2 * k - i - 1) / 2;  // pairs (i', j) with i' < i come first
        const uint64_t a = U[q];
        for (int64_t j = i + 1; j < k; ++j, ++e) {
            src[e] = a;
            dst[e] = U[uoff[h] + j];
        }
    }
}

__global__ void k_star(const uint64_t* U, int64_t Mu, const int64_t* uoff, int64_t H, const uint64_t* star_ids,
                       uint64_t* src, uint64_t* dst) {
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < Mu;
         q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t h = owner(uoff, H, q);
        src[q] = star_ids ? star_ids[h] : mix64((uint64_t)h ^ STAR_KEY);
        dst[q] = U[q];
    }
}

int upload(cleora_ctx* ctx, const void* p, size_t bytes, int on_device, const void** dev, void** owned) {
    *owned = nullptr;
    *dev = p;
    if (on_device || !p || bytes == 0) return CLEORA_OK;
    CL_TRY(dalloc_bytes(ctx, owned, bytes));
    CL_CUDA(ctx, cudaMemcpyAsync(*owned, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *dev = *owned;
    return CLEORA_OK;
}

// Expansion into pool buffers *src, *dst (device) with *E edges.
int expand(cleora_ctx* ctx, const uint64_t* members, const int64_t* hoff, int64_t H, int mode, const uint64_t* star_ids,
           int on_device, uint64_t** src_out, uint64_t** dst_out, int64_t* E_out) {
    *src_out = *dst_out = nullptr;
    *E_out = 0;
    if (H < 0 || (mode != CLEORA_EXPAND_CLIQUE && mode != CLEORA_EXPAND_STAR) || (H > 0 && !hoff))
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "bad hypergraph arguments");
    if (H == 0) return CLEORA_OK;
    if (H >= ((int64_t)1 << 31)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "more than 2^31 - 1 hyperedges");
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    int64_t M = 0, first = 0;
    if (on_device) {
        CL_CUDA(ctx, read_back(ctx, &M, hoff + H, 8, s));
        CL_CUDA(ctx, read_back(ctx, &first, hoff, 8, s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
    } else {
        M = hoff[H];
        first = hoff[0];
    }
    if (first != 0 || M < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "hyperedge offsets must start at 0");
    if (M > 0 && !members) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null members");
    const void *dm = nullptr, *dh = nullptr, *ds = nullptr;
    void *om = nullptr, *oh = nullptr, *os = nullptr;
    uint64_t *sorted = nullptr, *U = nullptr, *src = nullptr, *dst = nullptr;
    uint8_t *start = nullptr, *flag = nullptr;
    int64_t *flag64 = nullptr, *kd = nullptr;
    int64_t *uoff = nullptr, *cnt = nullptr, *eoff = nullptr, *scal = nullptr;
    void* tmp = nullptr;
    int rc = CLEORA_OK;
    auto cub_tmp = [&](size_t bytes) -> int {
        dfree(ctx, tmp);
        tmp = nullptr;
        return dalloc_bytes(ctx, &tmp, bytes ? bytes : 1);
    };
    do {
        if ((rc = upload(ctx, members, (size_t)M * 8, on_device, &dm, &om))) break;
        if ((rc = upload(ctx, hoff, (size_t)(H + 1) * 8, on_device, &dh, &oh))) break;
        if (mode == CLEORA_EXPAND_STAR && (rc = upload(ctx, star_ids, (size_t)H * 8, on_device, &ds, &os))) break;
        const int64_t* d_hoff = static_cast<const int64_t*>(dh);
        if ((rc = dalloc(ctx, &kd, (size_t)H))) break;
        if ((rc = dalloc(ctx, &uoff, (size_t)(H + 1)))) break;
        if ((rc = dalloc(ctx, &cnt, (size_t)H))) break;
        if ((rc = dalloc(ctx, &eoff, (size_t)(H + 1)))) break;
        if ((rc = dalloc(ctx, &scal, 1))) break;
        int64_t Mu = 0;
        cudaError_t e = cudaSuccess;
        if (M > 0) {
            // members sorted within each hyperedge, first occurrences flagged and kept
            if ((rc = dalloc(ctx, &sorted, (size_t)M))) break;
            if ((rc = dalloc(ctx, &start, (size_t)M))) break;
            if ((rc = dalloc(ctx, &flag, (size_t)M))) break;
            if ((rc = dalloc(ctx, &flag64, (size_t)M))) break;
            if ((rc = dalloc(ctx, &U, (size_t)M))) break;
            size_t tb = 0;
            e = cub::DeviceSegmentedSort::SortKeys(nullptr, tb, static_cast<const uint64_t*>(dm), sorted, M, H, d_hoff,
                                                   d_hoff + 1, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess)
                e = cub::DeviceSegmentedSort::SortKeys(tmp, tb, static_cast<const uint64_t*>(dm), sorted, M, H, d_hoff,
                                                       d_hoff + 1, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(start, 0, (size_t)M, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
            k_starts<<<grid_for(H, 256, sms), 256, 0, s>>>(d_hoff, H, start);
            k_distinct<<<grid_for(M, 256, sms), 256, 0, s>>>(sorted, start, M, flag, flag64);
            ctx->launches += 3;
            tb = 0;
            e = cub::DeviceSegmentedReduce::Sum(nullptr, tb, flag64, kd, H, d_hoff, d_hoff + 1, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess) e = cub::DeviceSegmentedReduce::Sum(tmp, tb, flag64, kd, H, d_hoff, d_hoff + 1, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
            tb = 0;
            e = cub::DeviceSelect::Flagged(nullptr, tb, sorted, flag, U, scal, M, s);
            if (e == cudaSuccess && (rc = cub_tmp(tb))) break;
            if (e == cudaSuccess) e = cub::DeviceSelect::Flagged(tmp, tb, sorted, flag, U, scal, M, s);
            if (e == cudaSuccess) e = read_back(ctx, &Mu, scal, 8, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
            ctx->launches += 2;
        } else {
            e = cudaMemsetAsync(kd, 0, (size_t)H * 8, s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
        }
        // offsets of the distinct members and of the edges
        k_edge_counts<<<grid_for(H, 256, sms), 256, 0, s>>>(kd, H, mode == CLEORA_EXPAND_STAR, cnt);
        ctx->launches++;
        size_t tb = 0;
        e = cub::DeviceScan::ExclusiveSum(nullptr, tb, cnt, eoff, H, s);  // totals: last offset + last count
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
        if ((rc = cub_tmp(tb))) break;
        e = cub::DeviceScan::ExclusiveSum(tmp, tb, cnt, eoff, H, s);
        if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, tb, kd, uoff, H, s);
        int64_t last_e = 0, last_c = 0;
        int64_t last_k = 0, last_u = 0;
        if (e == cudaSuccess) e = read_back(ctx, &last_e, eoff + H - 1, 8, s);
        if (e == cudaSuccess) e = read_back(ctx, &last_c, cnt + H - 1, 8, s);
        if (e == cudaSuccess) e = read_back(ctx, &last_u, uoff + H - 1, 8, s);
        if (e == cudaSuccess) e = read_back(ctx, &last_k, kd + H - 1, 8, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
        ctx->launches += 2;
        const int64_t E = last_e + last_c;
        if (last_u + last_k != Mu) { rc = fail(ctx, CLEORA_ERR_DEVICE, "expansion: member counts disagree"); break; }
        if (E == 0) break;
        if ((rc = dalloc(ctx, &src, (size_t)E))) break;
        if ((rc = dalloc(ctx, &dst, (size_t)E))) break;
        if (mode == CLEORA_EXPAND_CLIQUE)
            k_clique<<<grid_for(Mu, 256, sms), 256, 0, s>>>(U, Mu, uoff, kd, eoff, H, src, dst);
        else
            k_star<<<grid_for(Mu, 256, sms), 256, 0, s>>>(U, Mu, uoff, H, static_cast<const uint64_t*>(ds), src, dst);
        ctx->launches++;
        e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__); break; }
        *src_out = src;
        *dst_out = dst;
        src = dst = nullptr;
        *E_out = E;
    } while (0);
    dfree(ctx, om);
    dfree(ctx, oh);
    dfree(ctx, os);
    dfree(ctx, sorted);
    dfree(ctx, U);
    dfree(ctx, src);
    dfree(ctx, dst);
    dfree(ctx, start);
    dfree(ctx, flag);
    dfree(ctx, flag64);
    dfree(ctx, kd);
    dfree(ctx, uoff);
    dfree(ctx, cnt);
    dfree(ctx, eoff);
    dfree(ctx, scal);
    dfree(ctx, tmp);
    return rc;
}

}  // namespace
}  // namespace hyper
}  // namespace cleora

using namespace cleora;

extern "C" {

int cleora_hash_ids(cleora_ctx* ctx, const uint8_t* bytes, const int64_t* offsets, int64_t count, uint64_t seed,
                    uint64_t* out, int inputs_on_device, int out_on_device) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, CLEORA_ERR_CUDA, "cannot select device %d", ctx->device);
    if (count < 0 || (count > 0 && (!offsets || !out))) return fail(ctx, CLEORA_ERR_INVALID_ARG, "bad hash arguments");
    if (count == 0) return CLEORA_OK;
    cudaStream_t s = ctx->stream;
    int64_t total = 0, first = 0;
    if (inputs_on_device) {
        CL_CUDA(ctx, read_back(ctx, &total, offsets + count, 8, s));
        CL_CUDA(ctx, read_back(ctx, &first, offsets, 8, s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
    } else {
        total = offsets[count];
        first = offsets[0];
    }
    if (first != 0 || total < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "string offsets must start at 0");
    if (total > 0 && !bytes) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null bytes");
    const void *db = nullptr, *doff = nullptr;
    void *ob = nullptr, *ooff = nullptr, *dout = out;
    bool own_out = false;
    int rc = CLEORA_OK;
    do {
        if ((rc = hyper::upload(ctx, bytes, (size_t)total, inputs_on_device, &db, &ob))) break;
        if ((rc = hyper::upload(ctx, offsets, (size_t)(count + 1) * 8, inputs_on_device, &doff, &ooff))) break;
        if (!out_on_device) {
            if ((rc = dalloc_bytes(ctx, &dout, (size_t)count * 8))) break;
            own_out = true;
        }
        hyper::k_hash<<<grid_for(count, 256, ctx->num_sms), 256, 0, s>>>(
            static_cast<const uint8_t*>(db), static_cast<const int64_t*>(doff), count, seed,
            static_cast<uint64_t*>(dout));
        ctx->launches++;
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && own_out) e = cudaMemcpyAsync(out, dout, (size_t)count * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "hash", __FILE__, __LINE__);
    } while (0);
    dfree(ctx, ob);
    dfree(ctx, ooff);
    if (own_out) dfree(ctx, dout);
    cudaStreamSynchronize(s);
    return rc;
}

int cleora_expand_hypergraph(cleora_ctx* ctx, const uint64_t* members, const int64_t* hoff, int64_t num_hyperedges,
                             int mode, const uint64_t* star_ids, int inputs_on_device, uint64_t* src_out,
                             uint64_t* dst_out, int64_t capacity, int64_t* num_edges, int out_on_device) {
    if (!ctx || !num_edges) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, CLEORA_ERR_CUDA, "cannot select device %d", ctx->device);
    *num_edges = 0;
    uint64_t *src = nullptr, *dst = nullptr;
    int64_t E = 0;
    int rc = hyper::expand(ctx, members, hoff, num_hyperedges, mode, star_ids, inputs_on_device, &src, &dst, &E);
    if (rc == CLEORA_OK) {
        *num_edges = E;
        if ((src_out || dst_out) && E > capacity)
            rc = fail(ctx, CLEORA_ERR_INVALID_ARG, "the expansion has %lld edges, capacity %lld", (long long)E,
                      (long long)capacity);
    }
    const cudaMemcpyKind k = out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (rc == CLEORA_OK && E > 0 && src_out) {
        cudaError_t e = cudaMemcpyAsync(src_out, src, (size_t)E * 8, k, ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "expansion copy", __FILE__, __LINE__);
    }
    if (rc == CLEORA_OK && E > 0 && dst_out) {
        cudaError_t e = cudaMemcpyAsync(dst_out, dst, (size_t)E * 8, k, ctx->stream);
        if (e != cudaSuccess) rc = cuda_fail(ctx, e, "expansion copy", __FILE__, __LINE__);
    }
    dfree(ctx, src);
    dfree(ctx, dst);
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (rc == CLEORA_OK && e != cudaSuccess) rc = cuda_fail(ctx, e, "expansion", __FILE__, __LINE__);
    return rc;
}

int cleora_hypergraph_build(cleora_ctx* ctx, const uint64_t* members, const int64_t* hoff, int64_t num_hyperedges,
                            int mode, const uint64_t* star_ids, int inputs_on_device, int64_t* num_edges) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    if (!guard.ok) return fail(ctx, CLEORA_ERR_CUDA, "cannot select device %d", ctx->device);
    uint64_t *src = nullptr, *dst = nullptr;
    int64_t E = 0;
    int rc = hyper::expand(ctx, members, hoff, num_hyperedges, mode, star_ids, inputs_on_device, &src, &dst, &E);
    if (num_edges) *num_edges = E;
    if (rc == CLEORA_OK) rc = cleora_graph_build(ctx, src, dst, nullptr, E, 0, 1);
    dfree(ctx, src);
    dfree(ctx, dst);
    return rc;
}

}  // extern "C"
