// Graph build on the GPU: node ids and the CSR of M = D^-1 A
// (arXiv 2102.02302, Sec. 3.2 "Embedding": M_ab = e_ab / deg(v_a), e_ab the number of
// edges a->b or the sum of their weights; Sec. 4.5: undirected edges count both ways).
//
// Steps (all on the context's stream; sort, unique and compaction use CUB):
//   1. ids   = sorted distinct values of src ++ dst   (node index = rank of the id): a hash
//      set drops the repeats (a power-law edge list names each hub millions of times), and
//      only the distinct ids are sorted; a second hash table maps each id to its rank
//   2. entry keys (a << bits) | b, one per edge (two for an undirected non-loop edge,
//      interleaved 2e, 2e+1 so that a stable sort keeps duplicates in edge order)
//   3. stable radix sort of the keys (weights carried along when weighted)
//   4. runs of equal keys -> col, e_ab (count, or FP64 sum in edge order)
//   5. rowptr from the sorted rows; deg_a = FP64 sum of e_ab in ascending col
//   6. val = fp32(e_ab / deg_a) when needed; inv_deg = 1.0f / fp32(deg_a)
#include <algorithm>
#include <cmath>
#include <vector>

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

// Hash tables of ids.  The all-ones id is the empty-slot marker: it is never stored, and an
// edge list that contains it sets a flag instead (it sorts last, so its rank is n - 1).
constexpr uint64_t EMPTY_ID = ~0ull;

// HyperLogLog sketch of the distinct endpoints (Flajolet, Fusy, Gandouet and Meunier 2007),
// 2^HLL_P registers: register j keeps the largest rank (position of the first one bit) of
// the hashes whose top HLL_P bits are j.  It sizes the id set below.
constexpr int HLL_P = 12;
constexpr int HLL_M = 1 << HLL_P;

__global__ void k_hll(const uint64_t* src, const uint64_t* dst, int64_t E, unsigned int* regs) {
    __shared__ unsigned int r[HLL_M];
    for (int j = threadIdx.x; j < HLL_M; j += blockDim.x) r[j] = 0;
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < 2 * E;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = mix64((i < E ? src[i] : dst[i - E]) ^ 0x6A09E667F3BCC909ull);
        const uint64_t rest = h << HLL_P;
        const unsigned int rho = rest == 0 ? (unsigned int)(64 - HLL_P + 1) : (unsigned int)__clzll(rest) + 1u;
        atomicMax(r + (h >> (64 - HLL_P)), rho);
    }
    __syncthreads();
    for (int j = threadIdx.x; j < HLL_M; j += blockDim.x)
        if (r[j]) atomicMax(regs + j, r[j]);
}

// Distinct-count estimate from the registers (harmonic mean, linear counting when small).
double hll_estimate(const unsigned int* regs) {
    double z = 0.0;
    int zeros = 0;
    for (int j = 0; j < HLL_M; ++j) {
        z += std::ldexp(1.0, -(int)regs[j]);
        zeros += regs[j] == 0;
    }
    const double m = HLL_M;
    const double est = 0.7213 / (1.0 + 1.079 / m) * m * m / z;
    if (est <= 2.5 * m && zeros > 0) return m * std::log(m / zeros);
    return est;
}

// Set of distinct ids: linear probing over S slots.  A slot goes from empty to an id once,
// so a stale empty read only leads to a compare-and-swap that returns the slot's real
// content.  A probe sequence longer than `limit` sets *overflow and drops the id (the caller
// then retries with a table of more slots than ids, where every sequence ends).
__global__ void k_set_insert(const uint64_t* src, const uint64_t* dst, int64_t E, uint64_t* tab, uint64_t S,
                             uint64_t limit, int* has_empty, int* overflow) {
    constexpr int Q = 4;  // ids per thread and pass: their first probes are in flight together
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < 2 * E; i0 += Q * T) {
        uint64_t x[Q], slot[Q], cur[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t i = i0 + q * T;
            x[q] = i < 2 * E ? (i < E ? src[i] : dst[i - E]) : EMPTY_ID;
        }
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            slot[q] = __umul64hi(mix64(x[q] ^ 0x2545F4914F6CDD1Dull), S);
            cur[q] = x[q] != EMPTY_ID ? tab[slot[q]] : EMPTY_ID;
        }
#pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            if (x[q] == EMPTY_ID) {
                if (i0 + q * T < 2 * E) atomicOr(has_empty, 1);
                continue;
            }
            uint64_t s = slot[q], c = cur[q];
            uint64_t probe = 0;
            for (; probe < limit; ++probe) {
                if (c == x[q]) break;
                if (c == EMPTY_ID) {
                    const unsigned long long prev = atomicCAS(reinterpret_cast<unsigned long long*>(tab + s),
                                                              (unsigned long long)EMPTY_ID,
                                                              (unsigned long long)x[q]);
                    if (prev == EMPTY_ID || prev == x[q]) break;
                }
                s = (s + 1 == S) ? 0 : s + 1;
                c = tab[s];
            }
            if (probe == limit) atomicOr(overflow, 1);
        }
    }
}

struct NotEmptyId {
    __device__ __forceinline__ bool operator()(uint64_t x) const { return x != EMPTY_ID; }
};

// id -> rank table: 2^k slots of {id, rank} (at least twice the ids), linear probing.
__global__ void k_rank_insert(const uint64_t* ids, int64_t n, ulonglong2* tab, uint64_t mask) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t x = ids[i];
        if (x == EMPTY_ID) continue;
        uint64_t slot = mix64(x ^ 0x9E6C63D0676A9A99ull) & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
            const unsigned long long prev = atomicCAS(&tab[slot].x, (unsigned long long)EMPTY_ID,
                                                      (unsigned long long)x);
            if (prev == EMPTY_ID) {
                tab[slot].y = (unsigned long long)i;
                break;
            }
            slot = (slot + 1) & mask;
        }
    }
}

// First probe of id x in the id -> rank table (its home slot).
__device__ __forceinline__ ulonglong2 tab_first(const ulonglong2* tab, uint64_t mask, uint64_t x) {
    return tab[mix64(x ^ 0x9E6C63D0676A9A99ull) & mask];
}

// Rank of id x given its home slot's content `v`, or -1 when x is not in the table.
__device__ __forceinline__ int64_t rank_resolve(const ulonglong2* tab, uint64_t mask, uint64_t x, ulonglong2 v,
                                                int64_t n, bool has_empty) {
    if (x == EMPTY_ID) return has_empty ? n - 1 : -1;
    uint64_t slot = mix64(x ^ 0x9E6C63D0676A9A99ull) & mask;
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        if (v.x == x) return (int64_t)v.y;
        if (v.x == EMPTY_ID) return -1;
        slot = (slot + 1) & mask;
        v = tab[slot];
    }
    return -1;
}

// Entry key(s) of edge e from its endpoints' ranks.  `mode`: KEYS_DIRECTED one key (a, b);
// KEYS_PAIR (undirected) keys (a, b) and (b, a) at 2e, 2e + 1 (a self-loop once);
// KEYS_SYM (undirected) one key (min, max), the lower half being built later by transposing.
enum { KEYS_PAIR = 0, KEYS_DIRECTED = 1, KEYS_SYM = 2 };

__device__ __forceinline__ void emit_entry(int64_t e, int64_t ra, int64_t rb, const float* w, int mode,
                                           int bits, uint64_t invalid, uint64_t* keys, float* vals, int* missing) {
    if (ra < 0 || rb < 0) {  // cannot happen: every endpoint went into the table
        atomicOr(missing, 1);
        keys[mode != KEYS_PAIR ? e : 2 * e] = invalid;
        if (mode == KEYS_PAIR) keys[2 * e + 1] = invalid;
        return;
    }
    const uint64_t a = (uint64_t)ra, b = (uint64_t)rb;
    if (mode == KEYS_DIRECTED) {
        keys[e] = (a << bits) | b;
        if (vals) vals[e] = w[e];
    } else if (mode == KEYS_SYM) {
        keys[e] = a <= b ? ((a << bits) | b) : ((b << bits) | a);
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

__global__ void k_entries(const uint64_t* src, const uint64_t* dst, const float* w, int64_t E,
                          int mode, const ulonglong2* rank_tab, uint64_t mask, int64_t n, int has_empty,
                          int bits, uint64_t invalid, uint64_t* keys, float* vals, int* missing) {
    constexpr int Q = 4;  // edges per thread and pass: 2Q first probes in flight together
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e0 < E; e0 += Q * T) {
        uint64_t x[2 * Q];
        ulonglong2 v[2 * Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            const int64_t e = e0 + q * T;
            x[2 * q] = e < E ? src[e] : EMPTY_ID;
            x[2 * q + 1] = e < E ? dst[e] : EMPTY_ID;
        }
#pragma unroll
        for (int i = 0; i < 2 * Q; ++i)
            v[i] = x[i] != EMPTY_ID ? tab_first(rank_tab, mask, x[i]) : make_ulonglong2(EMPTY_ID, 0);
#pragma unroll 1
        for (int q = 0; q < Q; ++q) {
            const int64_t e = e0 + q * T;
            if (e >= E) break;
            const int64_t ra = rank_resolve(rank_tab, mask, x[2 * q], v[2 * q], n, has_empty != 0);
            const int64_t rb = rank_resolve(rank_tab, mask, x[2 * q + 1], v[2 * q + 1], n, has_empty != 0);
            emit_entry(e, ra, rb, w, mode, bits, invalid, keys, vals, missing);
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
        if (vals) {
            double acc = 0.0;
            for (int64_t i = s; i < t; ++i) acc = __dadd_rn(acc, (double)vals[i]);
            e[k] = acc;
        } else if (t - s != 1) {  // unweighted: e_ab = t - s, recomputed from the run starts
            atomicOr(not_unit, 1);
        }
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

// Largest row length: a warp maximum, then one atomic per warp (one atomic per row on the same
// address serialises in L2).  Every lane of the warp calls it.
__device__ __forceinline__ void warp_max_out(unsigned long long* out, unsigned long long v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0 && v) atomicMax(out, v);
}

// Start of run k among the sorted raw entries (run nnz ends at the last valid entry).
__device__ __forceinline__ int64_t run_start(const int64_t* start, int64_t nnz, const int64_t* m_valid, int64_t k) {
    return k < nnz ? start[k] : *m_valid;
}

// Unweighted graphs: e_ab is the length of run k, so deg_a, the sum of the row's e_ab, is
// the number of raw entries from the row's first run start to its last run end (an integer,
// exact in any order).
__global__ void k_degree_int(const int64_t* rowptr, const int64_t* start, int64_t nnz, const int64_t* m_valid,
                             int64_t n, double* deg, float* inv_deg, unsigned long long* max_len) {
    unsigned long long mx = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[r], t = rowptr[r + 1];
        const double s = (double)(run_start(start, nnz, m_valid, t) - run_start(start, nnz, m_valid, b));
        deg[r] = s;
        inv_deg[r] = s > 0.0 ? __fdiv_rn(1.0f, __double2float_rn(s)) : 0.0f;
        mx = max(mx, (unsigned long long)(t - b));
    }
    warp_max_out(max_len, mx);
}

// Weighted graphs: deg_a is the FP64 sum of e_ab in ascending column order, one thread per
// row (the order is part of the bit-exact definition of the stored values).
__global__ void k_degree(const int64_t* rowptr, const double* e, int64_t n, double* deg,
                         float* inv_deg, unsigned long long* max_len) {
    unsigned long long mx = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = rowptr[r], t = rowptr[r + 1];
        double s = 0.0;
        for (int64_t k = b; k < t; ++k) s = __dadd_rn(s, e[k]);
        deg[r] = s;
        inv_deg[r] = s > 0.0 ? __fdiv_rn(1.0f, __double2float_rn(s)) : 0.0f;
        mx = max(mx, (unsigned long long)(t - b));
    }
    warp_max_out(max_len, mx);
}

// val = fp32(e_ab / deg_a); e_ab from the weights' sums, or (unweighted) the run length.
__global__ void k_values(const int32_t* row, const double* e, const int64_t* start, const int64_t* m_valid,
                         const double* deg, int64_t nnz, float* val) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const double ek = e ? e[k] : (double)(run_start(start, nnz, m_valid, k + 1) - start[k]);
        val[k] = __double2float_rn(__ddiv_rn(ek, deg[row[k]]));
    }
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
    void reset() {
        dfree(ctx, p);
        p = nullptr;
    }
    T* release() {
        T* q = p;
        p = nullptr;
        return q;
    }
};

// --- undirected graphs from one (lo, hi) key per edge -----------------------------------
// Row r of the symmetric CSR is [lo < r of the pairs (lo, r)] ++ [the pairs (r, hi), hi >= r]:
// the second part is the sorted unique pairs' run of lo = r; the first part comes from the
// same pairs sorted stably by hi (ascending lo within each hi, as the pairs are sorted by lo).

// Multiplicities of unweighted pairs as FP64 (only when some pair repeats).
__global__ void k_counts_to_e(const int64_t* start, int64_t nu, int64_t m_valid, double* e) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x)
        e[u] = (double)((u + 1 < nu ? start[u + 1] : m_valid) - start[u]);
}

// Keys of the transposed half: hi, or n for a self-loop (no transposed copy; sorts last).
// (the sort's value is the pair index when the pairs carry values, else the lower end itself,
// which the placement then writes without a gather)
__global__ void k_transpose_keys(const int32_t* lo, const int32_t* hi, int64_t nu, uint32_t n, bool by_pair,
                                 uint32_t* tk, uint32_t* tv) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x) {
        tk[u] = lo[u] == hi[u] ? n : (uint32_t)hi[u];
        tv[u] = by_pair ? (uint32_t)u : (uint32_t)lo[u];
    }
}

// Number of sorted keys below n (the transposed entries; self-loop keys n come last).
__global__ void k_count_below(const uint32_t* tk, int64_t nu, uint32_t n, int64_t* out) {
    int64_t lo = 0, hi = nu;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (tk[mid] < n) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

__global__ void k_add_rowptr(const int64_t* a, const int64_t* b, int64_t n, int64_t* out) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r <= n;
         r += (int64_t)gridDim.x * blockDim.x)
        out[r] = a[r] + b[r];
}

// Lower part of each row: transposed entry i (row tk[i]; pair tv[i], or with no values its
// lower end tv[i] itself) at its rank in the row.
__global__ void k_place_low(const uint32_t* tk, const uint32_t* tv, int64_t nt, const int64_t* rowptr,
                            const int64_t* lowptr, const int32_t* lo, const double* e_u, int32_t* col,
                            double* e_out, int32_t* row_out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = tk[i], u = tv[i];
        const int64_t pos = rowptr[r] + (i - lowptr[r]);
        if (e_out) {
            col[pos] = lo[u];
            e_out[pos] = e_u[u];
            row_out[pos] = (int32_t)r;
        } else {
            col[pos] = (int32_t)u;
        }
    }
}

// Upper part (including the self-loop): pair u after the row's lower part.
__global__ void k_place_up(const int32_t* lo, const int32_t* hi, int64_t nu, const int64_t* rowptr,
                           const int64_t* lowptr, const int64_t* upptr, const double* e_u, int32_t* col,
                           double* e_out, int32_t* row_out) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nu;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = lo[u];
        const int64_t pos = rowptr[r] + (lowptr[r + 1] - lowptr[r]) + (u - upptr[r]);
        col[pos] = hi[u];
        if (e_out) e_out[pos] = e_u[u];
        if (row_out) row_out[pos] = (int32_t)r;
    }
}

// Unweighted graphs without repeated pairs: deg_a is the row length.
__global__ void k_degree_len(const int64_t* rowptr, int64_t n, double* deg, float* inv_deg,
                             unsigned long long* max_len) {
    unsigned long long mx = 0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = rowptr[r + 1] - rowptr[r];
        const double s = (double)l;
        deg[r] = s;
        inv_deg[r] = s > 0.0 ? __fdiv_rn(1.0f, __double2float_rn(s)) : 0.0f;
        mx = max(mx, (unsigned long long)l);
    }
    warp_max_out(max_len, mx);
}

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
    dfree_null(ctx, g.hot_bits);
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
        CL_CUDA(ctx, read_back(ctx, &bad, d_flag, sizeof(int), s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        if (bad) return fail(ctx, CLEORA_ERR_INVALID_ARG, "weights must be finite and > 0");
    }

    const int64_t m = directed ? E : 2 * E;  // entries before dedup
    // One buffer of 4E words: first the id set (load <= 1/2), then the two key buffers of
    // the entry sort (2E words each).
    DBuf<uint64_t> kk(ctx);
    CL_TRY(kk.alloc((size_t)(4 * E)));
    uint64_t* ka = kk.p;
    uint64_t* kb = kk.p + 2 * E;

    // 1. ids = sorted distinct endpoints
    int has_empty = 0;
    DBuf<ulonglong2> rank_tab(ctx);
    uint64_t rank_mask = 0;
    {
        // table size: 4x the sketch's distinct estimate (load about 1/4), at most 4E slots;
        // probe sequences are capped unless the table has more slots than there are ids
        const uint64_t S_full = (uint64_t)(4 * E);
        uint64_t S = S_full;
        if (E > 0 && ctx->opt[CLEORA_OPT_ID_SLOTS] > 0) {
            S = std::min<uint64_t>(S_full, (uint64_t)ctx->opt[CLEORA_OPT_ID_SLOTS]);
        } else if (E > 0) {
            DBuf<unsigned int> regs(ctx);
            CL_TRY(regs.alloc(HLL_M));
            CL_CUDA(ctx, cudaMemsetAsync(regs.p, 0, HLL_M * sizeof(unsigned int), s));
            k_hll<<<grid_for(2 * E, 256, sms), 256, 0, s>>>(src, dst, E, regs.p);
            CL_LAUNCHED(ctx);
            std::vector<unsigned int> hr(HLL_M);
            CL_CUDA(ctx, read_back(ctx, hr.data(), regs.p, HLL_M * sizeof(unsigned int), s));
            CL_CUDA(ctx, cudaStreamSynchronize(s));
            const double est = hll_estimate(hr.data());
            uint64_t want = 1 << 16;
            while ((double)want < 4.0 * est) want <<= 1;
            S = std::min(S_full, want);
        }
        int* d_overflow = reinterpret_cast<int*>(scal.p + 2);
        for (int attempt = 0; attempt < 2; ++attempt) {
            CL_CUDA(ctx, cudaMemsetAsync(kk.p, 0xff, S * sizeof(uint64_t), s));
            if (E == 0) break;
            k_set_insert<<<grid_for(2 * E, 256, sms), 256, 0, s>>>(src, dst, E, kk.p, S, S == S_full ? S : 4096,
                                                                    d_flag, d_overflow);
            CL_LAUNCHED(ctx);
            int ovf = 0;
            CL_CUDA(ctx, read_back(ctx, &ovf, d_overflow, sizeof(int), s));
            CL_CUDA(ctx, cudaStreamSynchronize(s));
            if (!ovf) break;
            if (S == S_full) return fail(ctx, CLEORA_ERR_DEVICE, "id set overflow");
            S = S_full;  // the estimate was far off: retry with room for every endpoint
            CL_CUDA(ctx, cudaMemsetAsync(d_overflow, 0, sizeof(int), s));
        }
        // count the distinct ids, then move them out of the table
        DBuf<uint64_t> ua(ctx);
        size_t tb = 0;
        NotEmptyId pred;
        CL_CUDA(ctx, cub::DeviceSelect::If(nullptr, tb, kk.p, scal.p, (int64_t)S, pred, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb));
        // in-place compaction keeps the selected ids in order at the front of the table
        CL_CUDA(ctx, cub::DeviceSelect::If(tmp.p, tb, kk.p, scal.p, (int64_t)S, pred, s));
        int64_t hv[2] = {0, 0};
        CL_CUDA(ctx, read_back(ctx, hv, scal.p, 2 * sizeof(int64_t), s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        has_empty = (int)(hv[1] & 0xffffffff);
        const int64_t n = hv[0] + (has_empty ? 1 : 0);
        if (n >= ((int64_t)1 << 31))
            return fail(ctx, CLEORA_ERR_INVALID_ARG, "graph has %lld nodes; the limit is 2^31-1",
                        (long long)n);
        CL_CUDA(ctx, cudaMemsetAsync(d_flag, 0, sizeof(int), s));
        g.n = n;
        CL_TRY(dalloc(ctx, &g.ids, (size_t)(n ? n : 1)));
        if (hv[0] > 0) {
            CL_TRY(ua.alloc((size_t)hv[0]));
            CL_CUDA(ctx, cudaMemcpyAsync(ua.p, kk.p, hv[0] * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
            cub::DoubleBuffer<uint64_t> db(ua.p, g.ids);
            size_t tsort = 0;
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(nullptr, tsort, db, hv[0], 0, 64, s));
            DBuf<unsigned char> tmps(ctx);
            CL_TRY(tmps.alloc(tsort));
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(tmps.p, tsort, db, hv[0], 0, 64, s));
            if (db.Current() != g.ids)
                CL_CUDA(ctx, cudaMemcpyAsync(g.ids, db.Current(), hv[0] * sizeof(uint64_t),
                                             cudaMemcpyDeviceToDevice, s));
        }
        if (has_empty) {
            const uint64_t e = EMPTY_ID;
            CL_CUDA(ctx, put_bytes(ctx, g.ids + hv[0], &e, sizeof(uint64_t), s));
        }
        // id -> rank table, at least twice as many slots as ids
        uint64_t slots = 2;
        while (slots < 2 * (uint64_t)n) slots <<= 1;
        rank_mask = slots - 1;
        CL_TRY(rank_tab.alloc((size_t)slots));
        CL_CUDA(ctx, cudaMemsetAsync(rank_tab.p, 0xff, slots * sizeof(ulonglong2), s));
        if (n > 0) {
            k_rank_insert<<<grid_for(n, 256, sms), 256, 0, s>>>(g.ids, n, rank_tab.p, rank_mask);
            CL_LAUNCHED(ctx);
        }
        CL_CUDA(ctx, cudaStreamSynchronize(s));  // the host-side copy of the sentinel id is done
    }
    const int64_t n = g.n;

    // 2. entry keys (and weights)
    const int bits = bit_width(n);  // n < 2^bits, so the all-ones key is never a real entry
    const uint64_t invalid = (bits * 2 >= 64) ? ~0ull : ((1ull << (2 * bits)) - 1ull);
    // undirected: one (min, max) key per edge while pair indices fit 32 bits
    const bool sym = !directed && E < ((int64_t)1 << 31);
    const int mode = directed ? KEYS_DIRECTED : (sym ? KEYS_SYM : KEYS_PAIR);
    const int64_t mk = sym ? E : m;  // keys emitted
    DBuf<float> va(ctx), vb(ctx);
    if (w) {
        CL_TRY(va.alloc((size_t)mk));
        CL_TRY(vb.alloc((size_t)mk));
    }
    if (E > 0) {
        k_entries<<<grid_for(E, 256, sms), 256, 0, s>>>(src, dst, w, E, mode, rank_tab.p, rank_mask, n,
                                                       has_empty, bits, invalid, ka, w ? va.p : nullptr, d_flag);
        CL_LAUNCHED(ctx);
        int missing = 0;
        CL_CUDA(ctx, read_back(ctx, &missing, d_flag, sizeof(int), s));
        CL_CUDA(ctx, cudaStreamSynchronize(s));
        if (missing) return fail(ctx, CLEORA_ERR_DEVICE, "endpoint missing from the id table");
    }
    rank_tab.reset();

    g.directed = directed != 0;
    if (sym) return csr_undirected(ctx, ka, kb, w ? va.p : nullptr, w ? vb.p : nullptr, E, 2 * E, n, bits, g);
    return csr_from_entries(ctx, ka, kb, w ? va.p : nullptr, w ? vb.p : nullptr, m, 2 * E, n, bits,
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
    CL_CUDA(ctx, read_back(ctx, &nnz, scal.p, sizeof(int64_t), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    g.nnz = nnz;

    DBuf<int32_t> rows(ctx);
    DBuf<double> e(ctx);  // e_ab of weighted graphs (unweighted: run lengths, from `start`)
    CL_TRY(rows.alloc((size_t)nnz));
    if (weighted) CL_TRY(e.alloc((size_t)nnz));
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
        k_degree_int<<<grid_for(n, 256, sms), 256, 0, s>>>(g.rowptr, start, nnz, scal.p + 3, n, g.deg, g.inv_deg,
                                                           reinterpret_cast<unsigned long long*>(scal.p + 2));
    CL_LAUNCHED(ctx);

    int64_t hv[3] = {0, 0, 0};
    CL_CUDA(ctx, read_back(ctx, hv, scal.p, 3 * sizeof(int64_t), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    const int not_unit = (int)(hv[1] & 0xffffffff);
    g.max_row_len = hv[2];
    g.has_val = weighted || not_unit;

    // stored values
    if (g.has_val) {
        CL_TRY(dalloc(ctx, &g.val, (size_t)(nnz ? nnz : 1)));
        k_values<<<grid_for(nnz, 256, sms), 256, 0, s>>>(rows.p, weighted ? e.p : nullptr, start, scal.p + 3,
                                                         g.deg, nnz, g.val);
        CL_LAUNCHED(ctx);
    }
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    g.built = true;
    return CLEORA_OK;
}

int csr_undirected(cleora_ctx* ctx, uint64_t* kbuf_a, uint64_t* kbuf_b, float* vbuf_a, float* vbuf_b, int64_t E,
                   int64_t kbuf_words, int64_t n, int bits, Graph& g) {
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    const bool weighted = vbuf_a != nullptr;
    DBuf<int64_t> scal(ctx);  // device scalars: [0] count, [1] flag, [2] max_len, [3] m_valid
    CL_TRY(scal.alloc(4));
    CL_CUDA(ctx, cudaMemsetAsync(scal.p, 0, 4 * sizeof(int64_t), s));
    int* d_flag = reinterpret_cast<int*>(scal.p + 1);
    const int64_t m_valid = E;  // no key is dropped

    // 1. stable sort of the (lo, hi) keys (weights carried along): duplicates stay in edge order
    uint64_t* keys = nullptr;
    float* vals = nullptr;
    {
        cub::DoubleBuffer<uint64_t> dk(kbuf_a, kbuf_b);
        size_t tb = 0;
        DBuf<unsigned char> tmp(ctx);
        if (weighted) {
            cub::DoubleBuffer<float> dv(vbuf_a, vbuf_b);
            CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(nullptr, tb, dk, dv, E, 0, 2 * bits, s));
            CL_TRY(tmp.alloc(tb));
            CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(tmp.p, tb, dk, dv, E, 0, 2 * bits, s));
            vals = dv.Current();
        } else {
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(nullptr, tb, dk, E, 0, 2 * bits, s));
            CL_TRY(tmp.alloc(tb));
            CL_CUDA(ctx, cub::DeviceRadixSort::SortKeys(tmp.p, tb, dk, E, 0, 2 * bits, s));
        }
        keys = dk.Current();
    }
    uint64_t* spare = (keys == kbuf_a) ? kbuf_b : kbuf_a;

    // 2. unique pairs: run starts (head flags and starts share the spare key buffer)
    uint8_t* head = reinterpret_cast<uint8_t*>(spare);
    int64_t* start = reinterpret_cast<int64_t*>(spare) + (E + 7) / 8;
    DBuf<int64_t> starts_buf(ctx);
    if ((E + 7) / 8 + E > kbuf_words) {
        CL_TRY(starts_buf.alloc((size_t)E));
        start = starts_buf.p;
    }
    k_heads<<<grid_for(E, 256, sms), 256, 0, s>>>(keys, E, ~0ull, head);
    CL_LAUNCHED(ctx);
    {
        size_t tb = 0;
        thrust::counting_iterator<int64_t> it(0);
        CL_CUDA(ctx, cub::DeviceSelect::Flagged(nullptr, tb, it, head, start, scal.p, E, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb));
        CL_CUDA(ctx, cub::DeviceSelect::Flagged(tmp.p, tb, it, head, start, scal.p, E, s));
    }
    CL_CUDA(ctx, put_bytes(ctx, scal.p + 3, &m_valid, sizeof(int64_t), s));
    int64_t nu = 0;
    CL_CUDA(ctx, read_back(ctx, &nu, scal.p, sizeof(int64_t), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));

    // 3. per pair: lo, hi, e (FP64 weight sum in edge order; unweighted: the multiplicity)
    DBuf<int32_t> plo(ctx), phi(ctx);
    DBuf<double> pe(ctx);
    CL_TRY(plo.alloc((size_t)nu));
    CL_TRY(phi.alloc((size_t)nu));
    if (weighted) CL_TRY(pe.alloc((size_t)nu));
    k_runs<<<grid_for(nu, 256, sms), 256, 0, s>>>(keys, vals, start, nu, scal.p + 3, bits, phi.p, plo.p,
                                                  weighted ? pe.p : nullptr, d_flag);
    CL_LAUNCHED(ctx);
    int flag = 0;
    CL_CUDA(ctx, read_back(ctx, &flag, d_flag, sizeof(int), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    const bool not_unit = flag != 0;
    const bool has_val = weighted || not_unit;
    if (!weighted && not_unit) {
        CL_TRY(pe.alloc((size_t)nu));
        k_counts_to_e<<<grid_for(nu, 256, sms), 256, 0, s>>>(start, nu, m_valid, pe.p);
        CL_LAUNCHED(ctx);
    }

    // 4. transposed half: pairs sorted stably by hi (the key buffers are free now)
    uint32_t* tk = reinterpret_cast<uint32_t*>(kbuf_a);
    uint32_t* tv = tk + nu;
    uint32_t* tk2 = tv + nu;
    uint32_t* tv2 = tk2 + nu;  // 16 nu bytes <= 16 E bytes of kbuf_a
    int64_t nt = 0;
    k_transpose_keys<<<grid_for(nu, 256, sms), 256, 0, s>>>(plo.p, phi.p, nu, (uint32_t)n, has_val, tk, tv);
    CL_LAUNCHED(ctx);
    {
        cub::DoubleBuffer<uint32_t> dk(tk, tk2), dv(tv, tv2);
        size_t tb = 0;
        CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(nullptr, tb, dk, dv, nu, 0, bits, s));
        DBuf<unsigned char> tmp(ctx);
        CL_TRY(tmp.alloc(tb));
        CL_CUDA(ctx, cub::DeviceRadixSort::SortPairs(tmp.p, tb, dk, dv, nu, 0, bits, s));
        tk = dk.Current();
        tv = dv.Current();
    }
    k_count_below<<<1, 1, 0, s>>>(tk, nu, (uint32_t)n, scal.p);
    CL_LAUNCHED(ctx);
    CL_CUDA(ctx, read_back(ctx, &nt, scal.p, sizeof(int64_t), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    const int64_t nnz = nu + nt;
    g.nnz = nnz;

    // 5. rowptr = (pairs with lo = r before) + (pairs with hi = r before)
    DBuf<int64_t> upptr(ctx), lowptr(ctx);
    CL_TRY(upptr.alloc((size_t)(n + 1)));
    CL_TRY(lowptr.alloc((size_t)(n + 1)));
    k_rowptr<<<grid_for(nu + 1, 256, sms), 256, 0, s>>>(plo.p, nu, n, upptr.p);
    k_rowptr<<<grid_for(nt + 1, 256, sms), 256, 0, s>>>(reinterpret_cast<const int32_t*>(tk), nt, n, lowptr.p);
    CL_LAUNCHED(ctx);
    CL_TRY(dalloc(ctx, &g.rowptr, (size_t)(n + 1)));
    k_add_rowptr<<<grid_for(n + 1, 256, sms), 256, 0, s>>>(upptr.p, lowptr.p, n, g.rowptr);
    CL_LAUNCHED(ctx);

    // 6. place both parts
    CL_TRY(dalloc(ctx, &g.col, (size_t)(nnz ? nnz : 1)));
    DBuf<double> e(ctx);
    DBuf<int32_t> rows(ctx);
    if (has_val) {
        CL_TRY(e.alloc((size_t)nnz));
        CL_TRY(rows.alloc((size_t)nnz));
    }
    k_place_low<<<grid_for(nt, 256, sms), 256, 0, s>>>(tk, tv, nt, g.rowptr, lowptr.p, plo.p, pe.p, g.col,
                                                       has_val ? e.p : nullptr, has_val ? rows.p : nullptr);
    k_place_up<<<grid_for(nu, 256, sms), 256, 0, s>>>(plo.p, phi.p, nu, g.rowptr, lowptr.p, upptr.p, pe.p, g.col,
                                                      has_val ? e.p : nullptr, has_val ? rows.p : nullptr);
    CL_LAUNCHED(ctx);

    // 7. degrees (weighted or repeated pairs: FP64 row sums in ascending column order)
    CL_TRY(dalloc(ctx, &g.deg, (size_t)(n ? n : 1)));
    CL_TRY(dalloc(ctx, &g.inv_deg, (size_t)(n ? n : 1)));
    unsigned long long* d_max = reinterpret_cast<unsigned long long*>(scal.p + 2);
    if (has_val)
        k_degree<<<grid_for(n, 256, sms), 256, 0, s>>>(g.rowptr, e.p, n, g.deg, g.inv_deg, d_max);
    else
        k_degree_len<<<grid_for(n, 256, sms), 256, 0, s>>>(g.rowptr, n, g.deg, g.inv_deg, d_max);
    CL_LAUNCHED(ctx);
    int64_t max_len = 0;
    CL_CUDA(ctx, read_back(ctx, &max_len, scal.p + 2, sizeof(int64_t), s));
    CL_CUDA(ctx, cudaStreamSynchronize(s));
    g.max_row_len = max_len;
    g.has_val = has_val;

    // 8. stored values
    if (has_val) {
        CL_TRY(dalloc(ctx, &g.val, (size_t)(nnz ? nnz : 1)));
        k_values<<<grid_for(nnz, 256, sms), 256, 0, s>>>(rows.p, e.p, nullptr, scal.p + 3, g.deg, nnz, g.val);
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
        CL_CUDA(ctx, read_back(ctx, &n, num.p, sizeof(int64_t), s));
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
    CL_CUDA(ctx, read_back(ctx, &bad, flag.p, sizeof(int), ctx->stream));
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
