// Host side of one Cleora iteration (arXiv 2102.02302, Algorithm 1, inner loop): kernel
// shape for (d, storage), the task plan of a graph, and the launch.
//
// Plan.  Rows longer than `split_len` entries are split into chunks of `split_len`; every
// other row belongs to a run of consecutive rows.  A new run starts where
// floor((rowptr[r] + ROW_COST * r) / task_nnz) changes, so runs hold about task_nnz entries
// (rows without entries still cost ROW_COST).  Tasks are ordered longest first: all split
// chunks, then the runs in row order.  The plan is built on the device and depends only on
// the graph and the two sizes, never on timing, so the summation order of every row is
// fixed by the graph's shape.
#include <mutex>
#include <vector>

#include <cudaTypedefs.h>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_sort.cuh>
#include <cub/device/device_select.cuh>
#include <thrust/iterator/counting_iterator.h>

#include "ring_kernels.cuh"

namespace cleora {
namespace {

constexpr int64_t ROW_COST = 8;

__device__ __forceinline__ int64_t run_key(const int64_t* rowptr, int64_t r, int64_t task_nnz) {
    return (rowptr[r] + ROW_COST * r) / task_nnz;
}

__global__ void k_plan_mark(const int64_t* rowptr, int64_t n, int64_t split_len, int64_t task_nnz,
                            uint8_t* brk) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const bool split = rowptr[r + 1] - rowptr[r] > split_len;
        bool b = split || r == 0;
        if (!b) {
            const bool prev_split = rowptr[r] - rowptr[r - 1] > split_len;
            b = prev_split || run_key(rowptr, r, task_nnz) != run_key(rowptr, r - 1, task_nnz);
        }
        brk[r] = b ? 1 : 0;
    }
}

// Per break i: chunks (split rows), normal-task flag and split flag.
__global__ void k_plan_counts(const int64_t* rowptr, const int32_t* brk_rows, int64_t nb,
                              int64_t split_len, int64_t* chunks, int64_t* normal, int64_t* split) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = brk_rows[i];
        const int64_t len = rowptr[r + 1] - rowptr[r];
        const bool s = len > split_len;
        chunks[i] = s ? (len + split_len - 1) / split_len : 0;
        normal[i] = s ? 0 : 1;
        split[i] = s ? 1 : 0;
    }
}

__global__ void k_plan_fill(const int32_t* brk_rows, int64_t nb, int64_t n, const int64_t* chunks,
                            const int64_t* cbase, const int64_t* nbase, const int64_t* sbase,
                            int64_t total_chunks, Task* tasks, int64_t* split_base) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nb;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int32_t r = brk_rows[i];
        const int64_t nc = chunks[i];
        if (nc > 0) {
            const int64_t sidx = sbase[i];
            split_base[sidx] = cbase[i];
            for (int64_t c = 0; c < nc; ++c) {
                Task t;
                t.a = r;
                t.b = (int32_t)sidx;
                t.c = (int32_t)c;
                t.k = (int32_t)nc;
                tasks[cbase[i] + c] = t;
            }
        } else {
            Task t;
            t.a = r;
            t.b = (int32_t)((i + 1 < nb) ? (int64_t)brk_rows[i + 1] : n);
            t.c = -1;
            t.k = 0;
            tasks[total_chunks + nbase[i]] = t;
        }
    }
}

// Quarter-octave bin of a count: 0 for 0, else 1 + floor(4 log2 c), at most 127 (double log2:
// non-decreasing in c, so a higher count never lands in a lower bin).
__device__ __forceinline__ int count_bin(uint32_t c) {
    if (c == 0) return 0;
    const int b = 1 + (int)(4.0 * log2((double)c));
    return b > 127 ? 127 : b;
}

__global__ void k_indegree(const int32_t* col, int64_t nnz, uint32_t* cnt) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt + col[k], 1u);
}

__global__ void k_rowlen(const int64_t* rowptr, int64_t n, uint32_t* cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = rowptr[r + 1] - rowptr[r];
        cnt[r] = (uint32_t)(l > 0xffffffffll ? 0xffffffffll : l);
    }
}

// Per-node bin (uint8) and the global histogram of bins.
__global__ void k_bins(const uint32_t* cnt, int64_t n, uint8_t* bin, unsigned long long* hist) {
    __shared__ unsigned int h[128];
    for (int i = threadIdx.x; i < 128; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int b = count_bin(cnt[r]);
        bin[r] = (uint8_t)b;
        atomicAdd(h + b, 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 128; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Count range [lo, hi] of the rows in bin b (atomic min / max).
__global__ void k_bin_range(const uint32_t* cnt, const uint8_t* bin, int64_t n, int b, unsigned* lohi) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        if (bin[r] == b) {
            atomicMin(lohi, cnt[r]);
            atomicMax(lohi + 1, cnt[r]);
        }
}

constexpr int FINE = 4096;  // buckets of the boundary bin's fine histogram

__device__ __forceinline__ int fine_bucket(uint32_t c, uint32_t lo, uint32_t hi) {
    return (int)(((uint64_t)(c - lo) * FINE) / ((uint64_t)(hi - lo) + 1));
}

__global__ void k_bin_fine(const uint32_t* cnt, const uint8_t* bin, int64_t n, int b, const unsigned* lohi,
                           unsigned long long* fine) {
    const uint32_t lo = lohi[0], hi = lohi[1];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x)
        if (bin[r] == b) atomicAdd(fine + fine_bucket(cnt[r], lo, hi), 1ull);
}

// Hot flag per row (in place of its bin): every row of a bin above b, and the rows of bin b
// whose fine bucket is at least fb (fb > FINE: none of bin b).
__global__ void k_hot_flags(const uint32_t* cnt, uint8_t* bin, int64_t n, int b, int fb, const unsigned* lohi) {
    const uint32_t lo = lohi[0], hi = lohi[1];
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int x = bin[r];
        bin[r] = (x > b || (x == b && fb <= FINE && fine_bucket(cnt[r], lo, hi) >= fb)) ? 1 : 0;
    }
}

// Hot flags of 32 consecutive entries as one bit word (a warp per word, a lane per entry:
// coalesced loads and one ballot), and the word's count.
__global__ void k_hot_words(const int32_t* col, int64_t nnz, const uint8_t* bin, int threshold, uint32_t* word,
                            int64_t* cnt, int64_t nw) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < nw; w += nwarps) {
        const int64_t k = w * 32 + lane;
        const bool hot = k < nnz && bin[__ldcs(col + k)] >= threshold;
        const uint32_t bits = __ballot_sync(0xffffffffu, hot);
        if (lane == 0) {
            word[w] = bits;
            cnt[w] = __popc(bits);
        }
    }
}

// Hot entries among positions [0, p) (base: exclusive prefix of the word counts).
__device__ __forceinline__ int64_t hot_before(const uint32_t* word, const int64_t* base, int64_t nw, int64_t p) {
    const int64_t w = p >> 5;
    if (w >= nw) return base[nw - 1] + __popc(word[nw - 1]);
    return base[w] + __popc(word[w] & ((1u << (p & 31)) - 1u));
}

// Per row: hot entries before its start (rowH, n + 1 values) and in the row (hot_cnt).
__global__ void k_row_hot(const int64_t* rowptr, int64_t n, const uint32_t* word, const int64_t* base, int64_t nw,
                          int64_t* rowH, int32_t* hot_cnt) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t hb = hot_before(word, base, nw, rowptr[r]);
        const int64_t he = hot_before(word, base, nw, rowptr[r + 1]);
        rowH[r] = hb;
        hot_cnt[r] = (int32_t)(he - hb);
        if (r == n - 1) rowH[n] = he;
    }
}

// Last row r in [lo, hi] with rowptr[r] <= k (the row holding entry k; empty rows skipped).
__device__ __forceinline__ int64_t row_of(const int64_t* rowptr, int64_t k, int64_t lo, int64_t hi) {
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo + 1) / 2;
        if (rowptr[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Stable hot-first partition of every row.  A warp takes a run of 32-entry words and one
// word at a time, a lane per entry, so that loads are coalesced and a row's hot entries (and
// its cold ones) are stored by consecutive lanes to consecutive places.  A hot entry k of row
// [beg, end) goes to beg + (hot entries of the row before k); a cold one after the row's hot
// part, to k - H(k) + H(end), H(p) = hot entries in [0, p).
constexpr int SCATTER_WORDS = 32;  // words per warp task

__global__ void __launch_bounds__(256) k_hot_scatter(const int64_t* rowptr, int64_t n, const int32_t* col,
                                                     const float* val, int64_t nnz, const uint32_t* word,
                                                     const int64_t* base, int64_t nw, const int64_t* rowH,
                                                     int32_t* col2, float* val2) {
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t w0 = warp * SCATTER_WORDS; w0 < nw; w0 += nwarps * SCATTER_WORDS) {
        const int64_t w1 = min(nw, w0 + SCATTER_WORDS);
        int64_t lo = 0, hi = 0;  // rows holding the task's first and last entries
        if (lane == 0) {
            lo = row_of(rowptr, w0 * 32, 0, n - 1);
            hi = row_of(rowptr, min(nnz, w1 * 32) - 1, lo, n - 1);
        }
        lo = __shfl_sync(FULL, lo, 0);
        hi = __shfl_sync(FULL, hi, 0);
        for (int64_t w = w0; w < w1; ++w) {
            const int64_t k = w * 32 + lane;
            const uint32_t bits = word[w];
            int64_t r = hi;
            if (k < nnz) {
                r = row_of(rowptr, k, lo, hi);
                const bool hot = (bits >> lane) & 1u;
                const int64_t H = base[w] + __popc(bits & ((1u << lane) - 1u));
                const int64_t pos = hot ? rowptr[r] + (H - rowH[r]) : k - H + rowH[r + 1];
                col2[pos] = col[k];
                if (val) val2[pos] = val[k];
            }
            lo = __shfl_sync(FULL, r, 31);  // the next word starts in this word's last row
        }
    }
}

int pow2ceil(int v) {
    int p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

Shape choose_shape(const cleora_ctx* ctx, int d, cleora_dtype dt) {
    return shape_for(d, dt, ctx->opt[CLEORA_OPT_VEC_BYTES], ctx->opt[CLEORA_OPT_ROW_MODE]);
}

Shape shape_for(int d, cleora_dtype dt, int64_t vec_opt, int64_t mode_opt) {
    Shape sh;
    const int es = dt == CLEORA_F32 ? 4 : 2;
    // automatic width: 16-byte vectors when a row has at least 32 of them (a full warp),
    // else 8-byte vectors, which put more lanes on a row (measured: BF16 d = 128 runs 8%
    // faster as a full warp of 8-byte gathers than as half-warps of 16-byte gathers)
    int vec = vec_opt == 8 ? 8 : vec_opt == 16 ? 16 : (d * es / 16 >= 32 ? 16 : 8);
    int chunks = d * es / vec;
    if (vec == 8 && pow2ceil((chunks + 31) / 32) > 8) {  // too many vectors per lane
        vec = 16;
        chunks = d * es / vec;
    }
    sh.vec = vec;
    sh.chunks = chunks;
    if (chunks <= 32) {
        sh.G = pow2ceil(chunks);
        sh.cpl = 1;
    } else {
        sh.G = 32;
        sh.cpl = pow2ceil((chunks + 31) / 32);
    }
    sh.mode = (mode_opt == 2 && sh.G < 32) ? 2 : 1;
    return sh;
}

void plan_release(cleora_ctx* ctx) {
    Plan& p = ctx->plan;
    dfree_null(ctx, p.tasks);
    dfree_null(ctx, p.split_base);
    dfree_null(ctx, p.split_count);
    dfree_null(ctx, p.counter);
    dfree_null(ctx, p.partials);
    p = Plan();
}

int plan_build(cleora_ctx* ctx, int64_t split_len, int64_t task_nnz) {
    plan_release(ctx);
    const Graph& g = ctx->g;
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    Plan& p = ctx->plan;
    p.split_len = split_len;
    p.task_nnz = task_nnz;
    CL_TRY(dalloc(ctx, &p.counter, 1));
    if (g.n == 0) {
        p.valid = true;
        return CLEORA_OK;
    }
    uint8_t* brk = nullptr;
    int32_t* rows = nullptr;
    int64_t* scal = nullptr;
    int64_t* work = nullptr;  // 6 arrays of nb int64
    int rc = CLEORA_OK;
    int64_t nb = 0;
    auto cleanup = [&]() {
        dfree(ctx, brk);
        dfree(ctx, rows);
        dfree(ctx, scal);
        dfree(ctx, work);
    };
    do {
        if ((rc = dalloc(ctx, &brk, (size_t)g.n))) break;
        if ((rc = dalloc(ctx, &rows, (size_t)g.n))) break;
        if ((rc = dalloc(ctx, &scal, 4))) break;
        k_plan_mark<<<grid_for(g.n, 256, sms), 256, 0, s>>>(g.rowptr, g.n, split_len, task_nnz, brk);
        ctx->launches++;
        size_t tb = 0;
        thrust::counting_iterator<int32_t> it(0);
        cudaError_t e = cub::DeviceSelect::Flagged(nullptr, tb, it, brk, rows, scal, g.n, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "select", __FILE__, __LINE__); break; }
        void* tmp = nullptr;
        if ((rc = dalloc_bytes(ctx, &tmp, tb))) break;
        e = cub::DeviceSelect::Flagged(tmp, tb, it, brk, rows, scal, g.n, s);
        dfree(ctx, tmp);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "select", __FILE__, __LINE__); break; }
        e = read_back(ctx, &nb, scal, sizeof(int64_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "plan count", __FILE__, __LINE__); break; }
        if ((rc = dalloc(ctx, &work, (size_t)(6 * nb)))) break;
        int64_t *chunks = work, *normal = work + nb, *split = work + 2 * nb;
        int64_t *cbase = work + 3 * nb, *nbase = work + 4 * nb, *sbase = work + 5 * nb;
        k_plan_counts<<<grid_for(nb, 256, sms), 256, 0, s>>>(g.rowptr, rows, nb, split_len, chunks,
                                                             normal, split);
        ctx->launches++;
        tb = 0;
        e = cub::DeviceScan::ExclusiveSum(nullptr, tb, chunks, cbase, nb, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "scan", __FILE__, __LINE__); break; }
        if ((rc = dalloc_bytes(ctx, &tmp, tb))) break;
        e = cub::DeviceScan::ExclusiveSum(tmp, tb, chunks, cbase, nb, s);
        if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, tb, normal, nbase, nb, s);
        if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, tb, split, sbase, nb, s);
        dfree(ctx, tmp);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "scan", __FILE__, __LINE__); break; }
        int64_t last[6];
        const int64_t* srcs[6] = {cbase + nb - 1, chunks + nb - 1, nbase + nb - 1,
                                  normal + nb - 1, sbase + nb - 1, split + nb - 1};
        for (int k = 0; k < 6 && e == cudaSuccess; ++k)
            e = read_back(ctx, &last[k], srcs[k], sizeof(int64_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "plan totals", __FILE__, __LINE__); break; }
        p.nsplit_chunks = last[0] + last[1];
        const int64_t total_normal = last[2] + last[3];
        p.nsplit_rows = last[4] + last[5];
        p.ntasks = p.nsplit_chunks + total_normal;
        if ((rc = dalloc(ctx, &p.tasks, (size_t)p.ntasks))) break;
        if ((rc = dalloc(ctx, &p.split_base, (size_t)(p.nsplit_rows ? p.nsplit_rows : 1)))) break;
        if ((rc = dalloc(ctx, &p.split_count, (size_t)(p.nsplit_rows ? p.nsplit_rows : 1)))) break;
        e = cudaMemsetAsync(p.split_count, 0, sizeof(int32_t) * (p.nsplit_rows ? p.nsplit_rows : 1), s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "memset", __FILE__, __LINE__); break; }
        k_plan_fill<<<grid_for(nb, 256, sms), 256, 0, s>>>(rows, nb, g.n, chunks, cbase, nbase, sbase,
                                                           p.nsplit_chunks, p.tasks, p.split_base);
        ctx->launches++;
        e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "plan fill", __FILE__, __LINE__); break; }
    } while (0);
    cleanup();
    if (rc == CLEORA_OK) p.valid = true;
    return rc;
}

int plan_ensure(cleora_ctx* ctx) {
    int64_t split_len = ctx->opt[CLEORA_OPT_SPLIT_LEN] > 0 ? ctx->opt[CLEORA_OPT_SPLIT_LEN] : DEFAULT_SPLIT_LEN;
    int64_t task_nnz = ctx->opt[CLEORA_OPT_TASK_NNZ] > 0 ? ctx->opt[CLEORA_OPT_TASK_NNZ] : DEFAULT_TASK_NNZ;
    Plan& p = ctx->plan;
    if (!p.valid || p.split_len != split_len || p.task_nnz != task_nnz)
        CL_TRY(plan_build(ctx, split_len, task_nnz));
    if (ctx->d > 0 && p.nsplit_chunks > 0 && p.partials_d != ctx->d) {
        dfree_null(ctx, p.partials);
        CL_TRY(dalloc(ctx, &p.partials, (size_t)(p.nsplit_chunks * ctx->d)));
        p.partials_d = ctx->d;
    }
    return CLEORA_OK;
}

// Entries of every row in ascending column order, from the hot-first layout: a segmented
// sort of each row's column indices (with their values) into the given buffers.
static int sort_rows(cleora_ctx* ctx, const int32_t* col, const float* val, int32_t* col_dst, float* val_dst) {
    const Graph& g = ctx->g;
    cudaStream_t s = ctx->stream;
    size_t tb = 0;
    cudaError_t e = val ? cub::DeviceSegmentedSort::SortPairs(nullptr, tb, col, col_dst, val, val_dst, g.nnz, g.n,
                                                              g.rowptr, g.rowptr + 1, s)
                        : cub::DeviceSegmentedSort::SortKeys(nullptr, tb, col, col_dst, g.nnz, g.n, g.rowptr,
                                                             g.rowptr + 1, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "row sort", __FILE__, __LINE__);
    void* tmp = nullptr;
    CL_TRY(dalloc_bytes(ctx, &tmp, tb ? tb : 1));
    e = val ? cub::DeviceSegmentedSort::SortPairs(tmp, tb, col, col_dst, val, val_dst, g.nnz, g.n, g.rowptr,
                                                  g.rowptr + 1, s)
            : cub::DeviceSegmentedSort::SortKeys(tmp, tb, col, col_dst, g.nnz, g.n, g.rowptr, g.rowptr + 1, s);
    dfree(ctx, tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "row sort", __FILE__, __LINE__);
    ctx->launches++;
    return CLEORA_OK;
}

int hot_restore(cleora_ctx* ctx) {
    Graph& g = ctx->g;
    if (g.hot_bits) {  // ring layout: rows are in ascending order already
        dfree_null(ctx, g.hot_bits);
        g.part_row_bytes = 0;
        g.part_budget = 0;
        g.hot_entries = 0;
    }
    if (!g.hot_cnt) return CLEORA_OK;
    int32_t* col2 = nullptr;
    float* val2 = nullptr;
    CL_TRY(dalloc(ctx, &col2, (size_t)g.nnz));
    if (g.has_val) {
        int rc = dalloc(ctx, &val2, (size_t)g.nnz);
        if (rc) { dfree(ctx, col2); return rc; }
    }
    int rc = sort_rows(ctx, g.col, g.has_val ? g.val : nullptr, col2, val2);
    if (rc) {
        dfree(ctx, col2);
        dfree(ctx, val2);
        return rc;
    }
    dfree(ctx, g.col);
    g.col = col2;
    if (g.has_val) {
        dfree(ctx, g.val);
        g.val = val2;
    }
    dfree_null(ctx, g.hot_cnt);
    g.part_row_bytes = 0;
    g.part_budget = 0;
    return CLEORA_OK;
}

// The ring runs only when asked for (staging = 2): measured on the 1.4B-edge graph it takes
// 128 ms (BF16) and 180 ms (FP32) per iteration against the register kernel's 72 and 120 ms --
// one bulk copy per gathered row costs the issuing warp more than it gains in depth.
bool use_ring(const cleora_ctx* ctx) {
    if (ctx->d == 0) return false;
    const Shape sh = choose_shape(ctx, ctx->d, ctx->dtype);
    return ring_shape(sh) && (ctx->opt[CLEORA_OPT_STAGING] == 2 || ctx->opt[CLEORA_OPT_STAGING] == 3);
}

// Tensor maps over both embedding buffers for the ring's 4-row gathers: a 2-D tensor of n rows
// of d elements (row stride d * element bytes), box d x 1 (one row per gathered coordinate).
int ring_tensor_maps(cleora_ctx* ctx) {
    ctx->tmap_ready = false;
    if (!use_ring(ctx) || ctx->opt[CLEORA_OPT_STAGING] != 3 || ctx->g.n == 0) return CLEORA_OK;
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
        cudaGetLastError();
    });
    if (!encode) return fail(ctx, CLEORA_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    const int es = ctx->dtype == CLEORA_F32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)ctx->d, (cuuint64_t)ctx->g.n};
    const cuuint64_t strides[1] = {(cuuint64_t)ctx->d * es};
    const cuuint32_t box[2] = {(cuuint32_t)ctx->d, 1};
    const cuuint32_t estr[2] = {1, 1};
    for (int k = 0; k < 2; ++k) {
        const CUresult r = encode(&ctx->tmap[k],
                                  ctx->dtype == CLEORA_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                                  2, ctx->T[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(ctx, CLEORA_ERR_CUDA, "tensor map encoding failed (%d)", (int)r);
    }
    ctx->tmap_ready = true;
    return CLEORA_OK;
}

// Marks the entries that point at the rows with the largest in-degree, as many rows as fit
// in the hot-row L2 budget at the current row size (whole quarter-octave bins from the top,
// then the boundary bin's rows from a 4096-bucket histogram of their exact counts).
//  * Register kernel: every row is partitioned hot-first (both parts keep ascending column
//    order); the kernel gathers the hot part with an L2 evict_last policy and the rest
//    evict_first, the policy uniform over each part, so no entry carries a mark.
//  * Ring kernel: rows keep ascending order; a bitmap over the entries gives each lane's bulk
//    copy its policy.
// Graphs whose whole T fits twice in the budget are left as they are (everything is reused).
int hot_partition(cleora_ctx* ctx) {
    Graph& g = ctx->g;
    const int64_t row_bytes = (int64_t)ctx->d * (ctx->dtype == CLEORA_F32 ? 4 : 2);
    const int64_t opt = ctx->opt[CLEORA_OPT_HOT_BYTES];
    const int64_t budget = opt == 0 ? DEFAULT_HOT_BYTES : (opt == 1 ? 0 : opt);
    const bool ring = use_ring(ctx);
    const bool uses = ring || (ctx->dtype == CLEORA_F32 ? prop::Tune<float>::POLICY : prop::Tune<__nv_bfloat16>::POLICY);
    const bool want = uses && budget > 0 && g.n > 0 && g.nnz > 0 && g.n * row_bytes > 2 * budget;
    if (!want && !g.hot_cnt && !g.hot_bits) return CLEORA_OK;
    if (want && g.part_row_bytes == row_bytes && g.part_budget == budget &&
        ((ring && g.hot_bits) || (!ring && g.hot_cnt)))
        return CLEORA_OK;
    CL_TRY(hot_restore(ctx));
    if (!want) return CLEORA_OK;
    cudaStream_t s = ctx->stream;
    const int sms = ctx->num_sms;
    const int64_t nw = (g.nnz + 31) / 32;
    uint32_t* cnt = nullptr;
    uint8_t* bin = nullptr;
    unsigned long long* hist = nullptr;  // 128 bins + FINE buckets
    unsigned* lohi = nullptr;
    uint32_t* word = nullptr;
    int64_t* wcnt = nullptr;
    int64_t* rowH = nullptr;
    int32_t* hot_cnt = nullptr;
    int32_t* col2 = nullptr;
    float* val2 = nullptr;
    void* tmp = nullptr;
    int rc = CLEORA_OK;
    do {
        if ((rc = dalloc(ctx, &cnt, (size_t)g.n))) break;
        if ((rc = dalloc(ctx, &bin, (size_t)g.n))) break;
        if ((rc = dalloc(ctx, &hist, 128 + FINE))) break;
        if ((rc = dalloc(ctx, &lohi, 2))) break;
        cudaError_t e = cudaMemsetAsync(hist, 0, (128 + FINE) * sizeof(unsigned long long), s);
        if (e == cudaSuccess && g.directed) e = cudaMemsetAsync(cnt, 0, g.n * sizeof(uint32_t), s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
        if (g.directed)
            k_indegree<<<grid_for(g.nnz, 256, sms), 256, 0, s>>>(g.col, g.nnz, cnt);
        else  // symmetric: in-degree = row length
            k_rowlen<<<grid_for(g.n, 256, sms), 256, 0, s>>>(g.rowptr, g.n, cnt);
        k_bins<<<grid_for(g.n, 256, sms), 256, 0, s>>>(cnt, g.n, bin, hist);
        ctx->launches += 2;
        unsigned long long h[128];
        e = read_back(ctx, h, hist, sizeof(h), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
        const int64_t rows = budget / row_bytes;
        int64_t acc = 0;
        int b = 127;  // whole bins above b are hot; b is the boundary bin
        for (; b >= 1; --b) {
            if (acc + (int64_t)h[b] > rows) break;
            acc += (int64_t)h[b];
        }
        if (b < 1) b = 0;  // every row with entries fits
        int fb = FINE + 1;  // bucket threshold inside bin b (none)
        if (b >= 1 && h[b] > 0 && acc < rows) {
            const unsigned init[2] = {0xffffffffu, 0u};
            e = put_bytes(ctx, lohi, init, sizeof(init), s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
            k_bin_range<<<grid_for(g.n, 256, sms), 256, 0, s>>>(cnt, bin, g.n, b, lohi);
            k_bin_fine<<<grid_for(g.n, 256, sms), 256, 0, s>>>(cnt, bin, g.n, b, lohi, hist + 128);
            ctx->launches += 2;
            std::vector<unsigned long long> f(FINE);
            e = read_back(ctx, f.data(), hist + 128, FINE * sizeof(unsigned long long), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
            for (int q = FINE - 1; q >= 0; --q) {  // the rows of the top buckets that still fit
                if (acc + (int64_t)f[q] > rows) break;
                acc += (int64_t)f[q];
                fb = q;
            }
        }
        if (acc == 0) break;  // not even one row fits: leave the rows as they are
        k_hot_flags<<<grid_for(g.n, 256, sms), 256, 0, s>>>(cnt, bin, g.n, b, fb, lohi);
        ctx->launches++;
        dfree_null(ctx, cnt);
        if ((rc = dalloc(ctx, &word, (size_t)nw))) break;
        if ((rc = dalloc(ctx, &wcnt, (size_t)nw))) break;
        k_hot_words<<<grid_for(nw * 32, 256, sms), 256, 0, s>>>(g.col, g.nnz, bin, 1, word, wcnt, nw);
        ctx->launches++;
        size_t tb = 0;
        e = cub::DeviceScan::ExclusiveSum(nullptr, tb, wcnt, wcnt, nw, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "scan", __FILE__, __LINE__); break; }
        if ((rc = dalloc_bytes(ctx, &tmp, tb ? tb : 1))) break;
        if (ring) {  // hot entries = the popcounts of the words (scanned in place)
            int64_t last_base = 0;
            uint32_t last_word = 0;
            e = cub::DeviceScan::ExclusiveSum(tmp, tb, wcnt, wcnt, nw, s);
            if (e == cudaSuccess)
                e = read_back(ctx, &last_base, wcnt + nw - 1, sizeof(int64_t), s);
            if (e == cudaSuccess)
                e = read_back(ctx, &last_word, word + nw - 1, sizeof(uint32_t), s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
            ctx->launches++;
            g.hot_entries = last_base + __builtin_popcount(last_word);
            g.hot_bits = word;
            word = nullptr;
            g.part_row_bytes = row_bytes;
            g.part_budget = budget;
            break;
        }
        if ((rc = dalloc(ctx, &rowH, (size_t)(g.n + 1)))) break;
        if ((rc = dalloc(ctx, &hot_cnt, (size_t)g.n))) break;
        if ((rc = dalloc(ctx, &col2, (size_t)g.nnz))) break;
        if (g.has_val && (rc = dalloc(ctx, &val2, (size_t)g.nnz))) break;
        e = cub::DeviceScan::ExclusiveSum(tmp, tb, wcnt, wcnt, nw, s);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "scan", __FILE__, __LINE__); break; }
        ctx->launches++;
        k_row_hot<<<grid_for(g.n, 256, sms), 256, 0, s>>>(g.rowptr, g.n, word, wcnt, nw, rowH, hot_cnt);
        const int64_t blocks = std::min<int64_t>((nw + 8 * SCATTER_WORDS - 1) / (8 * SCATTER_WORDS), (int64_t)sms * 8);
        k_hot_scatter<<<(unsigned)blocks, 256, 0, s>>>(g.rowptr, g.n, g.col, g.has_val ? g.val : nullptr, g.nnz,
                                                       word, wcnt, nw, rowH, col2, val2);
        ctx->launches += 2;
        int64_t hot_total = 0;
        e = read_back(ctx, &hot_total, rowH + g.n, sizeof(int64_t), s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "hot partition", __FILE__, __LINE__); break; }
        g.hot_entries = hot_total;
        dfree(ctx, g.col);
        g.col = col2;
        col2 = nullptr;
        if (g.has_val) {
            dfree(ctx, g.val);
            g.val = val2;
            val2 = nullptr;
        }
        g.hot_cnt = hot_cnt;
        hot_cnt = nullptr;
        g.part_row_bytes = row_bytes;
        g.part_budget = budget;
    } while (0);
    dfree(ctx, cnt);
    dfree(ctx, bin);
    dfree(ctx, hist);
    dfree(ctx, lohi);
    dfree(ctx, word);
    dfree(ctx, wcnt);
    dfree(ctx, rowH);
    dfree(ctx, hot_cnt);
    dfree(ctx, col2);
    dfree(ctx, val2);
    dfree(ctx, tmp);
    return rc;
}

int col_out(cleora_ctx* ctx, int32_t* col_dev) {
    const Graph& g = ctx->g;
    if (g.nnz == 0) return CLEORA_OK;
    if (g.hot_cnt) return sort_rows(ctx, g.col, nullptr, col_dev, nullptr);
    CL_CUDA(ctx, cudaMemcpyAsync(col_dev, g.col, g.nnz * sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    return CLEORA_OK;
}

int values_out_sorted(cleora_ctx* ctx, float* val_dev) {
    const Graph& g = ctx->g;
    int32_t* keys = nullptr;
    CL_TRY(dalloc(ctx, &keys, (size_t)g.nnz));
    const int rc = sort_rows(ctx, g.col, g.val, keys, val_dev);
    dfree(ctx, keys);
    return rc;
}

int propagate_step(cleora_ctx* ctx, const void* Tin, void* Tout) {
    const Graph& g = ctx->g;
    const Plan& p = ctx->plan;
    if (g.n == 0 || p.ntasks == 0) return CLEORA_OK;
    const Shape sh = choose_shape(ctx, ctx->d, ctx->dtype);
    prop::Args a;
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.val = g.val;
    a.Tin = static_cast<const unsigned char*>(Tin);
    a.Tout = static_cast<unsigned char*>(Tout);
    a.n = g.n;
    a.nnz = g.nnz;
    a.row_bytes = (int64_t)ctx->d * (ctx->dtype == CLEORA_F32 ? 4 : 2);
    a.chunks = sh.chunks;
    a.d = ctx->d;
    a.split_len = p.split_len;
    a.tasks = p.tasks;
    a.ntasks = p.ntasks;
    a.counter = p.counter;
    a.split_base = p.split_base;
    a.split_count = p.split_count;
    a.partials = p.partials;
    a.err = ctx->err_flag;
    a.hot_cnt = g.hot_cnt;
    CL_CUDA(ctx, cudaMemsetAsync(p.counter, 0, sizeof(unsigned long long), ctx->stream));
    const int bps = (int)ctx->opt[CLEORA_OPT_BLOCKS_PER_SM];
    cudaError_t e;
    int grid = 0;
    if (use_ring(ctx) && (reinterpret_cast<uintptr_t>(Tin) & 15) == 0) {
        a.hot_cnt = nullptr;
        a.hot_bits = g.hot_bits;
        a.test_wait_runout = (int)ctx->opt[CLEORA_OPT_TEST_RING_WAIT];
        const int st = ctx->opt[CLEORA_OPT_RING_STAGES] ? (int)ctx->opt[CLEORA_OPT_RING_STAGES] : DEFAULT_RING_STAGES;
        const CUtensorMap* tm = nullptr;
        if (ctx->opt[CLEORA_OPT_STAGING] == 3) {
            if (!ctx->tmap_ready) return fail(ctx, CLEORA_ERR_STATE, "no tensor maps: init again after setting staging");
            const int k = Tin == ctx->T[0] ? 0 : (Tin == ctx->T[1] ? 1 : -1);
            if (k < 0) return fail(ctx, CLEORA_ERR_STATE, "ring gathers read the context's embeddings only");
            tm = &ctx->tmap[k];
        }
        if (ctx->dtype == CLEORA_F32)
            e = sh.vec == 16 ? ring::launch_f32_v16(a, tm, g.has_val, st, ctx->num_sms, ctx->stream, &grid)
                             : ring::launch_f32_v8(a, tm, g.has_val, st, ctx->num_sms, ctx->stream, &grid);
        else
            e = sh.vec == 16 ? ring::launch_bf16_v16(a, tm, g.has_val, st, ctx->num_sms, ctx->stream, &grid)
                             : ring::launch_bf16_v8(a, tm, g.has_val, st, ctx->num_sms, ctx->stream, &grid);
        ctx->launches++;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "propagate launch", __FILE__, __LINE__);
        return CLEORA_OK;
    }
    if (g.hot_bits) return fail(ctx, CLEORA_ERR_STATE, "rows are laid out for the ring kernel");
    if (ctx->dtype == CLEORA_F32)
        e = sh.vec == 16 ? prop::launch_f32_v16(sh, a, g.has_val, bps, ctx->num_sms, ctx->stream, &grid)
                         : prop::launch_f32_v8(sh, a, g.has_val, bps, ctx->num_sms, ctx->stream, &grid);
    else
        e = sh.vec == 16 ? prop::launch_bf16_v16(sh, a, g.has_val, bps, ctx->num_sms, ctx->stream, &grid)
                         : prop::launch_bf16_v8(sh, a, g.has_val, bps, ctx->num_sms, ctx->stream, &grid);
    ctx->launches++;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "propagate launch", __FILE__, __LINE__);
    return CLEORA_OK;
}

}  // namespace cleora
