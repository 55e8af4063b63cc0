// cleora_propagate_noalloc: one propagation step that allocates no device memory.
//
// Who needs it: callers that may not take device memory from inside this library --
// a host framework whose allocator owns every byte of HBM and hands out fixed budgets,
// a latency-critical loop that cannot afford cudaMalloc/cudaFree (which can synchronise the
// device), or a job that must not fail halfway with out-of-memory.  They pass the graph
// (CSR) and both embedding buffers; the step's scratch lives in one file-scope device array
// of fixed size that every GPU loading the library holds until the process exits.
//
// Scratch layout (g_scratch, SCRATCH_BYTES = 8,618,240 bytes):
//   header   (256 B)   : work counter, split-row count, split-chunk count, overflow flag
//   split rows (8192)  : first partial slot (int64), arrival count (int32), row, chunks
//   chunk map (16384)  : split-row index of every split chunk
//   partials (8 MiB)   : FP32 partial sums, one d-wide slot per split chunk
// Three launches per call: reset the header, register the rows longer than split_len (each
// takes a range of chunk slots), then the propagate kernel over [split chunks | row blocks].
// Every call reuses the same array and keeps the previous call's contents; the header is
// cleared at the start of each call.  Two calls that overlap on the GPU (different streams,
// or the same array from two threads) race on it.
#include <mutex>

#include "propagate_kernels.cuh"

namespace cleora {
namespace noalloc {

constexpr int MAX_SPLIT_ROWS = 8192;
constexpr int MAX_CHUNKS = 16384;
constexpr size_t HEADER_BYTES = 256;
constexpr size_t ROWS_BYTES = (size_t)MAX_SPLIT_ROWS * (8 + 4 + 4 + 4);
constexpr size_t MAP_BYTES = (size_t)MAX_CHUNKS * 4;
constexpr size_t PARTIAL_BYTES = (size_t)8 << 20;
constexpr size_t SCRATCH_BYTES = HEADER_BYTES + ROWS_BYTES + MAP_BYTES + PARTIAL_BYTES;
constexpr int ROWS_PER_BLOCK = 32;

static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

struct Header {
    unsigned long long work;
    int nsplit;
    int nchunks;
    int overflow;
    int err;  // out-of-range column index seen (the step then skips that entry)
};

struct View {
    Header* hdr;
    int64_t* split_base;
    int32_t* split_count;
    int32_t* split_row;
    int32_t* split_nch;
    int32_t* chunk_map;
    float* partials;
};

__host__ __device__ inline View view_of(unsigned char* base) {
    View v;
    v.hdr = reinterpret_cast<Header*>(base);
    unsigned char* p = base + HEADER_BYTES;
    v.split_base = reinterpret_cast<int64_t*>(p);
    p += (size_t)MAX_SPLIT_ROWS * 8;
    v.split_count = reinterpret_cast<int32_t*>(p);
    p += (size_t)MAX_SPLIT_ROWS * 4;
    v.split_row = reinterpret_cast<int32_t*>(p);
    p += (size_t)MAX_SPLIT_ROWS * 4;
    v.split_nch = reinterpret_cast<int32_t*>(p);
    p += (size_t)MAX_SPLIT_ROWS * 4;
    v.chunk_map = reinterpret_cast<int32_t*>(p);
    p += MAP_BYTES;
    v.partials = reinterpret_cast<float*>(p);
    return v;
}

__global__ void k_reset(unsigned char* scratch) {
    Header* h = reinterpret_cast<Header*>(scratch);
    h->work = 0;
    h->nsplit = 0;
    h->nchunks = 0;
    h->overflow = 0;
    h->err = 0;
}

// Rows longer than split_len reserve a split-row entry and a range of chunk slots.
__global__ void k_register(unsigned char* scratch, const int64_t* rowptr, int64_t n, int64_t split_len,
                           int chunk_cap) {
    View v = view_of(scratch);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t len = rowptr[r + 1] - rowptr[r];
        if (len <= split_len) continue;
        const int nch = (int)((len + split_len - 1) / split_len);
        const int i = atomicAdd(&v.hdr->nsplit, 1);
        const int b = atomicAdd(&v.hdr->nchunks, nch);
        if (i >= MAX_SPLIT_ROWS || b + nch > chunk_cap) {  // excluded by the host-side bound
            atomicExch(&v.hdr->overflow, 1);
            continue;
        }
        v.split_base[i] = b;
        v.split_count[i] = 0;
        v.split_row[i] = (int32_t)r;
        v.split_nch[i] = nch;
        for (int c = 0; c < nch; ++c) v.chunk_map[b + c] = i;
    }
}

template <typename ST, int VEC, int CPL, int G, bool HV>
__global__ void __launch_bounds__(256) k_propagate_noalloc(prop::Args a, unsigned char* scratch) {
    using K = prop::Kern<ST, VEC, CPL, G, HV, true>;  // caller's CSR: check every index
    View v = view_of(scratch);
    const int lane = threadIdx.x & 31;
    const int g = lane / G, lg = lane % G;
    // ok_split is false only when the split table overflowed (the host bound excludes it);
    // long rows then run whole on the warp path instead of being left out
    const bool ok_split = v.hdr->overflow == 0;
    const int64_t nchunks = ok_split ? v.hdr->nchunks : 0;
    const int64_t nblocks = (a.n + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
    const int64_t total = nchunks + nblocks;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(&v.hdr->work, 1ull);
        t = __shfl_sync(prop::FULL, t, 0);
        if ((int64_t)t >= total) break;
        if ((int64_t)t < nchunks) {
            const int i = v.chunk_map[t];
            Task task;
            task.a = v.split_row[i];
            task.b = i;
            task.c = (int32_t)(t - v.split_base[i]);
            task.k = v.split_nch[i];
            K::split_chunk(a, task, lane, g, lg);
        } else {
            const int64_t rb = ((int64_t)t - nchunks) * ROWS_PER_BLOCK;
            const int64_t re = min(a.n, rb + ROWS_PER_BLOCK);
            if (ok_split) K::template rows_coop<true>(a, rb, re, lane, g, lg);
            else K::template rows_coop<false>(a, rb, re, lane, g, lg);
        }
        __syncwarp();
    }
}

template <typename ST, int VEC, bool HV>
cudaError_t launch_shape(const Shape& sh, const prop::Args& a, unsigned char* scratch, int sms,
                         cudaStream_t s) {
    auto go = [&](auto kern) -> cudaError_t {
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0);
        if (e != cudaSuccess) return e;
        if (bps < 1) bps = 1;
        kern<<<bps * sms, 256, 0, s>>>(a, scratch);
        return cudaGetLastError();
    };
    if (sh.cpl == 1) {
        switch (sh.G) {
            case 1: return go(k_propagate_noalloc<ST, VEC, 1, 1, HV>);
            case 2: return go(k_propagate_noalloc<ST, VEC, 1, 2, HV>);
            case 4: return go(k_propagate_noalloc<ST, VEC, 1, 4, HV>);
            case 8: return go(k_propagate_noalloc<ST, VEC, 1, 8, HV>);
            case 16: return go(k_propagate_noalloc<ST, VEC, 1, 16, HV>);
            case 32: return go(k_propagate_noalloc<ST, VEC, 1, 32, HV>);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (sh.cpl) {
        case 2: return go(k_propagate_noalloc<ST, VEC, 2, 32, HV>);
        case 4: return go(k_propagate_noalloc<ST, VEC, 4, 32, HV>);
        case 8: return go(k_propagate_noalloc<ST, VEC, 8, 32, HV>);
        default: return cudaErrorInvalidValue;
    }
}

// Per-device set-up: the device address of g_scratch and the SM count.
struct DeviceSetup {
    bool done = false;
    unsigned char* scratch = nullptr;
    int sms = 0;
};
constexpr int MAX_DEVICES = 64;
static DeviceSetup g_setup[MAX_DEVICES];
static std::mutex g_setup_mu;

cudaError_t setup_device(int dev, DeviceSetup* out) {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    DeviceSetup& st = g_setup[dev];
    if (!st.done) {
        void* ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_scratch);
        if (e != cudaSuccess) return e;
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        st.scratch = static_cast<unsigned char*>(ptr);
        st.sms = sms;
        st.done = true;
    }
    *out = st;
    return cudaSuccess;
}

}  // namespace noalloc
}  // namespace cleora

using namespace cleora;

extern "C" int cleora_noalloc_limits(int d, int64_t* scratch_bytes, int64_t* max_split_chunks) {
    if (d < 8 || d > 1024 || d % 8) return CLEORA_ERR_INVALID_ARG;
    if (scratch_bytes) *scratch_bytes = (int64_t)noalloc::SCRATCH_BYTES;
    if (max_split_chunks) {
        int64_t slots = (int64_t)(noalloc::PARTIAL_BYTES / ((size_t)d * sizeof(float)));
        *max_split_chunks = slots < noalloc::MAX_CHUNKS ? slots : noalloc::MAX_CHUNKS;
    }
    return CLEORA_OK;
}

extern "C" int cleora_propagate_noalloc(const int64_t* rowptr, const int32_t* col, const float* val,
                                        int64_t n, int64_t nnz, const void* T_in, void* T_out, int d,
                                        cleora_dtype storage, int64_t split_len, void* cuda_stream) {
    using namespace noalloc;
    if (n < 0 || nnz < 0 || n >= ((int64_t)1 << 31)) return CLEORA_ERR_INVALID_ARG;
    if (storage != CLEORA_F32 && storage != CLEORA_BF16) return CLEORA_ERR_INVALID_ARG;
    int64_t cap = 0;
    if (cleora_noalloc_limits(d, nullptr, &cap) != CLEORA_OK) return CLEORA_ERR_INVALID_ARG;
    if (n == 0) return CLEORA_OK;
    if (!rowptr || !T_in || !T_out || (nnz > 0 && !col)) return CLEORA_ERR_INVALID_ARG;
    // Chunk slots needed are at most 2 * nnz / split_len (every split row is longer than
    // split_len); the smallest split length the scratch can always hold is therefore:
    const int64_t min_len = (2 * nnz + cap - 1) / cap;
    if (split_len == 0) split_len = min_len > 256 ? min_len : 256;
    if (split_len < min_len || split_len < 1) return CLEORA_ERR_INVALID_ARG;
    // The kernel gathers and stores 16-byte vectors of T and reads rowptr, col and val
    // with their natural widths: a misaligned view (a tensor slice with a storage offset)
    // would fault on the device, so it is refused here, before anything is launched.
    const uintptr_t tin = reinterpret_cast<uintptr_t>(T_in), tout = reinterpret_cast<uintptr_t>(T_out);
    if (((tin | tout) & 15) || (reinterpret_cast<uintptr_t>(rowptr) & 7) ||
        (reinterpret_cast<uintptr_t>(col) & 3) || (reinterpret_cast<uintptr_t>(val) & 3))
        return CLEORA_ERR_INVALID_ARG;
    const uintptr_t tbytes = (uintptr_t)n * (uintptr_t)d * (storage == CLEORA_F32 ? 4u : 2u);
    if (tin < tout + tbytes && tout < tin + tbytes) return CLEORA_ERR_INVALID_ARG;  // overlap

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return CLEORA_ERR_CUDA;
    DeviceSetup st;
    if (setup_device(dev, &st) != cudaSuccess) {
        cudaGetLastError();
        return CLEORA_ERR_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    View v = view_of(st.scratch);

    Shape sh;
    {
        const int es = storage == CLEORA_F32 ? 4 : 2;
        sh.vec = 16;
        sh.chunks = d * es / 16;
        int g = 1;
        while (g < sh.chunks && g < 32) g <<= 1;
        sh.G = g;
        int c = 1;
        while (c * 32 < sh.chunks) c <<= 1;
        sh.cpl = sh.chunks <= 32 ? 1 : c;
        sh.mode = 1;
    }
    prop::Args a;
    a.rowptr = rowptr;
    a.col = col;
    a.val = val;
    a.Tin = static_cast<const unsigned char*>(T_in);
    a.Tout = static_cast<unsigned char*>(T_out);
    a.n = n;
    a.nnz = nnz;
    a.row_bytes = (int64_t)d * (storage == CLEORA_F32 ? 4 : 2);
    a.chunks = sh.chunks;
    a.d = d;
    a.split_len = split_len;
    a.skip_len = split_len;
    a.tasks = nullptr;
    a.ntasks = 0;
    a.counter = nullptr;
    a.split_base = v.split_base;
    a.split_count = v.split_count;
    a.partials = v.partials;
    a.err = &v.hdr->err;

    k_reset<<<1, 1, 0, s>>>(st.scratch);
    k_register<<<grid_for(n, 256, st.sms), 256, 0, s>>>(st.scratch, rowptr, n, split_len, (int)cap);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        const bool hv = val != nullptr;
        if (storage == CLEORA_F32)
            e = hv ? launch_shape<float, 16, true>(sh, a, st.scratch, st.sms, s)
                   : launch_shape<float, 16, false>(sh, a, st.scratch, st.sms, s);
        else
            e = hv ? launch_shape<__nv_bfloat16, 16, true>(sh, a, st.scratch, st.sms, s)
                   : launch_shape<__nv_bfloat16, 16, false>(sh, a, st.scratch, st.sms, s);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorInvalidValue ? CLEORA_ERR_INVALID_ARG : CLEORA_ERR_CUDA;
    }
    return CLEORA_OK;
}
