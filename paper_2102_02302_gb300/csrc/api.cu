// C ABI of the library (declared in include/cleora.h): context, memory, state machine.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"

namespace cleora {

int fail(cleora_ctx* ctx, int status, const char* fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return status;
}

int cuda_fail(cleora_ctx* ctx, cudaError_t e, const char* what, const char* file, int line) {
    const char* base = strrchr(file, '/');
    fail(ctx, 0, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), base ? base + 1 : file, line);
    cudaGetLastError();  // clear a non-sticky error so the context stays usable
    return e == cudaErrorMemoryAllocation ? CLEORA_ERR_OOM : CLEORA_ERR_CUDA;
}

int dalloc_bytes(cleora_ctx* ctx, void** p, size_t bytes) {
    *p = nullptr;
    if (ctx->inject_alloc_fail >= 0 && ctx->inject_alloc_fail-- == 0)
        return fail(ctx, CLEORA_ERR_OOM, "injected allocation failure (test hook)");
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {  // the pool keeps freed blocks: hand the unused ones back, try again
        cudaGetLastError();
        cudaMemPoolTrimTo(ctx->pool, 0);
        e = cudaMallocFromPoolAsync(p, bytes ? bytes : 16, ctx->pool, ctx->stream);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return fail(ctx, CLEORA_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes,
                    cudaGetErrorString(e));
    }
    return CLEORA_OK;
}

void dfree(cleora_ctx* ctx, void* p) {
    if (p) cudaFreeAsync(p, ctx->stream);
}

namespace {

#define GUARD(ctx)                                                                      \
    if (!(ctx)) return CLEORA_ERR_INVALID_ARG;                                          \
    DeviceGuard guard_((ctx)->device);                                                  \
    if (!guard_.ok) return fail(ctx, CLEORA_ERR_CUDA, "cannot select device %d", (ctx)->device)

void embeddings_release(cleora_ctx* ctx) {
    dfree_null(ctx, ctx->T[0]);
    dfree_null(ctx, ctx->T[1]);
    ctx->inited = false;
    ctx->iteration = 0;
    ctx->cur = 0;
}

size_t elem_size(cleora_dtype t) { return t == CLEORA_F32 ? 4 : 2; }

bool valid_dtype(int t) { return t == CLEORA_F32 || t == CLEORA_BF16; }

int copy_out(cleora_ctx* ctx, void* out, const void* dev, size_t bytes, int out_on_device) {
    if (bytes == 0) return CLEORA_OK;
    CL_CUDA(ctx, cudaMemcpyAsync(out, dev, bytes,
                                 out_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 ctx->stream));
    if (!out_on_device) CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return CLEORA_OK;
}

int check_err_flag(cleora_ctx* ctx) {
    int flag = 0;
    CL_CUDA(ctx, read_back(ctx, &flag, ctx->err_flag, sizeof(int), ctx->stream, false));
    CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (flag) {
        CL_CUDA(ctx, cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->stream));
        return fail(ctx, CLEORA_ERR_DEVICE, "a kernel reported an error (flags 0x%x: 1 column index out of "
                    "range, 2 bad task variant, 4 a shared-memory ring wait ran out)", flag);
    }
    return CLEORA_OK;
}

// Current embeddings -> `out` as `dtype` (device or host); host copies go through a
// bounded staging buffer when a conversion is needed.
// Device address of pinned host memory registered with CUDA (mapped into the device's
// address space), or NULL for pageable memory.
void* host_mapped(void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int export_T(cleora_ctx* ctx, void* out, cleora_dtype dtype, int out_on_device) {
    const int64_t count = ctx->g.n * (int64_t)ctx->d;
    if (count == 0) return CLEORA_OK;
    const void* src = ctx->T[ctx->cur];
    if (dtype == ctx->dtype) return copy_out(ctx, out, src, count * elem_size(dtype), out_on_device);
    if (out_on_device) return convert_impl(ctx, src, ctx->dtype, out, dtype, count);
    void* mapped = host_mapped(out);
    if (mapped) {  // pinned host memory: convert straight into it over the host link
        CL_TRY(convert_impl(ctx, src, ctx->dtype, mapped, dtype, count));
        CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return CLEORA_OK;
    }
    const int64_t slice = (int64_t)1 << 26;  // elements per staging slice
    void* stage = nullptr;
    CL_TRY(dalloc_bytes(ctx, &stage, (size_t)std::min(count, slice) * elem_size(dtype)));
    int rc = CLEORA_OK;
    for (int64_t off = 0; off < count && rc == CLEORA_OK; off += slice) {
        const int64_t c = std::min(slice, count - off);
        rc = convert_impl(ctx, static_cast<const char*>(src) + off * elem_size(ctx->dtype), ctx->dtype,
                          stage, dtype, c);
        if (rc == CLEORA_OK)
            rc = copy_out(ctx, static_cast<char*>(out) + off * elem_size(dtype), stage,
                          c * elem_size(dtype), 0);
    }
    dfree(ctx, stage);
    return rc;
}

int import_T(cleora_ctx* ctx, const void* in, cleora_dtype dtype, int in_on_device) {
    const int64_t count = ctx->g.n * (int64_t)ctx->d;
    if (count == 0) return CLEORA_OK;
    void* dst = ctx->T[ctx->cur];
    if (in_on_device) return convert_impl(ctx, in, dtype, dst, ctx->dtype, count);
    if (dtype == ctx->dtype) {
        CL_CUDA(ctx, cudaMemcpyAsync(dst, in, count * elem_size(dtype), cudaMemcpyHostToDevice, ctx->stream));
        CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return CLEORA_OK;
    }
    void* mapped = host_mapped(const_cast<void*>(in));
    if (mapped) {  // pinned host memory: convert straight out of it over the host link
        CL_TRY(convert_impl(ctx, mapped, dtype, dst, ctx->dtype, count));
        CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        return CLEORA_OK;
    }
    const int64_t slice = (int64_t)1 << 26;
    void* stage = nullptr;
    CL_TRY(dalloc_bytes(ctx, &stage, (size_t)std::min(count, slice) * elem_size(dtype)));
    int rc = CLEORA_OK;
    for (int64_t off = 0; off < count && rc == CLEORA_OK; off += slice) {
        const int64_t c = std::min(slice, count - off);
        cudaError_t e = cudaMemcpyAsync(stage, static_cast<const char*>(in) + off * elem_size(dtype),
                                        c * elem_size(dtype), cudaMemcpyHostToDevice, ctx->stream);
        if (e != cudaSuccess) { rc = cuda_fail(ctx, e, "copy in", __FILE__, __LINE__); break; }
        rc = convert_impl(ctx, stage, dtype, static_cast<char*>(dst) + off * elem_size(ctx->dtype),
                          ctx->dtype, c);
        if (rc == CLEORA_OK) {
            e = cudaStreamSynchronize(ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "copy in", __FILE__, __LINE__);
        }
    }
    dfree(ctx, stage);
    return rc;
}

}  // namespace

namespace {
struct Bytes32 {
    unsigned char b[32];
};
__global__ void k_put_bytes(unsigned char* dst, Bytes32 v, int n) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = v.b[i];
}
// Device bytes -> mapped host memory: 16-byte words when both ends and the size allow it.
__global__ void k_read_back(unsigned char* dst, const unsigned char* src, size_t n) {
    const size_t t0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x, T = (size_t)gridDim.x * blockDim.x;
    if ((((uintptr_t)dst | (uintptr_t)src | n) & 15) == 0) {
        for (size_t i = t0; i < n / 16; i += T)
            reinterpret_cast<uint4*>(dst)[i] = reinterpret_cast<const uint4*>(src)[i];
    } else {
        for (size_t i = t0; i < n; i += T) dst[i] = src[i];
    }
}
}  // namespace

cudaError_t read_back(cleora_ctx* ctx, void* host, const void* dev, size_t bytes, cudaStream_t s,
                      bool by_kernel) {
    if (bytes == 0) return cudaSuccess;
    unsigned char* h = static_cast<unsigned char*>(host);
    const unsigned char* d = static_cast<const unsigned char*>(dev);
    if (!ctx->host_stage) {  // (contexts always have one; kept for safety)
        cudaError_t e = cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, s);
        return e == cudaSuccess ? cudaStreamSynchronize(s) : e;
    }
    do {
        const size_t c = std::min(bytes, HOST_STAGE_BYTES);
        cudaError_t e;
        if (by_kernel) {
            k_read_back<<<(unsigned)std::min<size_t>(16, (c + 4095) / 4096), 256, 0, s>>>(ctx->host_stage_dev, d, c);
            ctx->launches += 1;
            e = cudaGetLastError();
        } else {
            e = cudaMemcpyAsync(ctx->host_stage, d, c, cudaMemcpyDeviceToHost, s);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return e;
        memcpy(h, ctx->host_stage, c);
        h += c;
        d += c;
        bytes -= c;
    } while (bytes > 0);
    return cudaSuccess;
}

cudaError_t put_bytes(cleora_ctx* ctx, void* dev, const void* host, size_t bytes, cudaStream_t s) {
    if (bytes > sizeof(Bytes32)) return cudaErrorInvalidValue;
    if (bytes == 0) return cudaSuccess;
    Bytes32 v;
    memcpy(v.b, host, bytes);
    k_put_bytes<<<1, 32, 0, s>>>(static_cast<unsigned char*>(dev), v, (int)bytes);
    ctx->launches += 1;
    return cudaGetLastError();
}


void ctx_release_all(cleora_ctx* ctx) {
    plan_release(ctx);
    embeddings_release(ctx);
    graph_release(ctx);
}

}  // namespace cleora

using namespace cleora;

extern "C" {

const char* cleora_status_string(int status) {
    switch (status) {
        case CLEORA_OK: return "ok";
        case CLEORA_ERR_INVALID_ARG: return "invalid argument";
        case CLEORA_ERR_OOM: return "out of memory";
        case CLEORA_ERR_CUDA: return "CUDA error";
        case CLEORA_ERR_STATE: return "call out of order";
        case CLEORA_ERR_TIMEOUT: return "timed out";
        case CLEORA_ERR_REJECTED: return "rejected";
        case CLEORA_ERR_DEVICE: return "device-reported error";
        case CLEORA_ERR_CANCELLED: return "cancelled";
        default: return "unknown status";
    }
}

int cleora_create(cleora_ctx** out, int device, void* cuda_stream) {
    return ctx_create(out, device, cuda_stream, nullptr);
}

}  // extern "C"

namespace cleora {

int ctx_create(cleora_ctx** out, int device, void* cuda_stream, cudaMemPool_t shared_pool) {
    if (!out) return CLEORA_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return CLEORA_ERR_INVALID_ARG;
    }
    cleora_ctx* ctx = new (std::nothrow) cleora_ctx();
    if (!ctx) return CLEORA_ERR_OOM;
    ctx->device = device;
    DeviceGuard guard(device);
    int rc = CLEORA_OK;
    do {
        if (!guard.ok) { rc = CLEORA_ERR_CUDA; break; }
        cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
        if (e != cudaSuccess) { rc = CLEORA_ERR_CUDA; break; }
        if (cuda_stream) {
            ctx->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
            if (e != cudaSuccess) { rc = CLEORA_ERR_CUDA; break; }
            ctx->own_stream = true;
        }
        if (shared_pool) {
            ctx->pool = shared_pool;
            ctx->own_pool = false;
        } else {
            cudaMemPoolProps props;
            memset(&props, 0, sizeof(props));
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = device;
            e = cudaMemPoolCreate(&ctx->pool, &props);
            if (e != cudaSuccess) { rc = CLEORA_ERR_CUDA; break; }
            uint64_t keep = UINT64_MAX;  // keep freed blocks for reuse until destroy
            cudaMemPoolSetAttribute(ctx->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        if ((rc = dalloc(ctx, &ctx->err_flag, 1)) != CLEORA_OK) break;
        e = cudaHostAlloc((void**)&ctx->host_stage, HOST_STAGE_BYTES, cudaHostAllocMapped);
        if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&ctx->host_stage_dev, ctx->host_stage, 0);
        if (e != cudaSuccess) {
            cudaGetLastError();
            if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
            ctx->host_stage = nullptr;
            rc = CLEORA_ERR_OOM;
            break;
        }
        e = cudaMemsetAsync(ctx->err_flag, 0, sizeof(int), ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) { rc = CLEORA_ERR_CUDA; break; }
    } while (0);
    if (rc != CLEORA_OK) {
        cudaGetLastError();
        cleora_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return CLEORA_OK;
}

}  // namespace cleora

extern "C" {

void cleora_destroy(cleora_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        if (ctx->stream) cudaStreamSynchronize(ctx->stream);
        if (ctx->pool) {
            plan_release(ctx);
            embeddings_release(ctx);
            graph_release(ctx);
            dfree_null(ctx, ctx->err_flag);
            if (ctx->stream) cudaStreamSynchronize(ctx->stream);
            if (ctx->own_pool) cudaMemPoolDestroy(ctx->pool);
        }
        if (ctx->host_stage) cudaFreeHost(ctx->host_stage);
        if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
        cudaGetLastError();
    }
    delete ctx;
}

const char* cleora_last_error(const cleora_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int cleora_sync(cleora_ctx* ctx) {
    GUARD(ctx);
    CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return check_err_flag(ctx);
}

int cleora_graph_build(cleora_ctx* ctx, const uint64_t* src, const uint64_t* dst, const float* weights,
                       int64_t num_edges, int directed, int inputs_on_device) {
    GUARD(ctx);
    if (num_edges < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "num_edges < 0");
    if (num_edges > 0 && (!src || !dst)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null edge array");
    if (num_edges > ((int64_t)1 << 40)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "too many edges");
    plan_release(ctx);
    embeddings_release(ctx);
    graph_release(ctx);
    if (num_edges == 0) {
        ctx->g.built = true;
        return plan_build(ctx, 1, 1);
    }
    const uint64_t* s = src;
    const uint64_t* t = dst;
    const float* w = weights;
    void *ds = nullptr, *dt = nullptr, *dw = nullptr;
    int rc = CLEORA_OK;
    if (!inputs_on_device) {
        const size_t eb = (size_t)num_edges * sizeof(uint64_t);
        do {
            if ((rc = dalloc_bytes(ctx, &ds, eb))) break;
            if ((rc = dalloc_bytes(ctx, &dt, eb))) break;
            if (weights && (rc = dalloc_bytes(ctx, &dw, (size_t)num_edges * sizeof(float)))) break;
            cudaError_t e = cudaMemcpyAsync(ds, src, eb, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess) e = cudaMemcpyAsync(dt, dst, eb, cudaMemcpyHostToDevice, ctx->stream);
            if (e == cudaSuccess && weights)
                e = cudaMemcpyAsync(dw, weights, (size_t)num_edges * sizeof(float), cudaMemcpyHostToDevice,
                                    ctx->stream);
            if (e != cudaSuccess) rc = cuda_fail(ctx, e, "edge upload", __FILE__, __LINE__);
        } while (0);
        s = static_cast<const uint64_t*>(ds);
        t = static_cast<const uint64_t*>(dt);
        w = static_cast<const float*>(dw);
    }
    if (rc == CLEORA_OK) rc = graph_build_impl(ctx, s, t, w, num_edges, directed ? 1 : 0);
    dfree(ctx, ds);
    dfree(ctx, dt);
    dfree(ctx, dw);
    if (rc == CLEORA_OK) rc = plan_ensure(ctx);
    if (rc != CLEORA_OK) {
        plan_release(ctx);
        graph_release(ctx);
    }
    return rc;
}

int cleora_num_nodes(const cleora_ctx* ctx, int64_t* n) {
    if (!ctx || !n) return CLEORA_ERR_INVALID_ARG;
    if (!ctx->g.built) return CLEORA_ERR_STATE;
    *n = ctx->g.n;
    return CLEORA_OK;
}

int cleora_num_entries(const cleora_ctx* ctx, int64_t* nnz) {
    if (!ctx || !nnz) return CLEORA_ERR_INVALID_ARG;
    if (!ctx->g.built) return CLEORA_ERR_STATE;
    *nnz = ctx->g.nnz;
    return CLEORA_OK;
}

int cleora_graph_info(const cleora_ctx* ctx, int64_t* n, int64_t* nnz, int* has_val, int64_t* max_row_len) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    if (!ctx->g.built) return CLEORA_ERR_STATE;
    if (n) *n = ctx->g.n;
    if (nnz) *nnz = ctx->g.nnz;
    if (has_val) *has_val = ctx->g.has_val ? 1 : 0;
    if (max_row_len) *max_row_len = ctx->g.max_row_len;
    return CLEORA_OK;
}

int cleora_node_ids(cleora_ctx* ctx, uint64_t* out, int out_on_device) {
    GUARD(ctx);
    if (!ctx->g.built) return fail(ctx, CLEORA_ERR_STATE, "no graph");
    if (!out && ctx->g.n) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null output");
    return copy_out(ctx, out, ctx->g.ids, ctx->g.n * sizeof(uint64_t), out_on_device);
}

int cleora_get_csr(cleora_ctx* ctx, int64_t* rowptr, int32_t* col, float* val, float* inv_deg, double* deg,
                   int out_on_device) {
    GUARD(ctx);
    const Graph& g = ctx->g;
    if (!g.built) return fail(ctx, CLEORA_ERR_STATE, "no graph");
    if (g.n == 0) {
        if (rowptr) {
            int64_t z = 0;
            if (out_on_device) CL_CUDA(ctx, put_bytes(ctx, rowptr, &z, 8, ctx->stream));
            else *rowptr = 0;
            CL_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        }
        return CLEORA_OK;
    }
    if (rowptr) CL_TRY(copy_out(ctx, rowptr, g.rowptr, (g.n + 1) * sizeof(int64_t), out_on_device));
    if (col && g.nnz) {  // ascending column order per row
        if (out_on_device) {
            CL_TRY(col_out(ctx, col));
        } else {
            int32_t* tmp = nullptr;
            CL_TRY(dalloc(ctx, &tmp, (size_t)g.nnz));
            int rc = col_out(ctx, tmp);
            if (rc == CLEORA_OK) rc = copy_out(ctx, col, tmp, g.nnz * sizeof(int32_t), 0);
            dfree(ctx, tmp);
            CL_TRY(rc);
        }
    }
    if (inv_deg) CL_TRY(copy_out(ctx, inv_deg, g.inv_deg, g.n * sizeof(float), out_on_device));
    if (deg) CL_TRY(copy_out(ctx, deg, g.deg, g.n * sizeof(double), out_on_device));
    if (val && g.nnz) {
        if (out_on_device) {
            CL_TRY(csr_values_out(ctx, val));
        } else {
            float* tmp = nullptr;
            CL_TRY(dalloc(ctx, &tmp, (size_t)g.nnz));
            int rc = csr_values_out(ctx, tmp);
            if (rc == CLEORA_OK) rc = copy_out(ctx, val, tmp, g.nnz * sizeof(float), 0);
            dfree(ctx, tmp);
            CL_TRY(rc);
        }
    }
    return CLEORA_OK;
}

int cleora_init(cleora_ctx* ctx, int d, uint64_t seed, cleora_dtype storage) {
    GUARD(ctx);
    if (!ctx->g.built) return fail(ctx, CLEORA_ERR_STATE, "init before graph_build");
    if (d < 8 || d > 1024 || d % 8 != 0)
        return fail(ctx, CLEORA_ERR_INVALID_ARG, "d must be a multiple of 8 in [8, 1024], got %d", d);
    if (!valid_dtype(storage)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "unknown storage type");
    embeddings_release(ctx);
    ctx->d = d;
    ctx->dtype = storage;
    const size_t bytes = (size_t)ctx->g.n * d * elem_size(storage);
    if (ctx->g.n) {
        CL_TRY(dalloc_bytes(ctx, &ctx->T[0], bytes));
        int rc = dalloc_bytes(ctx, &ctx->T[1], bytes);
        if (rc) { embeddings_release(ctx); return rc; }
    }
    int rc = plan_ensure(ctx);
    if (rc == CLEORA_OK) rc = init_impl(ctx, seed);
    if (rc == CLEORA_OK) rc = hot_partition(ctx);
    if (rc == CLEORA_OK) rc = ring_tensor_maps(ctx);
    if (rc != CLEORA_OK) { embeddings_release(ctx); return rc; }
    ctx->cur = 0;
    ctx->iteration = 0;
    ctx->inited = true;
    return CLEORA_OK;
}

int cleora_propagate(cleora_ctx* ctx, int iters, float* out, int out_on_device) {
    GUARD(ctx);
    if (!ctx->inited) return fail(ctx, CLEORA_ERR_STATE, "propagate before init");
    if (iters < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "iters < 0");
    CL_TRY(plan_ensure(ctx));
    for (int it = 0; it < iters; ++it) {
        CL_TRY(propagate_step(ctx, ctx->T[ctx->cur], ctx->T[ctx->cur ^ 1]));
        ctx->cur ^= 1;
        ctx->iteration += 1;
    }
    if (out) CL_TRY(export_T(ctx, out, CLEORA_F32, out_on_device));
    if (out && !out_on_device) return check_err_flag(ctx);
    return CLEORA_OK;
}

int cleora_iteration(const cleora_ctx* ctx, int* k) {
    if (!ctx || !k) return CLEORA_ERR_INVALID_ARG;
    if (!ctx->inited) return CLEORA_ERR_STATE;
    *k = ctx->iteration;
    return CLEORA_OK;
}

int cleora_get_embeddings(cleora_ctx* ctx, void* out, cleora_dtype dtype, int out_on_device) {
    GUARD(ctx);
    if (!ctx->inited) return fail(ctx, CLEORA_ERR_STATE, "no embeddings");
    if (!valid_dtype(dtype)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "unknown dtype");
    if (!out && ctx->g.n) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null output");
    return export_T(ctx, out, dtype, out_on_device);
}

int cleora_set_embeddings(cleora_ctx* ctx, const void* in, cleora_dtype dtype, int in_on_device, int iteration) {
    GUARD(ctx);
    if (!ctx->inited) return fail(ctx, CLEORA_ERR_STATE, "set_embeddings before init");
    if (!valid_dtype(dtype)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "unknown dtype");
    if (!in && ctx->g.n) return fail(ctx, CLEORA_ERR_INVALID_ARG, "null input");
    if (iteration < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "iteration < 0");
    CL_TRY(import_T(ctx, in, dtype, in_on_device));
    ctx->iteration = iteration;
    return CLEORA_OK;
}

int cleora_set_option(cleora_ctx* ctx, cleora_option opt, int64_t value) {
    if (!ctx) return CLEORA_ERR_INVALID_ARG;
    switch (opt) {
        case CLEORA_OPT_VEC_BYTES:
            if (value != 0 && value != 8 && value != 16) return fail(ctx, CLEORA_ERR_INVALID_ARG, "vec bytes");
            break;
        case CLEORA_OPT_ROW_MODE:
            if (value < 0 || value > 2) return fail(ctx, CLEORA_ERR_INVALID_ARG, "row mode");
            break;
        case CLEORA_OPT_SPLIT_LEN:
            if (value != 0 && (value < 256 || value > ((int64_t)1 << 30)))
                return fail(ctx, CLEORA_ERR_INVALID_ARG, "split length");
            break;
        case CLEORA_OPT_TASK_NNZ:
            if (value != 0 && (value < 64 || value > ((int64_t)1 << 30)))
                return fail(ctx, CLEORA_ERR_INVALID_ARG, "task size");
            break;
        case CLEORA_OPT_BLOCKS_PER_SM:
            if (value < 0 || value > 8) return fail(ctx, CLEORA_ERR_INVALID_ARG, "blocks per SM");
            break;
        case CLEORA_OPT_HOT_BYTES:
            if (value < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "hot bytes");
            break;
        case CLEORA_OPT_ID_SLOTS:
            if (value < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "id slots");
            break;
        case CLEORA_OPT_STAGING:
            if (value < 0 || value > 3) return fail(ctx, CLEORA_ERR_INVALID_ARG, "staging");
            break;
        case CLEORA_OPT_RING_STAGES:
            if (value != 0 && (value < 2 || value > 4)) return fail(ctx, CLEORA_ERR_INVALID_ARG, "ring stages");
            break;
        case CLEORA_OPT_CHUNK_BYTES:
            if (value < 0) return fail(ctx, CLEORA_ERR_INVALID_ARG, "chunk bytes");
            break;
        case CLEORA_OPT_TEST_RING_WAIT:
            if (value != 0 && value != 1) return fail(ctx, CLEORA_ERR_INVALID_ARG, "test hook");
            break;
        default:
            return fail(ctx, CLEORA_ERR_INVALID_ARG, "unknown option");
    }
    ctx->opt[opt] = value;
    return CLEORA_OK;
}

int cleora_get_option(const cleora_ctx* ctx, cleora_option opt, int64_t* value) {
    if (!ctx || !value || (int)opt < 0 || (int)opt >= OPT_COUNT) return CLEORA_ERR_INVALID_ARG;
    *value = ctx->opt[opt];
    return CLEORA_OK;
}

int cleora_launch_count(const cleora_ctx* ctx, int64_t* launches) {
    if (!ctx || !launches) return CLEORA_ERR_INVALID_ARG;
    *launches = ctx->launches;
    return CLEORA_OK;
}

int cleora_hot_entries(const cleora_ctx* ctx, int64_t* hot_entries) {
    if (!ctx || !hot_entries) return CLEORA_ERR_INVALID_ARG;
    if (!ctx->g.built) return CLEORA_ERR_STATE;
    *hot_entries = (ctx->g.hot_cnt || ctx->g.hot_bits) ? ctx->g.hot_entries : 0;
    return CLEORA_OK;
}

}  // extern "C"
