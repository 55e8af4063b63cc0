// T_0 ~ U(-1, 1) (arXiv 2102.02302, Sec. 3.2; Algorithm 1 "Initialize"), deterministic:
//   h = mix(mix(mix(seed) ^ id_i) ^ j),  T_0[i][j] = 2 * (h >> 40) * 2^-24 - 1,
// with mix the splitmix64 output function (Steele, Lea & Flood 2014).  The value is a
// multiple of 2^-23 in [-1, 1), exact in FP32; BF16 storage rounds it to nearest even.
// Also: storage-type conversions used by get/set_embeddings and FP32 output.
#include "common.cuh"

namespace cleora {
namespace {


// One 16-byte vector per thread-iteration: 4 FP32 or 8 BF16 elements.
__global__ void k_init_f32(const uint64_t* ids, int64_t n, int d, uint64_t mseed, float4* T) {
    const int vpr = d / 4;
    const int64_t total = n * vpr;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = v / vpr;
        const uint32_t j = (uint32_t)(v - i * vpr) * 4u;
        const uint64_t p = mix64(mseed ^ ids[i]);
        float4 o;
        o.x = init_value(p, j);
        o.y = init_value(p, j + 1);
        o.z = init_value(p, j + 2);
        o.w = init_value(p, j + 3);
        __stcs(T + v, o);
    }
}

__global__ void k_init_bf16(const uint64_t* ids, int64_t n, int d, uint64_t mseed, uint4* T) {
    const int vpr = d / 8;
    const int64_t total = n * vpr;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < total;
         v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = v / vpr;
        const uint32_t j = (uint32_t)(v - i * vpr) * 8u;
        const uint64_t p = mix64(mseed ^ ids[i]);
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            __nv_bfloat162 h = __floats2bfloat162_rn(init_value(p, j + 2 * k), init_value(p, j + 2 * k + 1));
            w[k] = *reinterpret_cast<uint32_t*>(&h);
        }
        __stcs(T + v, make_uint4(w[0], w[1], w[2], w[3]));
    }
}

__global__ void k_f32_to_bf16(const float* a, __nv_bfloat16* b, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __float2bfloat16_rn(a[i]);
}

__global__ void k_bf16_to_f32(const __nv_bfloat16* a, float* b, int64_t count) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        b[i] = __bfloat162float(a[i]);
}

// The same, 4 elements per step with one vector load and one vector store each (FP32 side
// 16-byte aligned, BF16 side 8-byte aligned), so that a warp's store is one contiguous run.
// The destination may be pinned host memory mapped into the device's address space: the
// stores then cross the host link directly, with no staging copy.
__global__ void k_f32_to_bf16_v4(const uint4* a, uint2* b, int64_t groups) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < groups;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint4 x = a[i];
        const __nv_bfloat162 lo = __floats2bfloat162_rn(__uint_as_float(x.x), __uint_as_float(x.y));
        const __nv_bfloat162 hi = __floats2bfloat162_rn(__uint_as_float(x.z), __uint_as_float(x.w));
        b[i] = make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
    }
}

__global__ void k_bf16_to_f32_v4(const uint2* a, uint4* b, int64_t groups) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < groups;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint2 x = a[i];
        b[i] = make_uint4(x.x << 16, x.x & 0xffff0000u, x.y << 16, x.y & 0xffff0000u);
    }
}

}  // namespace

int init_impl(cleora_ctx* ctx, uint64_t seed) {
    const Graph& g = ctx->g;
    if (g.n == 0) return CLEORA_OK;
    const uint64_t mseed = mix64(seed);  // the same for every element: computed once
    const int64_t vecs = g.n * (ctx->dtype == CLEORA_F32 ? ctx->d / 4 : ctx->d / 8);
    const unsigned grid = grid_for(vecs, 256, ctx->num_sms);
    if (ctx->dtype == CLEORA_F32)
        k_init_f32<<<grid, 256, 0, ctx->stream>>>(g.ids, g.n, ctx->d, mseed,
                                                  static_cast<float4*>(ctx->T[ctx->cur]));
    else
        k_init_bf16<<<grid, 256, 0, ctx->stream>>>(g.ids, g.n, ctx->d, mseed,
                                                   static_cast<uint4*>(ctx->T[ctx->cur]));
    CL_LAUNCHED(ctx);
    return CLEORA_OK;
}

int convert_impl(cleora_ctx* ctx, const void* src, cleora_dtype sdt, void* dst, cleora_dtype ddt,
                 int64_t count) {
    if (count == 0) return CLEORA_OK;
    const size_t es = sdt == CLEORA_F32 ? 4 : 2;
    if (sdt == ddt) {
        CL_CUDA(ctx, cudaMemcpyAsync(dst, src, count * es, cudaMemcpyDeviceToDevice, ctx->stream));
        return CLEORA_OK;
    }
    const uintptr_t fa = reinterpret_cast<uintptr_t>(sdt == CLEORA_F32 ? src : dst);
    const uintptr_t ba = reinterpret_cast<uintptr_t>(sdt == CLEORA_F32 ? dst : src);
    if (count % 4 == 0 && fa % 16 == 0 && ba % 8 == 0) {
        const int64_t groups = count / 4;
        const unsigned grid = grid_for(groups, 256, ctx->num_sms);
        if (sdt == CLEORA_F32)
            k_f32_to_bf16_v4<<<grid, 256, 0, ctx->stream>>>(static_cast<const uint4*>(src), static_cast<uint2*>(dst),
                                                            groups);
        else
            k_bf16_to_f32_v4<<<grid, 256, 0, ctx->stream>>>(static_cast<const uint2*>(src), static_cast<uint4*>(dst),
                                                            groups);
        CL_LAUNCHED(ctx);
        return CLEORA_OK;
    }
    const unsigned grid = grid_for(count, 256, ctx->num_sms);
    if (sdt == CLEORA_F32)
        k_f32_to_bf16<<<grid, 256, 0, ctx->stream>>>(static_cast<const float*>(src),
                                                     static_cast<__nv_bfloat16*>(dst), count);
    else
        k_bf16_to_f32<<<grid, 256, 0, ctx->stream>>>(static_cast<const __nv_bfloat16*>(src),
                                                     static_cast<float*>(dst), count);
    CL_LAUNCHED(ctx);
    return CLEORA_OK;
}

}  // namespace cleora
