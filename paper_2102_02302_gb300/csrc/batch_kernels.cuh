// Batched propagation: many independent graphs packed into one multi-graph CSR and run by
// one persistent launch per iteration step (per kernel family).
//
// A family is (storage type, gather bytes, vectors per lane, lanes per row); graphs whose d
// and storage land in the same family share one launch, whatever their row mode or value
// mode -- each task carries its graph, whose descriptor names the variant.  Every
// task runs exactly the device code the single-graph kernel runs for that graph, on the
// graph's own task plan, so a graph's result in the batch equals its single-graph result
// bit for bit under the same schedule.
#pragma once

#include "propagate_kernels.cuh"

namespace cleora {
namespace batch {

// Per-graph descriptor (device).
struct GDesc {
    int64_t node_off;     // first packed row (packed rowptr index)
    int64_t n;
    int64_t T_off;        // byte offset of the graph's rows in each ping-pong buffer
    int64_t out_off;      // FP32 element offset in the packed output
    int64_t split_off;    // first packed split row
    int64_t partial_off;  // first packed partial float
    int64_t split_len;
    uint64_t mseed;       // mix(seed)
    int32_t d, row_bytes, chunks, iters;
    int32_t variant;      // bit 4: per-entry values, bit 3: row mode 2, bits 0-2: log2(G)
    int32_t dtype;
    int32_t family;
    int32_t pad;
};

struct BTask {
    Task t;
    int32_t g;
    int32_t pad;
};

struct BatchArgs {
    const GDesc* gd;
    const BTask* tasks;
    int64_t ntasks;
    unsigned long long* counter;
    const int64_t* rowptr;
    const int32_t* col;
    const float* val;
    unsigned char* TA;
    unsigned char* TB;
    int64_t total_nnz;
    int64_t* split_base;
    int32_t* split_count;
    float* partials;
    int* err;
    int step;  // 1-based; odd steps read TA and write TB
    int hv;    // the family's graphs have per-entry values
};

constexpr int variant_of(int G, int mode, bool hv) {
    return (hv ? 16 : 0) | (mode == 2 ? 8 : 0) | (G == 1 ? 0 : G == 2 ? 1 : G == 4 ? 2 : G == 8 ? 3 : G == 16 ? 4 : 5);
}

// Vectors in flight per lane: the single-graph kernel's (0: prop::inflight), except lane
// groups of 16-byte gathers, which take 2 so that they fit 4 CTAs/SM.
template <int VEC, int G>
constexpr int batch_inflight() { return VEC == 16 && G < 32 ? 2 : 0; }

template <typename ST, int VEC, int CPL, int G, int MODE, bool HV>
__device__ __forceinline__ void run_task(const prop::Args& a, const Task& t, int lane) {
    using K = prop::Kern<ST, VEC, CPL, G, HV, false, batch_inflight<VEC, G>()>;
    const int g = lane / G, lg = lane % G;
    if (t.c >= 0) K::split_chunk(a, t, lane, g, lg);
    else if (MODE == 1 || G == 32) K::rows_coop(a, t.a, t.b, lane, g, lg);
    else K::rows_group(a, t.a, t.b, g, lg);
}

__device__ __forceinline__ void fill_args(prop::Args& a, const BatchArgs& ba, const GDesc& gd, bool odd) {
    a.rowptr = ba.rowptr + gd.node_off;
    a.col = ba.col;
    a.val = ba.val;
    a.Tin = (odd ? ba.TA : ba.TB) + gd.T_off;
    a.Tout = (odd ? ba.TB : ba.TA) + gd.T_off;
    a.n = gd.n;
    a.nnz = ba.total_nnz;
    a.row_bytes = gd.row_bytes;
    a.chunks = gd.chunks;
    a.d = gd.d;
    a.split_len = gd.split_len;
    a.skip_len = INT64_MAX;
    a.tasks = nullptr;
    a.ntasks = 0;
    a.counter = nullptr;
    a.split_base = ba.split_base + gd.split_off;
    a.split_count = ba.split_count + gd.split_off;
    a.partials = ba.partials + gd.partial_off;
    a.err = ba.err;
    a.hot_cnt = nullptr;
    a.hot_bits = nullptr;
    a.test_wait_runout = 0;
}

// A family is (storage, gather bytes, vectors per lane, lanes per row G, row mode, per-entry
// values): its kernel runs exactly one variant of the single-graph kernel's device code.  A
// task of another variant (none is ever packed into the family) raises bit 2 of the error
// flag.
// CTAs per SM a batch kernel is compiled for: its single-graph twin's where whole warps take
// the rows (4 at 64 registers, no spills), else a notch below it, since a batch task's
// arguments take registers where the twin's sit in the parameter bank.
template <typename ST, int VEC, int CPL, int G, bool HV>
constexpr int batch_min_blocks() {
    constexpr int m = prop::min_blocks<ST, VEC, CPL, G, HV>();
    // (whole-warp rows fit 64 registers at 4 CTAs/SM without spills; lane groups need 80)
    return m >= 8 ? 6 : m >= 6 ? 5 : m >= 4 ? (G == 32 || VEC == 16 ? 4 : 3) : 1;
}

template <typename ST, int VEC, int CPL, int G, int MODE, bool HV>
__global__ void __launch_bounds__(256, (batch_min_blocks<ST, VEC, CPL, G, HV>()))
k_batch(BatchArgs ba) {
    const int lane = threadIdx.x & 31;
    prop::Args a;
    const bool odd = ba.step & 1;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(ba.counter, 1ull);
        t = __shfl_sync(prop::FULL, t, 0);
        if (t >= (unsigned long long)ba.ntasks) break;
        const BTask bt = ba.tasks[t];
        const GDesc& gd = ba.gd[bt.g];
        fill_args(a, ba, gd, odd);
        if (gd.variant == variant_of(G, MODE, HV)) run_task<ST, VEC, CPL, G, MODE, HV>(a, bt.t, lane);
        else if (lane == 0) atomicOr(a.err, 2);
        __syncwarp();
    }
}


template <typename ST, int VEC>
struct BatchLaunch {
    template <int CPL, int G, int MODE = 1>
    static cudaError_t go(const BatchArgs& ba, int sms, cudaStream_t s, int* grid) {
        return ba.hv ? go_v<CPL, G, MODE, true>(ba, sms, s, grid) : go_v<CPL, G, MODE, false>(ba, sms, s, grid);
    }
    template <int CPL, int G, int MODE, bool HV>
    static cudaError_t go_v(const BatchArgs& ba, int sms, cudaStream_t s, int* grid) {
        auto kern = k_batch<ST, VEC, CPL, G, MODE, HV>;
        int bps = 0;
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0);
        if (e != cudaSuccess) return e;
        if (bps < 1) bps = 1;
        if (grid) *grid = bps * sms;
        kern<<<bps * sms, 256, 0, s>>>(ba);
        return cudaGetLastError();
    }
    static cudaError_t run(int cpl, int G, int mode, const BatchArgs& ba, int sms, cudaStream_t s, int* grid) {
        const bool m2 = mode == 2;
        if (cpl == 1) {
            switch (G) {
                case 1: return m2 ? go<1, 1, 2>(ba, sms, s, grid) : go<1, 1>(ba, sms, s, grid);
                case 2: return m2 ? go<1, 2, 2>(ba, sms, s, grid) : go<1, 2>(ba, sms, s, grid);
                case 4: return m2 ? go<1, 4, 2>(ba, sms, s, grid) : go<1, 4>(ba, sms, s, grid);
                case 8: return m2 ? go<1, 8, 2>(ba, sms, s, grid) : go<1, 8>(ba, sms, s, grid);
                case 16: return m2 ? go<1, 16, 2>(ba, sms, s, grid) : go<1, 16>(ba, sms, s, grid);
                case 32: return go<1, 32>(ba, sms, s, grid);
                default: return cudaErrorInvalidValue;
            }
        }
        if (G != 32) return cudaErrorInvalidValue;
        switch (cpl) {
            case 2: return go<2, 32>(ba, sms, s, grid);
            case 4: return go<4, 32>(ba, sms, s, grid);
            case 8: return go<8, 32>(ba, sms, s, grid);
            default: return cudaErrorInvalidValue;
        }
    }
};

cudaError_t launch_batch_f32_v16(int cpl, int G, int mode, const BatchArgs&, int sms, cudaStream_t, int*);
cudaError_t launch_batch_f32_v8(int cpl, int G, int mode, const BatchArgs&, int sms, cudaStream_t, int*);
cudaError_t launch_batch_bf16_v16(int cpl, int G, int mode, const BatchArgs&, int sms, cudaStream_t, int*);
cudaError_t launch_batch_bf16_v8(int cpl, int G, int mode, const BatchArgs&, int sms, cudaStream_t, int*);

}  // namespace batch
}  // namespace cleora
