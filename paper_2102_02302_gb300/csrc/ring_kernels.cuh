// Shared-memory ring propagate kernel: one Cleora iteration T_k = rownorm_L2(M T_{k-1})
// (arXiv 2102.02302, Algorithm 1: multiply by M, then L2-normalise rows) for row shapes a
// full warp covers with one vector per lane (rows of 32 x 8 or 32 x 16 bytes: BF16 d = 128 or
// 256, FP32 d = 64 or 128).
//
// Why: the register kernel keeps only a few gathered rows in flight per lane and spends
// ~25 instructions per CSR entry on shuffles, address arithmetic and unpacking; on graphs
// whose T is far larger than L2 it is bound by gather latency.  Here the gathers leave the
// register file:
//  * A task's entries [K0, K1) stream through windows of 32 consecutive entries, one entry
//    per lane.  Each lane copies the whole T row of its entry with one bulk copy
//    (cp.async.bulk, global -> shared::cta) into its slot of a warp-private ring of S stages;
//    the stage's mbarrier counts the bytes (expect_tx / complete_tx).  A warp instruction
//    thus requests 32 rows, and S - 1 windows stay in flight while one is summed.
//  * The L2 policy is chosen per lane from a hot-entry bitmap: entries pointing at the rows
//    that most entries share are copied evict_last, the rest evict_first.  Rows keep their
//    ascending column order.
//  * Column indices, hot words and values of window m + AHEAD - 1 are staged into a
//    metadata ring with 4-byte cp.async when window m is issued, so the producer never waits
//    on them.
//  * All 32 lanes sum the window out of shared memory (lane l owns bytes [l VEC, (l+1) VEC)
//    of every row) in FP32; BF16 values are added with the mixed-precision add.f32.bf16
//    (exact conversion, one rounding: the same result as converting then adding).  Row ends
//    inside a window close the row: norm by a shuffle butterfly, one streaming store.
//  * G4 (option staging = 3): instead of one bulk copy per row, lanes 0..7 each issue one TMA
//    tensor gather of 4 rows (cp.async.bulk.tensor.2d ... tile::gather4, a tensor map over T
//    with a one-row box) into 4 consecutive slots: 8 requests per window instead of 32.  The
//    L2 policy of a gather follows the majority of its 4 entries' hot bits.
//  * Every mbarrier wait is bounded; a wait that runs out raises bit 4 of the error flag,
//    the warp waits (bounded) for its copies in flight and leaves.
// Summation order is fixed by the graph and the task plan (windows of 32 entries from the
// task start, two-level sums), so results are deterministic.
#pragma once

#include <cuda.h>

#include <cstring>

#include "propagate_kernels.cuh"

namespace cleora {
namespace ring {

constexpr int WIN = 32;         // CSR entries per window: one per lane
constexpr int AHEAD = 8;        // windows whose metadata is requested before they are issued
constexpr uint64_t WAIT_NS = 500000000ull;  // a wait is abandoned after 0.5 s ...
constexpr uint32_t WAIT_TRIES = 1u << 26;   // ... or this many try_wait rounds
constexpr int ERR_WAIT = 4;     // error flag bit: a ring wait ran out

// Metadata slots per warp: a window's slot is rewritten AHEAD + S windows later, after the
// window has been summed (its values are read while summing).
template <int S> constexpr int meta_slots() { return AHEAD + S; }

template <typename ST, int VEC, bool HV, int S>
struct Layout {
    static constexpr int ROW = 32 * VEC;                  // bytes per T row
    static constexpr int STAGE = WIN * ROW;               // bytes per stage
    static constexpr int META = meta_slots<S>();
    static constexpr int META_BYTES = META * WIN * (HV ? 12 : 8);  // col, hot word (, value)
    // per warp: T stages, metadata, S "full" and S "empty" mbarriers; 128-byte multiple
    static constexpr int WARP_BYTES = ((S * STAGE + META_BYTES + 2 * S * 8) + 127) / 128 * 128;
};

// ---- PTX wrappers ----------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{.reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase with the given parity; false when it ran out.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t i = 1; i < WAIT_TRIES; ++i) {
        if (mbar_try(bar, parity)) return true;
        if ((i & 255) == 0 && globaltimer() - t0 > WAIT_NS) return false;
    }
    return false;
}
__device__ __forceinline__ void bulk_row(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar), "l"(pol)
        : "memory");
}
// Four rows r0..r3 of the tensor map's 2-D tensor (box: one row) into dst, dst + ROW, ...
__device__ __forceinline__ void gather4_rows(uint32_t dst, const CUtensorMap* tm, int32_t r0, int32_t r1, int32_t r2,
                                             int32_t r3, uint32_t bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1, {%2, %3, %4, %5, %6}], [%7], %8;" ::"r"(dst),
        "l"(tm), "r"(0), "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(bar), "l"(pol)
        : "memory");
}
__device__ __forceinline__ void cp4(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
template <typename ST, int VEC, bool HV, int S, bool G4 = false>
struct Ring {
    using L = Layout<ST, VEC, HV, S>;
    using K = prop::Kern<ST, VEC, 1, 32, HV>;
    using VT = typename K::VT;
    using Acc = typename K::Acc;
    static constexpr int ROW = L::ROW;
    static constexpr int META = L::META;

    // warp-private state
    unsigned char* tring;   // S stages of WIN rows
    int32_t* mcol;          // META x WIN
    uint32_t* mword;        // META x WIN
    float* mval;            // META x WIN (HV)
    uint32_t bar0;          // shared address of stage 0's "full" mbarrier (stage s at bar0 + 8 s);
                            // the "empty" ones follow at bar0 + 8 (S + s)
    uint32_t phase = 0;     // bit s: parity of stage s's next completion
    uint32_t ephase = 0;    // bit s: parity of stage s's next release
    uint32_t pending = 0;   // bit s: stage s holds an issued, unsummed window
    bool dead = false;      // a wait ran out
    uint64_t pol_hot, pol_cold;
    const CUtensorMap* tmap = nullptr;  // G4: the tensor map of T_in
    int lane;

    __device__ void setup(unsigned char* base, int lane_, bool partitioned) {
        lane = lane_;
        tring = base;
        unsigned char* p = base + S * L::STAGE;
        mcol = reinterpret_cast<int32_t*>(p);
        p += META * WIN * 4;
        mword = reinterpret_cast<uint32_t*>(p);
        p += META * WIN * 4;
        mval = reinterpret_cast<float*>(p);
        if (HV) p += META * WIN * 4;
        bar0 = smem_addr(p);
        if (lane == 0) {
            for (int s = 0; s < 2 * S; ++s) mbar_init(bar0 + 8 * s);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        // with a hot bitmap: hot rows evict_last, the rest evict_first; without: evict_normal
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol_hot));
        if (partitioned)
            asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol_cold));
        else
            asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol_cold));
    }

    // Metadata of window m (entries K0 + 32 m + lane) into its slot; one cp.async group.
    __device__ __forceinline__ void stage_meta(const prop::Args& a, int64_t K0, int64_t K1, int m) {
        const int64_t k = K0 + (int64_t)m * WIN + lane;
        if (k < K1) {
            const int slot = (m % META) * WIN + lane;
            cp4(smem_addr(mcol + slot), a.col + k);
            if (a.hot_bits) cp4(smem_addr(mword + slot), a.hot_bits + (k >> 5));
            if (HV) cp4(smem_addr(mval + slot), a.val + k);
        }
        cp_commit();
    }

    // Issue the row copies of window m into stage m % S.  Requests the metadata of window
    // m + AHEAD - 1 first, so that exactly AHEAD - 1 younger groups exist when waiting for m's.
    __device__ __forceinline__ void issue(const prop::Args& a, int64_t K0, int64_t K1, int m) {
        stage_meta(a, K0, K1, m + AHEAD - 1);
        cp_wait<AHEAD - 1>();
        const int s = m % S;
        const int64_t kb = K0 + (int64_t)m * WIN;
        const int nvalid = (int)min((int64_t)WIN, K1 - kb);
        const uint32_t bar = bar0 + 8 * s;
        if (G4) {  // 4-row tensor gathers; the staged metadata of every lane is read
            __syncwarp();
            const int ngroups = (nvalid + 3) / 4;
            if (lane == 0) mbar_expect(bar, (uint32_t)(ngroups * 4 * ROW + ((a.test_wait_runout && m == 0) ? ROW : 0)));
            __syncwarp();
            if (lane < ngroups) {
                const int base = (m % META) * WIN;
                int32_t r[4];
                int hot = 0;
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const int j = 4 * lane + t;
                    const int jj = j < nvalid ? j : 4 * lane;  // a group's tail repeats its first row
                    r[t] = mcol[base + jj];
                    if (a.hot_bits && j < nvalid) hot += (mword[base + jj] >> ((kb + jj) & 31)) & 1u;
                }
                gather4_rows(smem_addr(tring + s * L::STAGE + 4 * lane * ROW), tmap, r[0], r[1], r[2], r[3], bar,
                             hot >= 2 ? pol_hot : pol_cold);
            }
            pending |= 1u << s;
            return;
        }
        // a.test_wait_runout (test hook): the first window of the warp expects one row more
        // than it copies, so its wait runs out and the error path is taken
        const int extra = (a.test_wait_runout && m == 0) ? ROW : 0;
        if (lane == 0) mbar_expect(bar, (uint32_t)(nvalid * ROW + extra));
        __syncwarp();
        if (lane < nvalid) {
            const int slot = (m % META) * WIN + lane;
            const int32_t c = mcol[slot];
            bool hot = false;
            if (a.hot_bits) hot = (mword[slot] >> ((kb + lane) & 31)) & 1u;
            bulk_row(smem_addr(tring + s * L::STAGE + lane * ROW), a.Tin + (int64_t)c * ROW, ROW, bar,
                     hot ? pol_hot : pol_cold);
        }
        pending |= 1u << s;
    }

    // Wait for window m's rows; false (and the warp is dead) when the wait ran out.
    __device__ __forceinline__ bool ready(const prop::Args& a, int m) {
        const int s = m % S;
        const bool ok = mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
        if (!ok) {  // the stage stays pending: drain() waits for it once more
            if (lane == 0) atomicOr(a.err, ERR_WAIT);
            dead = true;
            return false;
        }
        phase ^= 1u << s;
        pending &= ~(1u << s);
        return true;
    }

    // Stage s has been read by every lane: the release (arrive) / acquire (wait) pair on its
    // "empty" barrier orders those reads before the async-proxy writes that refill it (the
    // producer-acquire pattern of TMA pipelines).
    __device__ __forceinline__ bool release(const prop::Args& a, int s) {
        __syncwarp();
        const uint32_t eb = bar0 + 8 * (S + s);
        if (lane == 0) mbar_arrive(eb);
        const bool ok = mbar_wait(eb, (ephase >> s) & 1u);
        ephase ^= 1u << s;
        if (!ok) {
            if (lane == 0) atomicOr(a.err, ERR_WAIT);
            dead = true;
        }
        return ok;
    }

    // Before leaving after a failed wait: wait (bounded) for every stage still in flight.
    __device__ void drain() {
        for (int s = 0; s < S; ++s)
            if (pending & (1u << s)) {
                mbar_wait(bar0 + 8 * s, (phase >> s) & 1u);
                phase ^= 1u << s;
            }
        pending = 0;
        cp_wait<0>();
    }

    // Add entries j in [j0, j1) of stage s to acc.v (two-level sums: the caller flushes).
    __device__ __forceinline__ void sum(Acc& acc, int s, int m, int j0, int j1) const {
        const unsigned char* base = tring + s * L::STAGE + lane * VEC;
        const float* vals = mval + (m % META) * WIN;
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            const VT x = *reinterpret_cast<const VT*>(base + j * ROW);
            if (HV) {
                K::add_vec(acc, 0, x, vals[j]);
            } else if (std::is_same<ST, __nv_bfloat16>::value) {
#pragma unroll
                for (int k = 0; k < K::W; ++k) {
                    const uint32_t w = prop::word(x, k);
                    acc.v[0][2 * k] = prop::add_lo(acc.v[0][2 * k], w);
                    acc.v[0][2 * k + 1] = prop::add_hi(acc.v[0][2 * k + 1], w);
                }
            } else {
#pragma unroll
                for (int k = 0; k < K::W; ++k) acc.v[0][k] += __uint_as_float(prop::word(x, k));
            }
        }
    }

    // Stream [K0, K1) through the ring; cons(acc-owner) gets each window's entries.
    template <class Cons>
    __device__ __forceinline__ void stream(const prop::Args& a, int64_t K0, int64_t K1, Cons& cons) {
        const int nwin = K1 > K0 ? (int)((K1 - K0 + WIN - 1) / WIN) : 0;
        if (nwin == 0) return;
        for (int m = 0; m < AHEAD - 1; ++m) stage_meta(a, K0, K1, m);
        for (int m = 0; m < S && m < nwin; ++m) issue(a, K0, K1, m);
        for (int m = 0; m < nwin; ++m) {
            if (!ready(a, m)) return;
            const int64_t kb = K0 + (int64_t)m * WIN;
            cons.window(*this, m % S, m, kb, min(K1, kb + WIN));
            if (m + S < nwin) {
                if (!release(a, m % S)) return;
                issue(a, K0, K1, m + S);
            }
        }
        cp_wait<0>();  // metadata groups past the end carry no copies; none stays pending
    }
};

// Rows [rb, re) of a normal task: rowptr in 32-row windows held by the lanes.
template <class R>
struct RowsCons {
    using Acc = typename R::Acc;
    using K = typename R::K;
    const prop::Args& a;
    int64_t r, re, wr;
    int64_t lo, hi;   // this lane's rowptr[wr + lane], rowptr[wr + lane + 1]
    int64_t beg, end; // current row
    Acc acc;
    int lane;

    __device__ RowsCons(const prop::Args& a_, int64_t rb, int64_t re_, int lane_)
        : a(a_), r(rb), re(re_), wr(rb), lo(0), hi(0), lane(lane_) {
        load_window();
        bounds();
        acc.zero();
    }
    __device__ __forceinline__ void load_window() {
        lo = hi = 0;
        if (wr + lane < re) {
            lo = a.rowptr[wr + lane];
            hi = a.rowptr[wr + lane + 1];
        }
    }
    __device__ __forceinline__ void bounds() {
        if (r >= re) return;
        if (r - wr == 32) {
            wr = r;
            load_window();
        }
        beg = __shfl_sync(prop::FULL, lo, (int)(r - wr));
        end = __shfl_sync(prop::FULL, hi, (int)(r - wr));
    }
    // Close every row that ends at position k (empty rows keep their own row).
    __device__ __forceinline__ void close_rows(int64_t k) {
        while (r < re && end == k) {
            if (beg == end) K::load_own(a, acc, r, lane);
            acc.flush();
            K::finish_row(a, acc, r, lane, true, prop::FULL);
            acc.zero();
            ++r;
            bounds();
        }
    }
    __device__ __forceinline__ void window(const R& ring, int s, int m, int64_t kb, int64_t ke) {
        int64_t k = kb;
        for (;;) {
            close_rows(k);
            if (k >= ke || r >= re) break;  // (every entry of [K0, K1) lies in rows < re)
            const int64_t stop = min(end, ke);
            ring.sum(acc, s, m, (int)(k - kb), (int)(stop - kb));
            acc.flush();
            k = stop;
        }
    }
};

// One chunk of a split row: every entry belongs to row t.a.
template <class R>
struct ChunkCons {
    using Acc = typename R::Acc;
    Acc acc;
    __device__ ChunkCons() { acc.zero(); }
    __device__ __forceinline__ void window(const R& ring, int s, int m, int64_t kb, int64_t ke) {
        ring.sum(acc, s, m, 0, (int)(ke - kb));
        acc.flush();
    }
};

template <typename ST, int VEC, bool HV, int S, bool G4>
__global__ void __launch_bounds__(256, 1) k_ring(prop::Args a, const __grid_constant__ CUtensorMap tmap) {
    using R = Ring<ST, VEC, HV, S, G4>;
    using L = typename R::L;
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    R ring;
    ring.setup(smem + (size_t)warp * L::WARP_BYTES, lane, a.hot_bits != nullptr);
    ring.tmap = &tmap;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1ull);
        t = __shfl_sync(prop::FULL, t, 0);
        if (t >= (unsigned long long)a.ntasks) break;
        const Task task = a.tasks[t];
        if (task.c >= 0) {
            const int64_t beg = a.rowptr[task.a], end = a.rowptr[task.a + 1];
            const int64_t k0 = beg + (int64_t)task.c * a.split_len;
            const int64_t k1 = min(end, k0 + a.split_len);
            ChunkCons<R> cons;
            ring.stream(a, k0, k1, cons);
            if (ring.dead) break;
            R::K::split_store_combine(a, task, cons.acc, lane, 0, lane);
        } else {
            RowsCons<R> cons(a, task.a, task.b, lane);
            const int64_t K0 = cons.beg, K1 = a.rowptr[task.b];
            ring.stream(a, K0, K1, cons);
            if (ring.dead) break;
            cons.close_rows(K1);
        }
        __syncwarp();
    }
    if (ring.dead) ring.drain();
}

// Launch helpers (per storage type and vector width, in their own translation units).
// tmap: NULL for one bulk copy per row, else the tensor map of T_in (4-row tensor gathers).
cudaError_t launch_f32_v8(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s, int* grid);
cudaError_t launch_f32_v16(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s, int* grid);
cudaError_t launch_bf16_v8(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s, int* grid);
cudaError_t launch_bf16_v16(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s, int* grid);

// Warps per CTA and CTAs per SM for a per-warp footprint: as many warps as fit in the SM's
// shared memory (up to 8 per CTA), one CTA per SM unless two fit.
template <typename ST, int VEC, bool HV, int S, bool G4>
cudaError_t launch(const prop::Args& a, const CUtensorMap& tmap, int sms, cudaStream_t st, int* grid_out) {
    using L = Layout<ST, VEC, HV, S>;
    auto kern = k_ring<ST, VEC, HV, S, G4>;
    int dev = 0, smem_max = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    int warps = smem_max / L::WARP_BYTES;
    if (warps > 8) warps = 8;
    if (warps < 1) return cudaErrorInvalidValue;
    const int bytes = warps * L::WARP_BYTES;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, bytes);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int grid = per_sm * sms;
    if (grid_out) *grid_out = grid;
    kern<<<grid, warps * 32, bytes, st>>>(a, tmap);
    return cudaGetLastError();
}

template <typename ST, int VEC, bool G4>
cudaError_t launch_stages(const prop::Args& a, const CUtensorMap& tm, bool hv, int stages, int sms, cudaStream_t s,
                          int* grid) {
    switch (stages) {
        case 2: return hv ? launch<ST, VEC, true, 2, G4>(a, tm, sms, s, grid) : launch<ST, VEC, false, 2, G4>(a, tm, sms, s, grid);
        case 3: return hv ? launch<ST, VEC, true, 3, G4>(a, tm, sms, s, grid) : launch<ST, VEC, false, 3, G4>(a, tm, sms, s, grid);
        case 4: return hv ? launch<ST, VEC, true, 4, G4>(a, tm, sms, s, grid) : launch<ST, VEC, false, 4, G4>(a, tm, sms, s, grid);
        default: return cudaErrorInvalidValue;
    }
}

template <typename ST, int VEC>
cudaError_t launch_any(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s,
                       int* grid) {
    if (tmap) return launch_stages<ST, VEC, true>(a, *tmap, hv, stages, sms, s, grid);
    CUtensorMap none;
    memset(&none, 0, sizeof(none));
    return launch_stages<ST, VEC, false>(a, none, hv, stages, sms, s, grid);
}

}  // namespace ring
}  // namespace cleora
