// Fused propagate kernel: one Cleora iteration T_k = rownorm_L2(M T_{k-1})
// (arXiv 2102.02302, Algorithm 1: multiply by M, then L2-normalise rows).
//
// Design (sm_103a):
//  * Persistent grid; each warp pulls tasks from a global counter.  A task is either a run
//    of consecutive rows holding about `task_nnz` entries, or one chunk of a long row.
//  * A row of T is covered by G lanes, each holding CPL vectors of VEC bytes (16 B or 8 B
//    gathers, coalesced across the G lanes).  The warp has P = 32/G lane groups:
//      mode 1: the groups split one row's entries and add their sums by xor-shuffles;
//      mode 2: each group owns its own rows (more rows in flight for short rows).
//  * Column indices (and values) are read once as a coalesced 32-entry window per warp and
//    broadcast by shuffles; rows keep reusing the window until they leave it.
//  * Accumulation and the row norm are FP32 for both storage types; the norm's reduction is
//    a fixed shuffle butterfly and the output is written once (streaming store).
//  * Long rows are split into chunks; each chunk's FP32 partial sum goes to a slot, and the
//    warp that finishes a row's last chunk adds the slots in a fixed order, normalises and
//    writes the row.  No floating-point atomics, so results are deterministic.
//  * Unit-weight graphs need no per-entry value: M_ab = 1/deg_a is the same for the whole
//    row, and the L2 normalisation removes that common factor exactly, so the kernel sums
//    neighbour rows and normalises.
#pragma once

#include <type_traits>

#include "common.cuh"

// Compile-time tuning knobs, chosen per storage type from measurements on GB300 (the
// 1.4B-edge power-law graph, d = 128):
//   FP32: one batch path, scalar FP32 adds, >= 4 CTAs/SM, 8 gathered vectors in flight per
//         lane (it moves DRAM bytes at the copy bandwidth; occupancy changes nothing);
//   BF16: a separate full-batch path, paired FP32 adds (-3.5% time); 8-byte whole-warp rows
//         (d = 128) at 8 CTAs/SM with 4 vectors in flight per lane (-10% time against 4 CTAs
//         with 8: latency-bound, so more warps beat deeper batches), other shapes at 4 CTAs
//         with 8 in flight;
//   both: L2 policies on the gathers of partitioned rows (hot segment evict_last, cold
//   segment evict_first).  Rows are partitioned only for graphs whose T is much larger than
//   the hot-row budget; the policy of a segment is uniform, so it costs no per-entry work.
// A -D on the command line overrides the choice for both types (experiments).
#ifndef CLEORA_COLD_POLICY
#define CLEORA_COLD_POLICY 0   // gathers of unmarked rows: 0 evict_first, 1 evict_normal
#endif

namespace cleora {
namespace prop {

constexpr unsigned FULL = 0xffffffffu;

struct Args {
    const int64_t* rowptr;
    const int32_t* col;
    const float* val;
    const unsigned char* Tin;
    unsigned char* Tout;
    int64_t n;
    int64_t nnz;
    int64_t row_bytes;
    int chunks;      // vectors per row
    int d;
    int64_t split_len;
    int64_t skip_len = INT64_MAX;  // rows_coop<true> skips longer rows (run as split chunks)
    const Task* tasks;
    int64_t ntasks;
    unsigned long long* counter;
    const int64_t* split_base;
    int32_t* split_count;
    float* partials;
    int* err;
    // Rows partitioned hot-first: the first hot_cnt[r] entries of row r point at rows kept in
    // L2 (gathered evict_last), the rest (in descending column order) are gathered
    // evict_first.  NULL: no partition, every gather evict_normal.
    const int32_t* hot_cnt = nullptr;
    // Hot flags of the entries in place (bit k & 31 of word k >> 5): entries that point at
    // the rows kept in L2, for the shared-memory ring kernel (rows keep ascending order).
    const uint32_t* hot_bits = nullptr;
    int test_wait_runout = 0;  // ring kernel test hook (see CLEORA_OPT_TEST_RING_WAIT)
};

// L2 policy of a gather: in a partitioned row the hot segment is loaded evict_last and the
// cold one evict_first; without a partition every gather is evict_normal.  Made where it is
// used (one instruction) rather than held in registers across the row loops.
__device__ __forceinline__ uint64_t seg_policy(bool partitioned, bool hot) {
    uint64_t p;
    if (!partitioned)
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    else if (hot)
        asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    else
#if CLEORA_COLD_POLICY == 0
        asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
#else
        asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
#endif
    return p;
}

template <typename ST> struct Tune;
// POLICY: gathers carry the L2 policy of their row segment (hot / cold); otherwise they are
// plain loads and the partition only changes the summation order.
template <> struct Tune<float> {
#ifdef CLEORA_POLICY_F32
    static constexpr bool POLICY = CLEORA_POLICY_F32;
#else
    static constexpr bool POLICY = true;
#endif
#ifdef CLEORA_FULL_BATCH
    static constexpr bool FULLB = CLEORA_FULL_BATCH;
#else
    static constexpr bool FULLB = false;
#endif
#ifdef CLEORA_MIN_BLOCKS_F32
    static constexpr int MINB = CLEORA_MIN_BLOCKS_F32;
#else
    static constexpr int MINB = 4;
#endif
#ifdef CLEORA_INFLIGHT_F32
    static constexpr int INFLIGHT = CLEORA_INFLIGHT_F32;
#else
    static constexpr int INFLIGHT = 8;  // gathered vectors in flight per lane and batch
#endif
#ifdef CLEORA_PACKED_F32
    static constexpr bool PACKED = CLEORA_PACKED_F32;
#else
    static constexpr bool PACKED = false;  // paired FP32 adds (add/fma .f32x2)
#endif
};
template <> struct Tune<__nv_bfloat16> {
#ifdef CLEORA_POLICY_BF16
    static constexpr bool POLICY = CLEORA_POLICY_BF16;
#else
    static constexpr bool POLICY = true;
#endif
#ifdef CLEORA_FULL_BATCH
    static constexpr bool FULLB = CLEORA_FULL_BATCH;
#else
    static constexpr bool FULLB = true;
#endif
#ifdef CLEORA_MIN_BLOCKS_BF16
    static constexpr int MINB = CLEORA_MIN_BLOCKS_BF16;
#else
    static constexpr int MINB = 0;  // per shape: min_blocks() below
#endif
#ifdef CLEORA_INFLIGHT_BF16
    static constexpr int INFLIGHT = CLEORA_INFLIGHT_BF16;
#else
    static constexpr int INFLIGHT = 0;  // per shape: inflight() below
#endif
#ifdef CLEORA_PACKED_BF16
    static constexpr bool PACKED = CLEORA_PACKED_BF16;
#else
    static constexpr bool PACKED = true;
#endif
};

template <int VEC> struct VecT;
template <> struct VecT<16> { using T = uint4; };
template <> struct VecT<8> { using T = uint2; };

__device__ __forceinline__ uint4 ld_gather(const uint4* p) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
    return r;
}
__device__ __forceinline__ uint2 ld_gather(const uint2* p) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.v2.u32 {%0,%1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
    return r;
}
__device__ __forceinline__ uint4 ld_gather(const uint4* p, uint64_t pol) {
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint2 ld_gather(const uint2* p, uint64_t pol) {
    uint2 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
        : "=r"(r.x), "=r"(r.y) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ void st_stream(uint4* p, uint4 v) { __stcs(p, v); }
__device__ __forceinline__ void st_stream(uint2* p, uint2 v) { __stcs(p, v); }

__device__ __forceinline__ uint32_t word(const uint4& v, int i) {
    return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ uint32_t word(const uint2& v, int i) { return i == 0 ? v.x : v.y; }
__device__ __forceinline__ void set_word(uint4& v, int i, uint32_t w) {
    if (i == 0) v.x = w; else if (i == 1) v.y = w; else if (i == 2) v.z = w; else v.w = w;
}
__device__ __forceinline__ void set_word(uint2& v, int i, uint32_t w) {
    if (i == 0) v.x = w; else v.y = w;
}

// a += x and a += w * x on two FP32 lanes at once (Blackwell's paired FP32 pipe:
// add/fma .f32x2, round-to-nearest like the scalar FADD/FFMA, so results are identical).
template <bool PACKED>
__device__ __forceinline__ void add2(float& a0, float& a1, float x0, float x1) {
    if (PACKED) {
        uint64_t a, x;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
        asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
        asm("add.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(x));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(a));
    } else {
        a0 += x0;
        a1 += x1;
    }
}
template <bool PACKED>
__device__ __forceinline__ void fma2(float& a0, float& a1, float w, float x0, float x1) {
    if (PACKED) {
        uint64_t a, x, ww;
        asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(a0), "f"(a1));
        asm("mov.b64 %0, {%1, %2};" : "=l"(x) : "f"(x0), "f"(x1));
        asm("mov.b64 %0, {%1, %1};" : "=l"(ww) : "f"(w));
        asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(a) : "l"(ww), "l"(x));
        asm("mov.b64 {%0, %1}, %2;" : "=f"(a0), "=f"(a1) : "l"(a));
    } else {
        a0 = fmaf(w, x0, a0);
        a1 = fmaf(w, x1, a1);
    }
}

// a += one BF16 half of w (low or high), FP32 result: the mixed-precision add.f32.bf16 converts
// the BF16 value exactly and rounds once, so it equals converting then adding.
__device__ __forceinline__ float add_lo(float a, uint32_t w) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n add.rn.f32.bf16 %0, l, %2;}" : "=f"(r) : "r"(w), "f"(a));
    return r;
}
__device__ __forceinline__ float add_hi(float a, uint32_t w) {
    float r;
    asm("{.reg .b16 l, h;\n mov.b32 {l, h}, %1;\n add.rn.f32.bf16 %0, h, %2;}" : "=f"(r) : "r"(w), "f"(a));
    return r;
}

// Element traits: FP32 has one element per 32-bit word, BF16 two.
template <typename ST> struct EL;
template <> struct EL<float> {
    static constexpr int PER_WORD = 1;
    __device__ static __forceinline__ void unpack(uint32_t w, float* f) { f[0] = __uint_as_float(w); }
    __device__ static __forceinline__ uint32_t pack(const float* f) { return __float_as_uint(f[0]); }
};
template <> struct EL<__nv_bfloat16> {
    static constexpr int PER_WORD = 2;
    __device__ static __forceinline__ void unpack(uint32_t w, float* f) {
        f[0] = __uint_as_float(w << 16);
        f[1] = __uint_as_float(w & 0xffff0000u);
    }
    __device__ static __forceinline__ uint32_t pack(const float* f) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[0], f[1]);
        return *reinterpret_cast<uint32_t*>(&h);
    }
};

// CHECK: verify every column index against n (a CSR that does not come from this library's
// own build); otherwise the index is trusted.
// Gathered vectors in flight per lane and batch.  Rows of 8-byte gathers over a whole warp
// (BF16 d = 128) run at full occupancy (latency-bound: more warps beat deeper batches): the
// full-row unit-weight variant takes 8 and still fits the 32 registers of 8 CTAs/SM without
// spills (2.8B-entry graph, same box: 62.38 ms against 62.87 with 4 and 64.2 with 6); the
// others take 4 (with 8 they spill); every other shape keeps 8 at 4 CTAs/SM (BF16 d = 256 on
// the 2M-node graph: 3.3 ms against 5.1 ms with 4 in flight at 6 CTAs/SM).
template <typename ST, int VEC, int CPL, int G, bool HV = false, bool FR = false>
constexpr int inflight() {
    if (Tune<ST>::INFLIGHT > 0) return Tune<ST>::INFLIGHT;
    if (VEC == 8 && CPL == 1 && G == 32) return std::is_same<ST, __nv_bfloat16>::value && !HV && FR ? 8 : 4;
    // lane groups of 16-byte gathers: 8 in flight do not fit the 64 registers of 4 CTAs/SM
    if (VEC == 16 && G < 32) return 4;
    return 8;
}

// INF: vectors in flight per lane (0: inflight()).  FR: full rows -- the row holds exactly
// CPL x G vectors, so no lane's vector index needs a bound test and the row stride is a
// compile-time constant.
template <typename ST, int VEC, int CPL, int G, bool HV, bool CHECK = false, int INF = 0, bool FR = false>
struct Kern {
    using VT = typename VecT<VEC>::T;
    static constexpr int64_t FR_ROW = (int64_t)CPL * G * VEC;  // row bytes of full rows
    __device__ static __forceinline__ bool in_row(const Args& a, int i, int lg) {
        return FR || i * G + lg < a.chunks;
    }
    __device__ static __forceinline__ int64_t row_bytes(const Args& a) { return FR ? FR_ROW : a.row_bytes; }
    static constexpr int W = VEC / 4;                       // 32-bit words per vector
    static constexpr int EPV = W * EL<ST>::PER_WORD;        // elements per vector
    static constexpr int P = 32 / G;                        // lane groups per warp
    static constexpr int IN = INF > 0 ? INF : inflight<ST, VEC, CPL, G, HV, FR>();
    static constexpr int U = CPL >= IN ? 1 : IN / CPL;  // entries per batch

    // Two-level sum: `v` collects at most one 32-entry window, then is added into `t`.  Every
    // serial FP32 chain stays short (window + windows-per-row) even for a row of thousands of
    // nearly equal neighbour rows, where one long chain would build a systematic error.
    struct Acc {
        float v[CPL][EPV];
        float t[CPL][EPV];
        __device__ __forceinline__ void zero() {
#pragma unroll
            for (int i = 0; i < CPL; ++i)
#pragma unroll
                for (int e = 0; e < EPV; ++e) v[i][e] = t[i][e] = 0.f;
        }
        __device__ __forceinline__ void flush() {
#pragma unroll
            for (int i = 0; i < CPL; ++i)
#pragma unroll
                for (int e = 0; e < EPV; e += 2) {
                    add2<Tune<ST>::PACKED>(t[i][e], t[i][e + 1], v[i][e], v[i][e + 1]);
                    v[i][e] = v[i][e + 1] = 0.f;
                }
        }
    };

    __device__ static __forceinline__ void add_vec(Acc& acc, int i, const VT& x, float w) {
        if (!HV && std::is_same<ST, __nv_bfloat16>::value) {  // no unpacking: mixed adds
#pragma unroll
            for (int k = 0; k < W; ++k) {
                acc.v[i][2 * k] = add_lo(acc.v[i][2 * k], word(x, k));
                acc.v[i][2 * k + 1] = add_hi(acc.v[i][2 * k + 1], word(x, k));
            }
            return;
        }
        float f[EPV];
#pragma unroll
        for (int k = 0; k < W; ++k) EL<ST>::unpack(word(x, k), f + k * EL<ST>::PER_WORD);
#pragma unroll
        for (int e = 0; e < EPV; e += 2) {
            if (HV) fma2<Tune<ST>::PACKED>(acc.v[i][e], acc.v[i][e + 1], w, f[e], f[e + 1]);
            else add2<Tune<ST>::PACKED>(acc.v[i][e], acc.v[i][e + 1], f[e], f[e + 1]);
        }
    }

    __device__ static __forceinline__ VT zero_vec() {
        VT z;
#pragma unroll
        for (int k = 0; k < W; ++k) set_word(z, k, 0u);
        return z;
    }

    // Entries j = j0 + u*P + g (u < U) of a window of column indices held one per lane
    // (`mc`, `mw`), restricted to j < jh; all 32 lanes execute the shuffles.  FULLB: every
    // entry of the batch is valid, so no entry needs a validity test.  Invalid entries load
    // nothing and add a zero vector (this form also keeps register use lowest).  `cp` is the
    // L2 policy of the whole segment.
    template <bool FULLB>
    __device__ static __forceinline__ void gather_batch(const Args& a, Acc& acc, int mc, float mw,
                                                        int j0, int jh, int g, int lg, uint64_t cp) {
        VT x[U][CPL];
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u * P + g;
            const int c = __shfl_sync(FULL, mc, j);  // (the source lane is taken mod 32)
            const float wu = HV ? __shfl_sync(FULL, mw, j) : 1.f;
            bool ok = FULLB || j < jh;
            if (CHECK && ok && (unsigned)c >= (unsigned)a.n) {  // corrupt index: flag, skip
                atomicOr(a.err, 1);
                ok = false;
            }
            w[u] = ok ? wu : 0.f;
            const VT* rp = reinterpret_cast<const VT*>(a.Tin + (int64_t)c * row_bytes(a)) + lg;
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                if (Tune<ST>::POLICY)
                    x[u][i] = (ok && in_row(a, i, lg)) ? ld_gather(rp + i * G, cp) : zero_vec();
                else
                    x[u][i] = (ok && in_row(a, i, lg)) ? ld_gather(rp + i * G) : zero_vec();
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < CPL; ++i) add_vec(acc, i, x[u][i], w[u]);
    }

    // Same for one lane group working alone (mode 2): window of G entries, entries j0+u.
    template <bool FULLB>
    __device__ static __forceinline__ void gather_batch_group(const Args& a, Acc& acc, int mc, float mw,
                                                              int j0, int jh, int lg, unsigned gmask,
                                                              uint64_t cp) {
        VT x[U][CPL];
        float w[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = j0 + u;
            const int c = __shfl_sync(gmask, mc, j, G);  // (the source lane is taken mod G)
            const float wu = HV ? __shfl_sync(gmask, mw, j, G) : 1.f;
            bool ok = FULLB || j < jh;
            if (CHECK && ok && (unsigned)c >= (unsigned)a.n) {
                atomicOr(a.err, 1);
                ok = false;
            }
            w[u] = ok ? wu : 0.f;
            const VT* rp = reinterpret_cast<const VT*>(a.Tin + (int64_t)c * row_bytes(a)) + lg;
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                if (Tune<ST>::POLICY)
                    x[u][i] = (ok && in_row(a, i, lg)) ? ld_gather(rp + i * G, cp) : zero_vec();
                else
                    x[u][i] = (ok && in_row(a, i, lg)) ? ld_gather(rp + i * G) : zero_vec();
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
#pragma unroll
            for (int i = 0; i < CPL; ++i) add_vec(acc, i, x[u][i], w[u]);
    }

    // Entries [jl, jh) of the current window under one policy.
    __device__ static __forceinline__ void gather_window(const Args& a, Acc& acc, int mc, float mw, int jl,
                                                         int jh, int g, int lg, uint64_t cp) {
        int j0 = jl;
        if (Tune<ST>::FULLB) {
#pragma unroll 1
            for (; j0 + P * U <= jh; j0 += P * U) gather_batch<true>(a, acc, mc, mw, j0, jh, g, lg, cp);
            if (j0 < jh) gather_batch<false>(a, acc, mc, mw, j0, jh, g, lg, cp);
        } else {
#pragma unroll 1
            for (; j0 < jh; j0 += P * U) gather_batch<false>(a, acc, mc, mw, j0, jh, g, lg, cp);
        }
    }

    // Own previous row (a row without entries keeps it, renormalised).
    __device__ static __forceinline__ void load_own(const Args& a, Acc& acc, int64_t r, int lg) {
        const VT* rp = reinterpret_cast<const VT*>(a.Tin + r * row_bytes(a));
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int q = i * G + lg;
            if (in_row(a, i, lg)) {
                VT x = ld_gather(rp + q);
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    float f[EL<ST>::PER_WORD];
                    EL<ST>::unpack(word(x, k), f);
#pragma unroll
                    for (int h = 0; h < EL<ST>::PER_WORD; ++h) acc.t[i][k * EL<ST>::PER_WORD + h] = f[h];
                }
            }
        }
    }

    // Sum the P groups' partial sums (fixed butterfly: every group ends with the same bits).
    __device__ static __forceinline__ void reduce_groups(Acc& acc) {
#pragma unroll
        for (int off = G; off < 32; off <<= 1)
#pragma unroll
            for (int i = 0; i < CPL; ++i)
#pragma unroll
                for (int e = 0; e < EPV; ++e) acc.t[i][e] += __shfl_xor_sync(FULL, acc.t[i][e], off);
    }

    // L2-normalise within a lane group and store the row (group 0 stores in mode 1).
    __device__ static __forceinline__ void finish_row(const Args& a, Acc& acc, int64_t r, int lg,
                                                      bool store, unsigned gmask) {
        float ss = 0.f;
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            if (in_row(a, i, lg)) {
#pragma unroll
                for (int e = 0; e < EPV; ++e) ss = fmaf(acc.t[i][e], acc.t[i][e], ss);
            }
        }
#pragma unroll
        for (int off = 1; off < G; off <<= 1) ss += __shfl_xor_sync(gmask, ss, off);
        const float inv = ss > 0.f ? 1.0f / sqrtf(ss) : 0.f;
        if (!store) return;
        VT* op = reinterpret_cast<VT*>(a.Tout + r * row_bytes(a));
#pragma unroll
        for (int i = 0; i < CPL; ++i) {
            const int q = i * G + lg;
            if (in_row(a, i, lg)) {
                VT x;
#pragma unroll
                for (int k = 0; k < W; ++k) {
                    float f[EL<ST>::PER_WORD];
#pragma unroll
                    for (int h = 0; h < EL<ST>::PER_WORD; ++h) f[h] = acc.t[i][k * EL<ST>::PER_WORD + h] * inv;
                    set_word(x, k, EL<ST>::pack(f));
                }
                st_stream(op + q, x);
            }
        }
    }

    // Accumulate entries [k0, k1) with the whole warp (groups interleave entries).
    __device__ static __forceinline__ void range_coop(const Args& a, Acc& acc, int64_t k0, int64_t k1,
                                                      int64_t hot_end, int lane, int g, int lg) {
        const bool part = a.hot_cnt != nullptr;
        int64_t cb = -64;
        int mc = 0;
        float mw = 0.f;
        for (int64_t k = k0; k < k1;) {
            if (k >= cb + 32) {
                cb = k;
                const int m = (int)min((int64_t)32, k1 - cb);
                mc = 0;
                mw = 0.f;
                if (lane < m) {
                    mc = __ldcs(a.col + cb + lane);
                    if (HV) mw = __ldcs(a.val + cb + lane);
                }
            }
            // a segment ends at the window's end, the range's end or the row's hot boundary
            const bool hot = k < hot_end;
            const int64_t stop = hot ? min(k1, hot_end) : k1;
            const int jh = (int)min((int64_t)32, stop - cb);
            gather_window(a, acc, mc, mw, (int)(k - cb), jh, g, lg, seg_policy(part, hot));
            acc.flush();
            k = cb + jh;
        }
    }

    // Mode 1: the warp walks rows [rb, re) one at a time; rowptr and column windows are
    // loaded 32 at a time and reused across consecutive rows.  SKIP: leave out rows longer
    // than a.skip_len (a caller that runs those rows as split chunks).
    template <bool SKIP = false>
    __device__ static void rows_coop(const Args& a, int64_t rb, int64_t re, int lane, int g, int lg) {
        int64_t wr = rb, lo = 0, hi = 0;
        if (wr + lane < re) {
            lo = a.rowptr[wr + lane];
            hi = a.rowptr[wr + lane + 1];
        }
        int64_t cb = -64;  // column window [cb, cb + 32)
        int mc = 0;
        float mw = 0.f;
        for (int64_t r = rb; r < re; ++r) {
            if (r - wr == 32) {
                wr = r;
                lo = hi = 0;
                if (wr + lane < re) {
                    lo = a.rowptr[wr + lane];
                    hi = a.rowptr[wr + lane + 1];
                }
            }
            const int64_t beg = __shfl_sync(FULL, lo, (int)(r - wr));
            const int64_t end = __shfl_sync(FULL, hi, (int)(r - wr));
            // hot count: one broadcast load per row (a lane register holding 32 rows' counts,
            // like rowptr, costs the register that keeps the FP32 kernel from spilling)
            const int64_t hot_end = beg + (a.hot_cnt ? a.hot_cnt[r] : 0);
            if (SKIP && end - beg > a.skip_len) continue;
            Acc acc;
            acc.zero();
            if (beg == end) {
                if (g == 0) load_own(a, acc, r, lg);
            }
            for (int64_t k = beg; k < end;) {
                if (k < cb || k >= cb + 32) {
                    cb = k;
                    mc = 0;
                    mw = 0.f;
                    if (cb + lane < a.nnz) {
                        mc = __ldcs(a.col + cb + lane);
                        if (HV) mw = __ldcs(a.val + cb + lane);
                    }
                }
                // a segment ends at the window's end, the row's end or its hot boundary
                const bool hot = k < hot_end;
                const int64_t stop = hot ? min(end, hot_end) : end;
                const int jh = (int)min((int64_t)32, stop - cb);
                gather_window(a, acc, mc, mw, (int)(k - cb), jh, g, lg, seg_policy(a.hot_cnt != nullptr, hot));
                acc.flush();
                k = cb + jh;
            }
            reduce_groups(acc);
            finish_row(a, acc, r, lg, g == 0, FULL);
        }
    }

    // Mode 2: lane group g owns rows rb + g, rb + g + P, ...
    __device__ static void rows_group(const Args& a, int64_t rb, int64_t re, int g, int lg) {
        const unsigned gmask = (G == 32) ? FULL : (((1u << G) - 1u) << (g * G));
        for (int64_t r = rb + g; r < re; r += P) {
            const int64_t beg = a.rowptr[r], end = a.rowptr[r + 1];
            const int64_t hot_end = beg + (a.hot_cnt ? a.hot_cnt[r] : 0);
            Acc acc;
            acc.zero();
            if (beg == end) load_own(a, acc, r, lg);
            for (int64_t cb = beg; cb < end; cb += G) {
                const int jh = (int)min((int64_t)G, end - cb);
                int mc = 0;
                float mw = 0.f;
                if (lg < jh) {
                    mc = __ldcs(a.col + cb + lg);
                    if (HV) mw = __ldcs(a.val + cb + lg);
                }
                const int hj = (int)max((int64_t)0, min((int64_t)jh, hot_end - cb));
#pragma unroll 1
                for (int part = 0; part < 2; ++part) {
                    const int pb = part == 0 ? 0 : hj, pe = part == 0 ? hj : jh;
                    const uint64_t cp = seg_policy(a.hot_cnt != nullptr, part == 0);
                    int j0 = pb;
#pragma unroll 1
                    for (; j0 + U <= pe; j0 += U)
                        gather_batch_group<true>(a, acc, mc, mw, j0, pe, lg, gmask, cp);
                    if (j0 < pe) gather_batch_group<false>(a, acc, mc, mw, j0, pe, lg, gmask, cp);
                }
                acc.flush();
            }
            finish_row(a, acc, r, lg, true, gmask);
        }
    }

    // One chunk of a split row; the last chunk to finish combines all partial slots.
    __device__ static void split_chunk(const Args& a, const Task& t, int lane, int g, int lg) {
        const int64_t r = t.a;
        const int64_t beg = a.rowptr[r], end = a.rowptr[r + 1];
        const int64_t k0 = beg + (int64_t)t.c * a.split_len;
        const int64_t k1 = min(end, k0 + a.split_len);
        Acc acc;
        acc.zero();
        range_coop(a, acc, k0, k1, beg + (a.hot_cnt ? a.hot_cnt[r] : 0), lane, g, lg);
        split_store_combine(a, t, acc, lane, g, lg);
    }

    // A split chunk's partial sum (in acc.t) goes to its slot; the warp that finishes the
    // row's last chunk adds all slots in a fixed order, normalises and writes the row.
    __device__ static void split_store_combine(const Args& a, const Task& t, Acc& acc, int lane, int g, int lg) {
        const int64_t r = t.a;
        reduce_groups(acc);
        const int64_t base = a.split_base[t.b];
        float* slot = a.partials + (base + t.c) * (int64_t)a.d;
        if (g == 0) {
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int q = i * G + lg;
                if (in_row(a, i, lg)) {
#pragma unroll
                    for (int e = 0; e < EPV; ++e) __stcg(slot + q * EPV + e, acc.t[i][e]);
                }
            }
        }
        __threadfence();
        __syncwarp();
        int prev = 0;
        if (lane == 0) prev = atomicAdd(a.split_count + t.b, 1);
        prev = __shfl_sync(FULL, prev, 0);
        if (prev != t.k - 1) return;
        // Last arrival: add slots 0..k-1 (group g takes c = g, g+P, ...), then the butterfly.
        __threadfence();
        acc.zero();
        for (int c = g, m = 0; c < t.k; c += P, ++m) {
            const float* s = a.partials + (base + c) * (int64_t)a.d;
#pragma unroll
            for (int i = 0; i < CPL; ++i) {
                const int q = i * G + lg;
                if (in_row(a, i, lg)) {
#pragma unroll
                    for (int e = 0; e < EPV; ++e) acc.v[i][e] += __ldcg(s + q * EPV + e);
                }
            }
            if ((m & 31) == 31) acc.flush();
        }
        acc.flush();
        reduce_groups(acc);
        finish_row(a, acc, r, lg, g == 0, FULL);
        if (lane == 0) a.split_count[t.b] = 0;  // ready for the next launch
    }
};

// CTAs per SM the kernel is compiled for (its register budget is 65536 / (256 x that)).
// Rows of more than two vectors per lane leave it to the compiler.  BF16 8-byte whole-warp
// rows: as many as fit without spilling at 4 vectors in flight (8, or 6 with per-entry
// values); every other shape: Tune's count (FP32) or 4.
template <typename ST, int VEC, int CPL, int G, bool HV>
constexpr int min_blocks() {
    if (CPL > 2) return 1;
    if (!std::is_same<ST, __nv_bfloat16>::value) return Tune<ST>::MINB;
    if (Tune<ST>::MINB > 0) return Tune<ST>::MINB;
    if (VEC == 8 && CPL == 1 && G == 32) return HV ? 6 : 8;  // no spills at 4 in flight
    return 4;
}

template <typename ST, int VEC, int CPL, int G, int MODE, bool HV, bool FR = false>
__global__ void __launch_bounds__(256, (min_blocks<ST, VEC, CPL, G, HV>()))
k_propagate(Args a) {
    using K = Kern<ST, VEC, CPL, G, HV, false, 0, FR>;
    const int lane = threadIdx.x & 31;
    const int g = lane / G, lg = lane % G;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(a.counter, 1ull);
        t = __shfl_sync(FULL, t, 0);
        if (t >= (unsigned long long)a.ntasks) break;
        const Task task = a.tasks[t];
        if (task.c >= 0) {
            K::split_chunk(a, task, lane, g, lg);
        } else if (MODE == 1 || G == 32) {
            K::rows_coop(a, task.a, task.b, lane, g, lg);
        } else {
            K::rows_group(a, task.a, task.b, g, lg);
        }
        __syncwarp();
    }
}

// Host-side launcher for one storage type, vector width and value mode.
template <typename ST, int VEC, bool HV>
struct Launch {
    template <int CPL, int G, int MODE, bool FR = false>
    static cudaError_t go(const Args& a, int blocks_per_sm, int num_sms, cudaStream_t s, int* grid_out) {
        auto kern = k_propagate<ST, VEC, CPL, G, MODE, HV, FR>;
        int bps = blocks_per_sm;
        if (bps <= 0) {
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0);
            if (e != cudaSuccess) return e;
            if (bps < 1) bps = 1;
        }
        int grid = bps * num_sms;
        if (grid_out) *grid_out = grid;
        kern<<<grid, 256, 0, s>>>(a);
        return cudaGetLastError();
    }

    static cudaError_t run(const Shape& sh, const Args& a, int bps, int sms, cudaStream_t s, int* grid) {
        const int m = sh.mode;
        if (sh.cpl == 1) {
            switch (sh.G) {
                case 1:  return m == 2 ? go<1, 1, 2>(a, bps, sms, s, grid) : go<1, 1, 1>(a, bps, sms, s, grid);
                case 2:  return m == 2 ? go<1, 2, 2>(a, bps, sms, s, grid) : go<1, 2, 1>(a, bps, sms, s, grid);
                case 4:  return m == 2 ? go<1, 4, 2>(a, bps, sms, s, grid) : go<1, 4, 1>(a, bps, sms, s, grid);
                case 8:  return m == 2 ? go<1, 8, 2>(a, bps, sms, s, grid) : go<1, 8, 1>(a, bps, sms, s, grid);
                case 16: return m == 2 ? go<1, 16, 2>(a, bps, sms, s, grid) : go<1, 16, 1>(a, bps, sms, s, grid);
                case 32: return sh.chunks == 32 ? go<1, 32, 1, true>(a, bps, sms, s, grid)
                                                : go<1, 32, 1>(a, bps, sms, s, grid);
                default: return cudaErrorInvalidValue;
            }
        }
        // (the full-row variant only for one vector per lane: with two, the 2M-node d = 256
        // FP32 graph took 5.24 ms per iteration against 4.29 ms without it)
        if (sh.G != 32) return cudaErrorInvalidValue;
        switch (sh.cpl) {
            case 2: return go<2, 32, 1>(a, bps, sms, s, grid);
            case 4: return go<4, 32, 1>(a, bps, sms, s, grid);
            case 8: return go<8, 32, 1>(a, bps, sms, s, grid);
            default: return cudaErrorInvalidValue;
        }
    }
};

// Entry points defined in the per-type translation units.
cudaError_t launch_f32_v16(const Shape&, const Args&, bool hv, int bps, int sms, cudaStream_t, int*);
cudaError_t launch_f32_v8(const Shape&, const Args&, bool hv, int bps, int sms, cudaStream_t, int*);
cudaError_t launch_bf16_v16(const Shape&, const Args&, bool hv, int bps, int sms, cudaStream_t, int*);
cudaError_t launch_bf16_v8(const Shape&, const Args&, bool hv, int bps, int sms, cudaStream_t, int*);

}  // namespace prop
}  // namespace cleora
