// GPU implementation of synth.chung_lu_undirected_idx and synth.node_ids (input generation
// only; no arithmetic of the embedding method).  Same counter-based splitmix64 draws, same
// integer inverse-CDF thresholds, same dedup rounds as the numpy code, so both produce the
// same edge list bit for bit.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_select.cuh>

namespace {

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

uint64_t mix_host(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int64_t sample(const uint64_t* thr, int64_t n, uint64_t h) {
    const uint64_t r = h >> 11;  // first i with r < thr[i]
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (thr[mid] <= r) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void k_candidates(const uint64_t* thr, int64_t n, uint64_t key_src, uint64_t key_dst,
                             uint64_t c0, int64_t m, uint64_t* out) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t cnt = c0 + (uint64_t)t;
        const int64_t u = sample(thr, n, mix(key_src ^ cnt));
        const int64_t v = sample(thr, n, mix(key_dst ^ cnt));
        const uint64_t a = (uint64_t)(u < v ? u : v), b = (uint64_t)(u < v ? v : u);
        out[t] = (u == v) ? ~0ull : ((a << 32) | b);
    }
}

__global__ void k_count_valid(const uint64_t* keys, int64_t m, int64_t* out) {
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (keys[mid] != ~0ull) lo = mid + 1; else hi = mid;
    }
    *out = lo;
}

__global__ void k_to_ids(const uint64_t* keys, int64_t count, uint64_t idkey, uint64_t* src,
                         uint64_t* dst) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < count;
         t += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t k = keys[t];
        src[t] = mix((k >> 32) ^ idkey);
        dst[t] = mix((k & 0xffffffffull) ^ idkey);
    }
}

unsigned grid(int64_t items) {
    int64_t b = (items + 255) / 256;
    if (b > 152 * 64) b = 152 * 64;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

extern "C" {

// Sorted unique undirected edge keys (u << 32 | v, u < v).  *keys_out is a cudaMalloc'd
// device array of *count_out keys; free it with synth_free.  Returns a cudaError_t.
int synth_undirected_keys(const uint64_t* thr_host, int64_t n, int64_t E, uint64_t seed,
                          int max_rounds, uint64_t** keys_out, int64_t* count_out,
                          uint64_t* counter_end_out) {
    cudaError_t e = cudaSuccess;
    uint64_t* thr = nullptr;
    uint64_t* have = nullptr;
    int64_t nh = 0;
    int64_t* d_num = nullptr;
    const uint64_t kseed = mix_host(seed);
    const uint64_t key_src = mix_host(kseed ^ 1ull), key_dst = mix_host(kseed ^ 2ull);
    uint64_t c = 0;
#define SY(x) do { e = (x); if (e != cudaSuccess) goto done; } while (0)
    SY(cudaMalloc(&thr, n * sizeof(uint64_t)));
    SY(cudaMemcpy(thr, thr_host, n * sizeof(uint64_t), cudaMemcpyHostToDevice));
    SY(cudaMalloc(&d_num, 2 * sizeof(int64_t)));
    for (int round = 0; round < max_rounds; ++round) {
        const int64_t need = E - nh;
        if (need <= 0) break;
        const int64_t m = need + need / 8 + 1024;
        const int64_t tot = nh + m;
        uint64_t *a = nullptr, *b = nullptr;
        void* tmp = nullptr;
        size_t tb = 0, tu = 0;
        SY(cudaMalloc(&a, tot * sizeof(uint64_t)));
        SY(cudaMalloc(&b, tot * sizeof(uint64_t)));
        if (nh) SY(cudaMemcpy(a, have, nh * sizeof(uint64_t), cudaMemcpyDeviceToDevice));
        k_candidates<<<grid(m), 256>>>(thr, n, key_src, key_dst, c, m, a + nh);
        SY(cudaGetLastError());
        c += (uint64_t)m;
        {
            cub::DoubleBuffer<uint64_t> db(a, b);
            SY(cub::DeviceRadixSort::SortKeys(nullptr, tb, db, tot));
            SY(cub::DeviceSelect::Unique(nullptr, tu, db.Current(), db.Alternate(), d_num, tot));
            SY(cudaMalloc(&tmp, tb > tu ? tb : tu));
            SY(cub::DeviceRadixSort::SortKeys(tmp, tb, db, tot));
            uint64_t* sorted = db.Current();
            uint64_t* uniq = db.Alternate();
            SY(cub::DeviceSelect::Unique(tmp, tu, sorted, uniq, d_num, tot));
            int64_t nu = 0;
            SY(cudaMemcpy(&nu, d_num, sizeof(int64_t), cudaMemcpyDeviceToHost));
            k_count_valid<<<1, 1>>>(uniq, nu, d_num + 1);
            SY(cudaGetLastError());
            int64_t nv = 0;
            SY(cudaMemcpy(&nv, d_num + 1, sizeof(int64_t), cudaMemcpyDeviceToHost));
            cudaFree(tmp);
            cudaFree(have);
            cudaFree(sorted);
            SY(cudaMalloc(&have, (nv ? nv : 1) * sizeof(uint64_t)));
            SY(cudaMemcpy(have, uniq, nv * sizeof(uint64_t), cudaMemcpyDeviceToDevice));
            cudaFree(uniq);
            nh = nv;
        }
    }
    *keys_out = have;
    *count_out = nh;
    if (counter_end_out) *counter_end_out = c;
    have = nullptr;
done:
#undef SY
    cudaFree(thr);
    cudaFree(d_num);
    if (have) cudaFree(have);
    return (int)e;
}

// External ids of both endpoints: id(i) = mix(i ^ mix(seed ^ ID_KEY)).
int synth_keys_to_ids(const uint64_t* keys, int64_t count, uint64_t seed, uint64_t id_key,
                      uint64_t* src, uint64_t* dst) {
    const uint64_t idkey = mix_host(seed ^ id_key);
    k_to_ids<<<grid(count), 256>>>(keys, count, idkey, src, dst);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return (int)e;
}

void synth_free(void* p) { cudaFree(p); }

}  // extern "C"
