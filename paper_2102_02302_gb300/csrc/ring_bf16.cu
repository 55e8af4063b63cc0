// Shared-memory ring propagate kernels instantiated for storage type __nv_bfloat16.
#include "ring_kernels.cuh"

namespace cleora {
namespace ring {

cudaError_t launch_bf16_v8(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s,
                            int* grid) {
    return launch_any<__nv_bfloat16, 8>(a, tmap, hv, stages, sms, s, grid);
}

cudaError_t launch_bf16_v16(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s,
                            int* grid) {
    return launch_any<__nv_bfloat16, 16>(a, tmap, hv, stages, sms, s, grid);
}

}  // namespace ring
}  // namespace cleora
