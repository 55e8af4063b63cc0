// Shared-memory ring propagate kernels instantiated for storage type float.
#include "ring_kernels.cuh"

namespace cleora {
namespace ring {

cudaError_t launch_f32_v8(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s,
                            int* grid) {
    return launch_any<float, 8>(a, tmap, hv, stages, sms, s, grid);
}

cudaError_t launch_f32_v16(const prop::Args& a, const CUtensorMap* tmap, bool hv, int stages, int sms, cudaStream_t s,
                            int* grid) {
    return launch_any<float, 16>(a, tmap, hv, stages, sms, s, grid);
}

}  // namespace ring
}  // namespace cleora
