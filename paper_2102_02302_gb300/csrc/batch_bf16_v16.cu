// Batched propagate kernels instantiated for storage type __nv_bfloat16 and 16-byte gathers.
#include "batch_kernels.cuh"

namespace cleora {
namespace batch {

cudaError_t launch_batch_bf16_v16(int cpl, int G, int mode, const BatchArgs& ba, int sms, cudaStream_t s, int* grid) {
    return BatchLaunch<__nv_bfloat16, 16>::run(cpl, G, mode, ba, sms, s, grid);
}

}  // namespace batch
}  // namespace cleora
