// Propagate kernels instantiated for storage type __nv_bfloat16 and 8-byte gathers.
#include "propagate_kernels.cuh"

namespace cleora {
namespace prop {

cudaError_t launch_bf16_v8(const Shape& sh, const Args& a, bool hv, int bps, int sms, cudaStream_t s,
                      int* grid) {
    return hv ? Launch<__nv_bfloat16, 8, true>::run(sh, a, bps, sms, s, grid)
              : Launch<__nv_bfloat16, 8, false>::run(sh, a, bps, sms, s, grid);
}

}  // namespace prop
}  // namespace cleora
