// MMSE detection kernels of the 16-layer class (kernel in mmse_impl.cuh).
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t mmse_launch_class16(const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                                const float2 *beam, float2 *xhat, uint8_t *bits, uint32_t *status, cudaStream_t st) {
    return mmse_detail::launch_nd<16>(a, total_sc, H, beam, xhat, bits, status, st);
}

}  // namespace pusch
