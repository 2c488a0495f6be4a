// MMSE detection kernel of the 32-layer class with the estimate interpolated from the LS pilot table
// (kernel in mmse_impl.cuh).
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t mmse_launch_class32_fused(const mmse_detail::MmseArgs &a, long long total_sc, const float2 *beam,
                                      const float2 *pilots, float2 *xhat, uint8_t *bits, uint32_t *status,
                                      cudaStream_t st) {
    return mmse_detail::launch_nd<32, true>(a, total_sc, nullptr, beam, pilots, xhat, bits, status, st);
}

}  // namespace pusch
