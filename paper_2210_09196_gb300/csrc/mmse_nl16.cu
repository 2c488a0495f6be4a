// MMSE detection kernels of the 16-layer class (kernel in mmse_impl.cuh).
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t mmse_launch_class16(bool fused, const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                                const float2 *beam, const float2 *pilots, float2 *xhat, uint8_t *bits,
                                uint32_t *status, cudaStream_t st) {
    using namespace mmse_detail;
    return fused ? launch_nd<16, true>(a, total_sc, H, beam, pilots, xhat, bits, status, st)
                 : launch_nd<16, false>(a, total_sc, H, beam, pilots, xhat, bits, status, st);
}

}  // namespace pusch
