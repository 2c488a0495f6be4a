// MMSE detection kernel of the 32-layer class reading a stored estimate (kernel in mmse_impl.cuh); the
// fused variant is in mmse_nl32f.cu.
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t mmse_launch_class32(bool fused, const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                                const float2 *beam, const float2 *pilots, float2 *xhat, uint8_t *bits,
                                uint32_t *status, cudaStream_t st) {
    if (fused) return mmse_launch_class32_fused(a, total_sc, beam, pilots, xhat, bits, status, st);
    return mmse_detail::launch_nd<32, false>(a, total_sc, H, beam, pilots, xhat, bits, status, st);
}

}  // namespace pusch
