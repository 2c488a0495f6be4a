// MMSE detection kernels of the layer classes 2, 4 and 8 (kernel in mmse_impl.cuh).
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t mmse_launch_class(int nl_class, const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                              const float2 *beam, float2 *xhat, uint8_t *bits, uint32_t *status, cudaStream_t st) {
    using namespace mmse_detail;
    if (nl_class == 2) return launch_nd<2>(a, total_sc, H, beam, xhat, bits, status, st);
    if (nl_class == 4) return launch_nd<4>(a, total_sc, H, beam, xhat, bits, status, st);
    return launch_nd<8>(a, total_sc, H, beam, xhat, bits, status, st);
}

}  // namespace pusch
