// OFDM demodulation FFTs writing the FP16-plane (mixed form) output; the transform itself is in fft_impl.cuh.
#include "fft_impl.cuh"

namespace pusch {

cudaError_t launch_fft_f16(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                         float *scales, uint32_t *err, cudaStream_t st) {
    if (g.in_fp16) return fft_detail::launch_out<__half2, fft_detail::kOutF16>(g, rows, in, out, tw, scales, err, st);
    return fft_detail::launch_out<float2, fft_detail::kOutF16>(g, rows, in, out, tw, scales, err, st);
}

}  // namespace pusch
