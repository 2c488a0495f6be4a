// OFDM demodulation (Section II; Table I "OFDM dem."): dispatch on the cell's arithmetic form: the tensor-core
// FFT (fft_tc.cu) for the mixed form's 4096-point FP16 rows, the FFT kernels of fft_impl.cuh otherwise.
#include "fft_impl.cuh"

namespace pusch {

cudaError_t launch_fft(const Geometry &g, int n_slots, const void *time_in, void *freq_out, const float2 *twiddle,
                       uint32_t *err, cudaStream_t st) {
    if (reinterpret_cast<uintptr_t>(time_in) % 16 != 0) return cudaErrorMisalignedAddress;
    const long long rows = (long long)n_slots * g.n_sym * g.n_rx;
    if (rows == 0) return cudaSuccess;
    if (rows > 0x7fffffffLL) return cudaErrorInvalidValue;   // row indices are 32-bit in the epilogues
    if (fft_tc_supported(g)) return launch_fft_tc(g, rows, time_in, freq_out, twiddle, err, st);
    if (g.form == PUSCH_FORM_MIXED) return launch_fft_f16(g, rows, time_in, freq_out, twiddle, nullptr, err, st);
    if (g.form == PUSCH_FORM_FP8)
        return launch_fft_e4m3(g, rows, time_in, freq_out, twiddle, fp8_scales(g, n_slots, freq_out), err, st);
    return launch_fft_c64(g, rows, time_in, freq_out, twiddle, nullptr, err, st);
}

}  // namespace pusch
