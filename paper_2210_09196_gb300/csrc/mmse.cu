// MMSE MIMO detection (Eq. 2): argument set-up and dispatch on the layer class; the kernel and its
// design notes are in mmse_impl.cuh.
#include "mmse_impl.cuh"

namespace pusch {
namespace {

using mmse_detail::MmseArgs;

template <bool FUSED>
cudaError_t launch_any(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, const float2 *pilots,
                       float2 *x_hat, uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2) {
    MmseArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.n_sym = g.n_sym;
    a.n_data = g.n_data;
    a.qam_bits = g.qam_bits;
    a.comb = g.comb;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    a.load = g.noise_var + g.loading;
    a.loading = g.loading;
    a.sigma2 = sigma2;
    a.kmax = ls_pilots_per_layer(g);
    for (int d = 0; d < 16; ++d) a.data_sym[d] = g.data_sym[d];
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    if (g.n_data > 14) return cudaErrorInvalidValue;
    const long long total_sc = (long long)n_slots * g.n_sc;
    if (total_sc == 0) return cudaSuccess;
    const int nl = g.n_layers;
    if (nl <= 8) return mmse_launch_class(nl <= 2 ? 2 : (nl <= 4 ? 4 : 8), FUSED, a, total_sc, H, beam, pilots, x_hat,
                                          bits, status, st);
    if (nl <= 16) return mmse_launch_class16(FUSED, a, total_sc, H, beam, pilots, x_hat, bits, status, st);
    return mmse_launch_class32(FUSED, a, total_sc, H, beam, pilots, x_hat, bits, status, st);
}

}  // namespace

cudaError_t launch_mmse(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, float2 *x_hat,
                        uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2) {
    return launch_any<false>(g, n_slots, H, beam, nullptr, x_hat, bits, status, st, sigma2);
}

cudaError_t launch_mmse_fused(const Geometry &g, int n_slots, const float2 *beam, const float2 *ls,
                              float2 *x_hat, uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2) {
    return launch_any<true>(g, n_slots, nullptr, beam, ls, x_hat, bits, status, st, sigma2);
}

}  // namespace pusch
