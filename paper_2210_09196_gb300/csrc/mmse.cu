// MMSE MIMO detection (Eq. 2): argument set-up and dispatch on the layer class; the kernel and its
// design notes are in mmse_impl.cuh.
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t launch_mmse(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, float2 *x_hat,
                        uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2, bool time_groups) {
    mmse_detail::MmseArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.n_sym = g.n_sym;
    a.n_data = g.n_data;
    a.qam_bits = g.qam_bits;
    a.load = g.noise_var + g.loading;
    a.loading = g.loading;
    a.sigma2 = sigma2;
    a.n_groups = time_groups ? g.n_groups : 1;
    a.group_k = time_groups ? g.chol_every : g.n_data;
    a.h_group_stride = (long long)n_slots * g.n_sc * g.n_layers * g.n_beams;
    a.dmrs_lo = g.dmrs0 < g.dmrs1 ? g.dmrs0 : g.dmrs1;
    a.dmrs_hi = g.dmrs0 < g.dmrs1 ? g.dmrs1 : g.dmrs0;
    if (g.n_data > 14) return cudaErrorInvalidValue;
    const long long total_sc = (long long)n_slots * g.n_sc;
    if (total_sc == 0) return cudaSuccess;
    const int nl = g.n_layers;
    if (nl <= 8) return mmse_launch_class(nl <= 2 ? 2 : (nl <= 4 ? 4 : 8), a, total_sc, H, beam, x_hat, bits, status, st);
    if (nl <= 16) return mmse_launch_class16(a, total_sc, H, beam, x_hat, bits, status, st);
    return mmse_launch_class32(a, total_sc, H, beam, x_hat, bits, status, st);
}

}  // namespace pusch
