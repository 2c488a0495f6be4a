// MMSE MIMO detection (Eq. 2): argument set-up and dispatch on the layer class; the kernel and its
// design notes are in mmse_impl.cuh.
#include "mmse_impl.cuh"

namespace pusch {

cudaError_t launch_mmse(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, float2 *x_hat,
                        uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2, bool time_groups,
                        const float2 *ls) {
    if (ls && (time_groups || !mmse_interp_supported(g, beam, ls))) return cudaErrorNotSupported;
    mmse_detail::MmseArgs a;
    a.ls = ls;
    a.kmax = ls ? ls_pilots_per_layer(g) : 0;
    a.comb = g.comb;
    for (int l = 0; l < 32; ++l) a.port[l] = l < g.n_layers ? g.port[l] : 0;
    a.warps = g.det_warps;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.n_sym = g.n_sym;
    a.n_data = g.n_data;
    a.qam_bits = g.qam_bits;
    a.load = g.noise_var + g.loading;
    a.loading = g.loading;
    a.sigma2 = sigma2;
    a.dmrs_lo = g.dmrs0 < g.dmrs1 ? g.dmrs0 : g.dmrs1;
    a.dmrs_hi = g.dmrs0 < g.dmrs1 ? g.dmrs1 : g.dmrs0;
    if (g.n_data > 14) return cudaErrorInvalidValue;
    const long long total_sc = (long long)n_slots * g.n_sc;
    if (total_sc == 0) return cudaSuccess;
    const int nl = g.n_layers;
    // one launch per detection group: group q detects data symbols [q K, q K + K) with its own estimate
    // (H + q * stride); one group of all data symbols when the estimate does not vary in time
    const int groups = time_groups ? g.n_groups : 1;
    const int K = time_groups ? g.chol_every : g.n_data;
    const long long stride = (long long)n_slots * g.n_sc * g.n_layers * g.n_beams;
    for (int q = 0; q < groups; ++q) {
        a.d_first = q * K;
        a.n_det = g.n_data - q * K < K ? g.n_data - q * K : K;
        const float2 *Hq = H + q * stride;
        cudaError_t e;
        if (nl <= 8)
            e = mmse_launch_class(nl <= 2 ? 2 : (nl <= 4 ? 4 : 8), a, total_sc, Hq, beam, x_hat, bits, status, st);
        else if (nl <= 16)
            e = mmse_launch_class16(a, total_sc, Hq, beam, x_hat, bits, status, st);
        else
            e = mmse_launch_class32(a, total_sc, Hq, beam, x_hat, bits, status, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

bool mmse_interp_supported(const Geometry &g, const float2 *beam, const float2 *ls) {
    return g.n_layers > 8 && g.n_layers <= 32 && (g.n_beams == 32 || g.n_beams == 64) && g.chol_every == 0 &&
           reinterpret_cast<uintptr_t>(beam) % 16 == 0 && reinterpret_cast<uintptr_t>(ls) % 16 == 0;
}

int mmse_warp_choices_for(int n_layers, int n_beams, int *out) {
    using namespace mmse_detail;
    if (n_layers <= 2) return mmse_warp_choices<2>(n_beams, out);
    if (n_layers <= 4) return mmse_warp_choices<4>(n_beams, out);
    if (n_layers <= 8) return mmse_warp_choices<8>(n_beams, out);
    if (n_layers <= 16) return mmse_warp_choices<16>(n_beams, out);
    return mmse_warp_choices<32>(n_beams, out);
}

}  // namespace pusch
