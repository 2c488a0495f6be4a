// pusch_slot_noalloc: the whole receive chain (the kernels of pusch_slot) for callers that cannot allocate
// device memory. Its intermediates (FFT output, beamformed grid, channel estimate), the FFT twiddle table
// and its status words live in one file-scope static device buffer of PUSCH_NOALLOC_SCRATCH_BYTES instead
// of a handle's workspace, so a call performs no cudaMalloc / cudaFree and needs no handle.
//
// The buffer is shared by every call in the process on a given device and keeps the last call's
// contents; everything a call reads from it is written earlier in the same call. Calls whose work
// overlaps on the GPU (two streams, or two host threads) race on it.
#include <stdio.h>

#include "internal.cuh"

// The static buffer: every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[PUSCH_NOALLOC_SCRATCH_BYTES];

namespace {

// Records the message returned by pusch_last_error() on this thread.
pusch_status na_fail(pusch_status st, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    if (e != cudaSuccess)
        snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof buf, "%s", msg);
    pusch::set_last_error(buf);
    return st;
}

// The FFT twiddle table (pusch::fft_twiddle_table): exp(-2 pi i q / n), then exp(-2 pi i q / (4 n)), q < n,
// computed in double precision and rounded once to float.
__global__ void noalloc_twiddle_kernel(float2 *tw, int n) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q < 2 * n) {
        double s, c;
        sincospi(-2.0 * (double)(q % n) / (double)(q < n ? n : 4 * n), &s, &c);
        tw[q] = make_float2((float)c, (float)s);
    }
}

__global__ void noalloc_status_kernel(uint32_t *status, uint32_t *kernel_err) {
    status[0] = 0u;
    status[1] = 0u;
    status[2] = 0xffffffffu;
    status[3] = 0u;
    kernel_err[0] = 0u;
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Device address of the static buffer in the current device's context, looked up on every call (not cached:
// after cudaDeviceReset, or in another context on the same device, the library's device code is loaded again
// and the buffer may sit at another address). Once the module is loaded the lookup is a host-side table read.
pusch_status scratch_for_current_device(unsigned char **out) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return na_fail(PUSCH_ERR_CUDA, "cudaGetSymbolAddress of the static buffer", e);
    *out = static_cast<unsigned char *>(p);
    return PUSCH_OK;
}

}  // namespace

extern "C" pusch_status pusch_slot_noalloc(const pusch_cell_cfg *cfg, int n_slots, const void *time_in,
                                           const void *W, const void *pilots, void *x_hat, uint8_t *bits,
                                           uint32_t *status, void *stream) {
    if (n_slots < 0) return na_fail(PUSCH_ERR_ARG, "pusch_slot_noalloc: n_slots < 0");
    size_t ws = 0;
    pusch_status st = pusch_workspace_size(cfg, n_slots > 0 ? n_slots : 1, &ws);  // validates cfg, no allocation
    if (st != PUSCH_OK) return st;  // message already set by pusch_workspace_size
    if (n_slots == 0) return PUSCH_OK;
    if (!time_in || !W || !pilots || !x_hat || !bits) return na_fail(PUSCH_ERR_ARG, "pusch_slot_noalloc: NULL buffer");

    if (cfg->chol_every != 0)
        return na_fail(PUSCH_ERR_UNSUPPORTED, "pusch_slot_noalloc: chol_every > 0 needs a handle (pusch_slot)");
    const pusch::Geometry g = pusch::make_geometry(*cfg);
    const size_t tw_b = up256((size_t)pusch::fft_twiddle_count(g.n_fft) * sizeof(float2));
    const size_t words_b = 256;  // status sink (16 B) + kernel error word (16 B)
    const size_t freq_b = up256(pusch::freq_bytes_of(g, n_slots));
    const size_t beam_b = up256((size_t)n_slots * g.n_sym * g.n_sc * g.n_beams * sizeof(float2));
    const size_t H_b = up256((size_t)n_slots * g.n_sc * g.n_layers * g.n_beams * sizeof(float2));
    const size_t ls_b = up256((size_t)n_slots * g.n_layers * pusch::ls_pilots_per_layer(g) * g.n_beams * sizeof(float2));
    const bool est = cfg->noise_var == PUSCH_NOISE_ESTIMATE;
    const size_t ne_b = est ? up256((size_t)n_slots * (pusch::kNoiseParts * sizeof(float2) + sizeof(float))) : 0;
    const size_t need = tw_b + words_b + freq_b + beam_b + H_b + ls_b + ne_b;
    if (need > (size_t)PUSCH_NOALLOC_SCRATCH_BYTES) {
        char buf[512];
        snprintf(buf, sizeof buf,
                 "pusch_slot_noalloc: %d slot(s) of this cell need %zu bytes of scratch, more than the static "
                 "buffer's %u bytes; pass fewer slots per call or use pusch_slot with a handle",
                 n_slots, need, (unsigned)PUSCH_NOALLOC_SCRATCH_BYTES);
        return na_fail(PUSCH_ERR_UNSUPPORTED, buf);
    }

    unsigned char *base = nullptr;
    if ((st = scratch_for_current_device(&base)) != PUSCH_OK) return st;
    float2 *tw = reinterpret_cast<float2 *>(base);
    uint32_t *sink = reinterpret_cast<uint32_t *>(base + tw_b);
    uint32_t *tc_err = sink + 4;
    void *freq = base + tw_b + words_b;
    float2 *beam = reinterpret_cast<float2 *>(base + tw_b + words_b + freq_b);
    float2 *H = reinterpret_cast<float2 *>(base + tw_b + words_b + freq_b + beam_b);
    float2 *lsw = reinterpret_cast<float2 *>(base + tw_b + words_b + freq_b + beam_b + H_b);
    float2 *ne_partial = reinterpret_cast<float2 *>(base + tw_b + words_b + freq_b + beam_b + H_b + ls_b);
    float *sigma2 = reinterpret_cast<float *>(ne_partial + (size_t)n_slots * pusch::kNoiseParts);
    uint32_t *stat = status ? status : sink;
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    noalloc_twiddle_kernel<<<(2 * g.n_fft + 255) / 256, 256, 0, s>>>(tw, g.n_fft);
    noalloc_status_kernel<<<1, 1, 0, s>>>(stat, tc_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc set-up launch", e);
    if ((e = pusch::launch_fft(g, n_slots, time_in, freq, tw, tc_err, s)) != cudaSuccess)
        return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc fft launch", e);
    e = pusch::launch_beamform(g, n_slots, freq, static_cast<const float2 *>(W), beam, tc_err, s);
    if (e != cudaSuccess) return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc beamforming launch", e);
    // as in pusch_slot: the detector interpolates the estimate from the LS table itself where it can
    const bool fused = pusch::mmse_interp_supported(g, beam, lsw);
    if (fused)
        e = pusch::launch_ls_pilots(g, n_slots, beam, static_cast<const float2 *>(pilots), lsw, s);
    else
        e = pusch::launch_chest_ls(g, n_slots, beam, static_cast<const float2 *>(pilots), H, lsw, s);
    if (e != cudaSuccess) return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc channel estimation launch", e);
    if (est && (e = pusch::launch_noise_est(g, n_slots, beam, static_cast<const float2 *>(pilots), ne_partial, sigma2,
                                            s)) != cudaSuccess)
        return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc noise estimation launch", e);
    if ((e = pusch::launch_mmse(g, n_slots, H, beam, static_cast<float2 *>(x_hat), bits, stat, s,
                                est ? sigma2 : nullptr, false, fused ? lsw : nullptr)) != cudaSuccess)
        return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc detection launch", e);
    if ((e = pusch::launch_status_fold(stat, tc_err, s)) != cudaSuccess)
        return na_fail(PUSCH_ERR_CUDA, "pusch_slot_noalloc status fold", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}
