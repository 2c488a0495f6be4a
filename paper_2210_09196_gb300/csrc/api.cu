// C ABI of libpusch: handle management, host-side validation and the stage / chain entry points.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>
#include <vector>

#include "internal.cuh"
#include "tune_cache.cuh"


namespace {

thread_local char g_err[512] = "";

constexpr int kSlotStages = 4;  // pusch_slot stages: FFT, beamforming, LS pilot table, detection

pusch_status fail(pusch_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

pusch_status ok() {
    g_err[0] = '\0';
    return PUSCH_OK;
}

pusch_status cuda_fail(cudaError_t e, const char *what) {
    return fail(PUSCH_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

pusch_status validate_cfg(const pusch_cell_cfg *c) {
    if (!c) return fail(PUSCH_ERR_ARG, "cfg is NULL");
    if (!is_pow2(c->n_fft) || c->n_fft < 64 || c->n_fft > 4096)
        return fail(PUSCH_ERR_UNSUPPORTED, "n_fft=%d: must be a power of two in [64, 4096]", c->n_fft);
    if (c->n_sc < 1 || c->n_sc > c->n_fft) return fail(PUSCH_ERR_ARG, "n_sc=%d out of [1, n_fft]", c->n_sc);
    if (c->n_rx < 1 || c->n_rx > 1024) return fail(PUSCH_ERR_UNSUPPORTED, "n_rx=%d out of [1, 1024]", c->n_rx);
    if (c->n_beams < 1 || c->n_beams > 64)
        return fail(PUSCH_ERR_UNSUPPORTED, "n_beams=%d out of [1, 64]", c->n_beams);
    if (c->n_layers < 1 || c->n_layers > 32 || c->n_layers > c->n_beams)
        return fail(PUSCH_ERR_ARG, "n_layers=%d out of [1, min(32, n_beams)]", c->n_layers);
    if (c->dmrs_type == 0 && (c->comb < 1 || c->comb > c->n_sc))
        return fail(PUSCH_ERR_ARG, "comb=%d out of [1, n_sc]", c->comb);
    if (c->dmrs_type != 0 && c->dmrs_type != 1) return fail(PUSCH_ERR_ARG, "dmrs_type must be 0 or 1");
    if (c->dmrs_type == 0) {
        for (int l = 0; l < c->n_layers; ++l)
            if (c->port[l] < 0 || c->port[l] >= c->comb)
                return fail(PUSCH_ERR_ARG, "port[%d]=%d out of [0, comb)", l, c->port[l]);
    } else {
        if (c->n_layers > 4) return fail(PUSCH_ERR_ARG, "type-1 DMRS carries at most 4 ports (n_layers=%d)", c->n_layers);
        if (c->n_sc % 4 != 0) return fail(PUSCH_ERR_ARG, "type-1 DMRS needs n_sc %% 4 == 0 (n_sc=%d)", c->n_sc);
        for (int l = 0; l < c->n_layers; ++l) {
            if (c->port[l] < 0 || c->port[l] > 3) return fail(PUSCH_ERR_ARG, "port[%d]=%d out of [0, 3]", l, c->port[l]);
            for (int m = 0; m < l; ++m)
                if (c->port[m] == c->port[l]) return fail(PUSCH_ERR_ARG, "ports must be distinct");
        }
    }
    if (c->qam_bits != 2 && c->qam_bits != 4) return fail(PUSCH_ERR_ARG, "qam_bits=%d: 2 or 4", c->qam_bits);
    if (c->in_fp16 != 0 && c->in_fp16 != 1) return fail(PUSCH_ERR_ARG, "in_fp16 must be 0 or 1");
    if (c->form != PUSCH_FORM_FP32 && c->form != PUSCH_FORM_MIXED && c->form != PUSCH_FORM_FP8)
        return fail(PUSCH_ERR_ARG, "unknown form %d", c->form);
    if (c->n_sym < 3 || c->n_sym > 16) return fail(PUSCH_ERR_ARG, "n_sym=%d out of [3, 16]", c->n_sym);
    if (c->dmrs_sym[0] < 0 || c->dmrs_sym[0] >= c->n_sym || c->dmrs_sym[1] < 0 || c->dmrs_sym[1] >= c->n_sym ||
        c->dmrs_sym[0] == c->dmrs_sym[1])
        return fail(PUSCH_ERR_ARG, "dmrs_sym must be two distinct symbols of the slot");
    if (c->noise_var != PUSCH_NOISE_ESTIMATE && (!(c->noise_var >= 0.f) || !isfinite(c->noise_var)))
        return fail(PUSCH_ERR_ARG, "noise_var must be >= 0 or PUSCH_NOISE_ESTIMATE");
    if (!(c->loading >= 0.f) || !isfinite(c->loading)) return fail(PUSCH_ERR_ARG, "loading must be >= 0");
    if (c->chol_every < 0 || c->chol_every > c->n_sym - 2)
        return fail(PUSCH_ERR_ARG, "chol_every=%d out of [0, n_sym - 2]", c->chol_every);
    if ((c->cp != 0 && c->cp != 1) || (c->shift_7p5khz != 0 && c->shift_7p5khz != 1))
        return fail(PUSCH_ERR_ARG, "cp and shift_7p5khz must be 0 or 1");
    if (c->cp && c->n_fft < 512)
        return fail(PUSCH_ERR_UNSUPPORTED, "cyclic prefixes need n_fft >= 512 (n_fft=%d)", c->n_fft);
    if (c->form == PUSCH_FORM_MIXED) {
        pusch::Geometry g = pusch::make_geometry(*c);
        if (!pusch::bf_tc_supported(g))
            return fail(PUSCH_ERR_UNSUPPORTED,
                        "mixed form needs n_beams a multiple of 8 and n_rx a multiple of 8 whose W operand fits "
                        "in shared memory");
    }
    if (c->form == PUSCH_FORM_FP8) {
        pusch::Geometry g = pusch::make_geometry(*c);
        if (!pusch::bf_fp8_supported(g))
            return fail(PUSCH_ERR_UNSUPPORTED, "FP8 form needs n_beams a multiple of 8 and n_rx a multiple of 16 "
                                               "up to 512 whose W operand fits in shared memory");
    }
    return PUSCH_OK;
}

size_t freq_bytes(const pusch::Geometry &g, int n_slots) { return pusch::freq_bytes_of(g, n_slots); }
size_t beam_bytes(const pusch::Geometry &g, int n_slots) {
    return (size_t)n_slots * g.n_sym * g.n_sc * g.n_beams * sizeof(float2);
}
size_t ls_bytes(const pusch::Geometry &g, int n_slots) {
    // one table (the two-symbol mean), or one per DMRS symbol when the estimate varies in time
    return (g.chol_every > 0 ? 2 : 1) * (size_t)n_slots * g.n_layers * pusch::ls_pilots_per_layer(g) * g.n_beams *
           sizeof(float2);
}
size_t time_bytes(const pusch::Geometry &g, int n_slots) {
    return (size_t)n_slots * pusch::time_elems_per_slot(g) * (g.in_fp16 ? 4 : 8);
}
size_t pilot_bytes(const pusch::Geometry &g, int n_slots) {
    return (size_t)n_slots * g.n_layers * 2 * g.n_sc * sizeof(float2);
}
size_t xhat_count(const pusch::Geometry &g, int n_slots) {
    return (size_t)n_slots * g.n_layers * g.n_data * g.n_sc;
}
size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t H_bytes(const pusch::Geometry &g, int n_slots) {
    return (size_t)g.n_groups * n_slots * g.n_sc * g.n_layers * g.n_beams * sizeof(float2);
}

constexpr int kMaxChunks = 16;  // pusch_set_pipeline limit

// The FFT output of a chunk run is a self-contained buffer of the chunk's slots (the FP8 form keeps its
// scales after its own planes), so chunk c starts after the 256-byte-aligned buffers of the chunks before it.
// Slack over one buffer of all slots: at most 2 x 256 bytes of alignment per chunk.
size_t freq_ws_bytes(const pusch::Geometry &g, int max_slots) {
    return align256(freq_bytes(g, max_slots)) + 2 * 256 * kMaxChunks;
}

size_t workspace_bytes(const pusch::Geometry &g, int max_slots) {
    size_t b = align256(pusch::fft_twiddle_count(g.n_fft) * sizeof(float2));
    b += freq_ws_bytes(g, max_slots) + align256(beam_bytes(g, max_slots)) + align256(ls_bytes(g, max_slots));
    b += align256(H_bytes(g, max_slots));
    b += align256((size_t)max_slots * pusch::kNoiseParts * sizeof(float2)) + align256((size_t)max_slots * sizeof(float));
    return b;
}

pusch_status check_handle(const pusch_handle *h, int n_slots) {
    if (!h) return fail(PUSCH_ERR_ARG, "handle is NULL");
    if (n_slots < 0 || n_slots > h->max_slots)
        return fail(PUSCH_ERR_ARG, "n_slots=%d out of [0, max_slots=%d]", n_slots, h->max_slots);
    return PUSCH_OK;
}

__global__ void status_init_kernel(uint32_t *status) {
    status[0] = 0u;
    status[1] = 0u;
    status[2] = 0xffffffffu;
    status[3] = 0u;
}

pusch_status reset_status(uint32_t *status, cudaStream_t st) {
    status_init_kernel<<<1, 1, 0, st>>>(status);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "status reset");
    return PUSCH_OK;
}

}  // namespace

namespace pusch {

void set_last_error(const char *msg) { snprintf(g_err, sizeof g_err, "%s", msg); }

Geometry make_geometry(const pusch_cell_cfg &c) {
    Geometry g;
    memset(&g, 0, sizeof g);
    g.n_rx = c.n_rx;
    g.n_fft = c.n_fft;
    g.n_sc = c.n_sc;
    g.n_beams = c.n_beams;
    g.n_layers = c.n_layers;
    g.comb = c.comb;
    g.qam_bits = c.qam_bits;
    g.in_fp16 = c.in_fp16;
    g.form = c.form;
    g.n_sym = c.n_sym;
    g.dmrs0 = c.dmrs_sym[0];
    g.dmrs1 = c.dmrs_sym[1];
    g.noise_var = c.noise_var;
    g.loading = c.loading;
    g.chol_every = c.chol_every;
    g.cp = c.cp;
    g.cp0 = c.cp ? 352 * c.n_fft / 4096 : 0;
    g.cp1 = c.cp ? 288 * c.n_fft / 4096 : 0;
    g.slot_len = (long long)c.n_sym * c.n_fft + (c.cp ? g.cp0 + (long long)(c.n_sym - 1) * g.cp1 : 0);
    g.shift = c.shift_7p5khz;
    g.sc_pitch = sc_pitch_of(c.form, c.n_sc);
    for (int l = 0; l < 32; ++l) g.port[l] = l < c.n_layers ? c.port[l] : 0;
    g.dmrs_type = c.dmrs_type;
    if (c.dmrs_type == 1) {  // the estimate lives at the CDM pair centres: spacing 4, offset 1 + CDM group
        g.comb = 4;
        for (int l = 0; l < c.n_layers; ++l) g.port[l] = 1 + c.port[l] / 2;
    }
    int nd = 0;
    for (int s = 0; s < c.n_sym; ++s)
        if (s != g.dmrs0 && s != g.dmrs1 && nd < 16) g.data_sym[nd++] = s;
    g.n_data = nd;
    // detection groups: one (the two-symbol mean) or groups of chol_every data symbols at their mean time
    const int K = c.chol_every > 0 ? c.chol_every : (nd > 0 ? nd : 1);
    g.n_groups = c.chol_every > 0 ? (nd + K - 1) / K : 1;
    for (int q = 0; q < g.n_groups && q < 16; ++q) {
        double t = 0.0;
        int cnt = 0;
        for (int d = q * K; d < nd && d < (q + 1) * K; ++d, ++cnt)
            t += (double)(g.data_sym[d] - g.dmrs0) / (double)(g.dmrs1 - g.dmrs0);
        g.group_t[q] = cnt ? (float)(t / cnt) : 0.5f;
    }
    return g;
}

}  // namespace pusch

extern "C" {

const char *pusch_last_error(void) { return g_err; }

const char *pusch_version(void) { return "pusch-gb300 0.1 (sm_103a)"; }

int pusch_sc_pitch(const pusch_cell_cfg *cfg) {
    if (!cfg) return 0;
    return pusch::sc_pitch_of(cfg->form, cfg->n_sc);
}

size_t pusch_freq_bytes(const pusch_cell_cfg *cfg, int n_slots) {
    if (validate_cfg(cfg) != PUSCH_OK || n_slots < 0) return 0;
    return pusch::freq_bytes_of(pusch::make_geometry(*cfg), n_slots);
}

pusch_status pusch_workspace_size(const pusch_cell_cfg *cfg, int max_slots, size_t *bytes) {
    pusch_status st = validate_cfg(cfg);
    if (st != PUSCH_OK) return st;
    if (max_slots < 1) return fail(PUSCH_ERR_ARG, "max_slots must be >= 1");
    if (!bytes) return fail(PUSCH_ERR_ARG, "bytes is NULL");
    *bytes = workspace_bytes(pusch::make_geometry(*cfg), max_slots);
    return ok();
}

pusch_status pusch_create(pusch_handle **out, const pusch_cell_cfg *cfg, int max_slots) {
    if (!out) return fail(PUSCH_ERR_ARG, "handle output pointer is NULL");
    *out = nullptr;
    pusch_status st = validate_cfg(cfg);
    if (st != PUSCH_OK) return st;
    if (max_slots < 1) return fail(PUSCH_ERR_ARG, "max_slots must be >= 1");
    pusch_handle *h = new (std::nothrow) pusch_handle();
    if (!h) return fail(PUSCH_ERR_ARG, "out of host memory");
    h->cfg = *cfg;
    h->geo = pusch::make_geometry(*cfg);
    h->max_slots = max_slots;
    cudaGetDevice(&h->device);
    const pusch::Geometry &g = h->geo;

    cudaError_t e;
    const std::vector<float2> tw = pusch::fft_twiddle_table(g.n_fft);
    if ((e = cudaMalloc(&h->twiddle, tw.size() * sizeof(float2))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMemcpy(h->twiddle, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
        goto cuda_error;
    if ((e = cudaMalloc((void **)&h->kernel_err, 16)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMemset(h->kernel_err, 0, 16)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc(&h->freq, freq_ws_bytes(g, max_slots))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&h->beam, beam_bytes(g, max_slots))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&h->ls, ls_bytes(g, max_slots))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&h->H, H_bytes(g, max_slots))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&h->status_sink, 4 * sizeof(uint32_t))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&h->ne_partial, (size_t)max_slots * pusch::kNoiseParts * sizeof(float2))) !=
        cudaSuccess)
        goto cuda_error;
    if ((e = cudaMalloc((void **)&h->sigma2, (size_t)max_slots * sizeof(float))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMemset(h->sigma2, 0, (size_t)max_slots * sizeof(float))) != cudaSuccess) goto cuda_error;
    *out = h;
    return ok();
cuda_error:
    pusch_destroy(h);
    return cuda_fail(e, "pusch_create allocation");
}

pusch_status pusch_destroy(pusch_handle *h) {
    if (!h) return ok();
    cudaDeviceSynchronize();
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    for (int j = 0; j < 2; ++j) {
        if (h->pipe[j]) cudaStreamDestroy(h->pipe[j]);
        if (h->ev_join[j]) cudaEventDestroy(h->ev_join[j]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    cudaFree(h->twiddle);
    cudaFree(h->kernel_err);
    cudaFree(h->freq);
    cudaFree(h->beam);
    cudaFree(h->ls);
    cudaFree(h->H);
    cudaFree(h->status_sink);
    cudaFree(h->ne_partial);
    cudaFree(h->sigma2);
    cudaFree(h->h_time);
    cudaFree(h->h_pilots);
    cudaFree(h->h_xhat);
    cudaFree(h->h_bits);
    cudaFree(h->h_status);
    delete h;
    return ok();
}

pusch_status pusch_ofdm_fft(pusch_handle *h, int n_slots, const void *time_in, void *freq_out, void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!time_in || !freq_out) return fail(PUSCH_ERR_ARG, "pusch_ofdm_fft: NULL buffer");
    cudaError_t e = pusch::launch_fft(h->geo, n_slots, time_in, freq_out, h->twiddle, h->kernel_err,
                                        (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "fft launch");
    return ok();
}

pusch_status pusch_beamform(pusch_handle *h, int n_slots, const void *freq_in, const void *W, void *beam_out,
                            void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!freq_in || !W || !beam_out) return fail(PUSCH_ERR_ARG, "pusch_beamform: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = pusch::launch_beamform(h->geo, n_slots, freq_in, (const float2 *)W, (float2 *)beam_out,
                                           h->kernel_err, s, &h->bf_tune);
    if (e != cudaSuccess) return cuda_fail(e, "beamforming launch");
    return ok();
}

pusch_status pusch_chest_ls(pusch_handle *h, int n_slots, const void *beam, const void *pilots, void *H_hat,
                            void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!beam || !pilots || !H_hat) return fail(PUSCH_ERR_ARG, "pusch_chest_ls: NULL buffer");
    cudaError_t e = pusch::launch_ls_pilots(h->geo, n_slots, (const float2 *)beam, (const float2 *)pilots, h->ls,
                                            (cudaStream_t)stream);
    if (e == cudaSuccess) e = pusch::launch_chest_interp(h->geo, n_slots, h->ls, (float2 *)H_hat, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "channel estimation launch");
    return ok();
}

pusch_status pusch_noise_estimate(pusch_handle *h, int n_slots, const void *beam, const void *pilots, float *sigma2,
                                  void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!beam || !pilots) return fail(PUSCH_ERR_ARG, "pusch_noise_estimate: NULL buffer");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = pusch::launch_noise_est(h->geo, n_slots, (const float2 *)beam, (const float2 *)pilots,
                                            h->ne_partial, h->sigma2, s);
    if (e != cudaSuccess) return cuda_fail(e, "noise estimation launch");
    if (sigma2 && (e = cudaMemcpyAsync(sigma2, h->sigma2, (size_t)n_slots * sizeof(float), cudaMemcpyDeviceToDevice,
                                       s)) != cudaSuccess)
        return cuda_fail(e, "noise estimate copy");
    return ok();
}

pusch_status pusch_mmse_detect(pusch_handle *h, int n_slots, const void *H_hat, const void *beam, void *x_hat,
                               uint8_t *bits, uint32_t *status, void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (!H_hat || !beam || !x_hat || !bits) {
        if (n_slots == 0) return ok();
        return fail(PUSCH_ERR_ARG, "pusch_mmse_detect: NULL buffer");
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *stat = status ? status : h->status_sink;
    if ((st = reset_status(stat, s)) != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    const float *sg2 = h->cfg.noise_var == PUSCH_NOISE_ESTIMATE ? h->sigma2 : nullptr;
    cudaError_t e = pusch::launch_mmse(h->geo, n_slots, (const float2 *)H_hat, (const float2 *)beam, (float2 *)x_hat,
                                       bits, stat, s, sg2);
    if (e != cudaSuccess) return cuda_fail(e, "detection launch");
    // expired waits of this handle's kernels since the last report (stage calls included)
    if ((e = pusch::launch_status_fold(stat, h->kernel_err, s)) != cudaSuccess) return cuda_fail(e, "status fold");
    return ok();
}

}  // extern "C"

namespace {

// Chunk c of a batch of n slots split into k contiguous runs whose sizes differ by at most one.
void chunk_of(int n, int k, int c, int &s0, int &nc) {
    const int q = n / k, r = n % k;
    s0 = c * q + (c < r ? c : r);
    nc = q + (c < r ? 1 : 0);
}

// Profiling records for one call of `runs` chunk runs (nullptr: not timed).
cudaEvent_t *take_records(pusch_handle *h, int runs) {
    if (h->prof_records + runs > h->prof_max_records) return nullptr;
    cudaEvent_t *ev = &h->prof_events[(size_t)h->prof_records * (kSlotStages + 1)];
    h->prof_records += runs;
    ++h->prof_calls;
    return ev;
}

// The chain over slots [s0, s0 + n) of a call, on stream s, in the handle's workspace slice of those slots
// (freq_off: byte offset of the chunk's FFT output buffer). ev: kSlotStages + 1 events or nullptr.
// fft_ctas > 0: the FFT's CTAs per SM for this run (the pipelined runs' default, see slot_batch).
pusch_status run_chain(pusch_handle *h, int s0, int n, size_t freq_off, const void *time_in, const void *W,
                       const void *pilots, void *x_hat, uint8_t *bits, uint32_t *stat, cudaStream_t s,
                       cudaEvent_t *ev, int fft_ctas = 0) {
    const pusch::Geometry &g = h->geo;
    const char *tin = (const char *)time_in + time_bytes(g, s0);
    const float2 *pil = (const float2 *)((const char *)pilots + pilot_bytes(g, s0));
    float2 *xh = (float2 *)x_hat + xhat_count(g, s0);
    uint8_t *bt = bits + xhat_count(g, s0);
    void *freq = (char *)h->freq + freq_off;
    float2 *beam = h->beam + beam_bytes(g, s0) / sizeof(float2);
    float2 *ls = h->ls + ls_bytes(g, s0) / sizeof(float2);
    float2 *H = h->H + H_bytes(g, s0) / sizeof(float2);
    float2 *ne_partial = h->ne_partial + (size_t)s0 * pusch::kNoiseParts;
    float *sigma2 = h->sigma2 + s0;
    cudaError_t e;
    if (ev) cudaEventRecord(ev[0], s);
    if (fft_ctas > 0) {
        pusch::Geometry gf = g;
        gf.fft_cap = fft_ctas;
        e = pusch::launch_fft(gf, n, tin, freq, h->twiddle, h->kernel_err, s);
    } else {
        e = pusch::launch_fft(g, n, tin, freq, h->twiddle, h->kernel_err, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "fft launch");
    if (ev) cudaEventRecord(ev[1], s);
    if ((e = pusch::launch_beamform(g, n, freq, (const float2 *)W, beam, h->kernel_err, s, &h->bf_tune)) != cudaSuccess)
        return cuda_fail(e, "beamforming launch");
    if (ev) cudaEventRecord(ev[2], s);
    const bool est = h->cfg.noise_var == PUSCH_NOISE_ESTIMATE;
    const bool tv = g.chol_every > 0;
    // the two-symbol-mean table: the estimate itself, or the noise estimator's reference when the estimate
    // varies in time
    if ((!tv || est) && (e = pusch::launch_ls_pilots(g, n, beam, pil, ls, s)) != cudaSuccess)
        return cuda_fail(e, "LS pilot table launch");
    if (est && (e = pusch::launch_noise_est(g, n, beam, pil, ne_partial, sigma2, s)) != cudaSuccess)
        return cuda_fail(e, "noise estimation launch");
    // the detector interpolates the estimate from the LS table itself where it can (the interpolated estimate
    // then never goes through HBM); else the interpolation kernel writes it
    const bool fused = !tv && pusch::mmse_interp_supported(g, beam, ls);
    if (tv) {  // per-DMRS-symbol tables and one estimate per detection group
        if ((e = pusch::launch_chest_time(g, n, beam, pil, H, ls, s)) != cudaSuccess)
            return cuda_fail(e, "time-varying estimate launch");
    } else if (!fused && (e = pusch::launch_chest_interp(g, n, ls, H, s)) != cudaSuccess) {
        return cuda_fail(e, "estimate interpolation launch");
    }
    if (ev) cudaEventRecord(ev[3], s);
    if ((e = pusch::launch_mmse(g, n, H, beam, xh, bt, stat, s, est ? sigma2 : nullptr, tv, fused ? ls : nullptr)) !=
        cudaSuccess)
        return cuda_fail(e, "detection launch");
    if (ev) cudaEventRecord(ev[4], s);
    return PUSCH_OK;
}

// Fork: the pipeline streams wait for everything issued so far on s.
pusch_status pipe_fork(pusch_handle *h, cudaStream_t s) {
    cudaError_t e = cudaEventRecord(h->ev_fork, s);
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) e = cudaStreamWaitEvent(h->pipe[j], h->ev_fork, 0);
    return e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "pipeline fork");
}

// Join: s waits for everything issued on the pipeline streams.
pusch_status pipe_join(pusch_handle *h, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
        e = cudaEventRecord(h->ev_join[j], h->pipe[j]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_join[j], 0);
    }
    return e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "pipeline join");
}

// Copies of one chunk for pusch_slot_host: `in` = host->device inputs before the chain, else outputs back.
pusch_status chunk_copies(pusch_handle *h, bool in, int s0, int n, const void *time_host, const void *pil_host,
                          void *xhat_host, uint8_t *bits_host, cudaStream_t s) {
    const pusch::Geometry &g = h->geo;
    cudaError_t e;
    if (in) {
        e = cudaMemcpyAsync((char *)h->h_time + time_bytes(g, s0), (const char *)time_host + time_bytes(g, s0),
                            time_bytes(g, n), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char *)h->h_pilots + pilot_bytes(g, s0), (const char *)pil_host + pilot_bytes(g, s0),
                                pilot_bytes(g, n), cudaMemcpyHostToDevice, s);
        return e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "input copy");
    }
    const size_t x0 = xhat_count(g, s0), nx = xhat_count(g, n);
    e = cudaMemcpyAsync((float2 *)xhat_host + x0, h->h_xhat + x0, nx * sizeof(float2), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits_host + x0, h->h_bits + x0, nx, cudaMemcpyDeviceToHost, s);
    return e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "output copy");
}

// pusch_slot / pusch_slot_host body: the status reset on s, then the chain, as one run on s or as chunk runs
// alternating over the two pipeline streams. With host buffers (time_host != nullptr) each run is bracketed
// by its own input and output copies on its stream, so copies of one chunk overlap the kernels of another.
pusch_status slot_batch(pusch_handle *h, int n_slots, const void *time_in, const void *W, const void *pilots,
                        void *x_hat, uint8_t *bits, uint32_t *stat, cudaStream_t s, const void *time_host,
                        const void *pil_host, void *xhat_host, uint8_t *bits_host) {
    pusch_status st;
    if ((st = reset_status(stat, s)) != PUSCH_OK) return st;
    const int k = h->pipeline < n_slots ? h->pipeline : n_slots;
    // Chunk runs on two streams with device-resident inputs: unless pusch_autotune chose a cap, the tensor-core
    // FFT takes two CTAs per SM (of four) so that the other stream's detector CTAs fit beside it (deployment
    // cell, two runs: 35,190 slots/s against 34,657 with four, whose shared memory leaves no room). With host
    // buffers the other stream carries copies, and the capped FFT only lengthens each run (8,241 against 9,915
    // slots/s end to end), so it keeps four.
    const int fft_ctas = (k > 1 && !time_host && h->geo.fft_cap == 0 && pusch::fft_tc_supported(h->geo)) ? 2 : 0;
    cudaEvent_t *ev = h->prof_events.empty() ? nullptr : take_records(h, k);
    if (k > 1 && (st = pipe_fork(h, s)) != PUSCH_OK) return st;
    size_t freq_off = 0;
    for (int c = 0; c < k && st == PUSCH_OK; ++c) {
        int s0, nc;
        chunk_of(n_slots, k, c, s0, nc);
        cudaStream_t cs = k > 1 ? h->pipe[c & 1] : s;
        if (time_host) st = chunk_copies(h, true, s0, nc, time_host, pil_host, nullptr, nullptr, cs);
        if (st == PUSCH_OK)
            st = run_chain(h, s0, nc, freq_off, time_in, W, pilots, x_hat, bits, stat, cs,
                           ev ? ev + (size_t)c * (kSlotStages + 1) : nullptr, fft_ctas);
        if (st == PUSCH_OK && time_host)
            st = chunk_copies(h, false, s0, nc, nullptr, nullptr, xhat_host, bits_host, cs);
        freq_off += align256(freq_bytes(h->geo, nc));
    }
    // joined on every path once forked: whatever reached the pipeline streams stays ordered before the caller's
    // later work (the first error is the one reported)
    if (k > 1) {
        const pusch_status sj = pipe_join(h, s);
        if (st == PUSCH_OK) st = sj;
    }
    return st;
}

}  // namespace

extern "C" {

pusch_status pusch_slot(pusch_handle *h, int n_slots, const void *time_in, const void *W, const void *pilots,
                        void *x_hat, uint8_t *bits, uint32_t *status, void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!time_in || !W || !pilots || !x_hat || !bits) return fail(PUSCH_ERR_ARG, "pusch_slot: NULL buffer");
    uint32_t *stat = status ? status : h->status_sink;
    st = slot_batch(h, n_slots, time_in, W, pilots, x_hat, bits, stat, (cudaStream_t)stream, nullptr, nullptr, nullptr,
                    nullptr);
    if (st != PUSCH_OK) return st;
    const cudaError_t e = pusch::launch_status_fold(stat, h->kernel_err, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "status fold");
    return ok();
}

pusch_status pusch_set_pipeline(pusch_handle *h, int n_chunks) {
    if (!h) return fail(PUSCH_ERR_ARG, "handle is NULL");
    if (n_chunks < 1 || n_chunks > kMaxChunks) return fail(PUSCH_ERR_ARG, "n_chunks=%d out of [1, %d]", n_chunks,
                                                             kMaxChunks);
    if (n_chunks > 1 && !h->ev_fork) {
        cudaError_t e = cudaSuccess;
        for (int j = 0; j < 2 && e == cudaSuccess; ++j) {
            e = cudaStreamCreateWithFlags(&h->pipe[j], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join[j], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            for (int j = 0; j < 2; ++j) {
                if (h->pipe[j]) cudaStreamDestroy(h->pipe[j]);
                if (h->ev_join[j]) cudaEventDestroy(h->ev_join[j]);
                h->pipe[j] = nullptr;
                h->ev_join[j] = nullptr;
            }
            if (h->ev_fork) cudaEventDestroy(h->ev_fork);
            h->ev_fork = nullptr;
            return cuda_fail(e, "pipeline streams");
        }
    }
    h->pipeline = n_chunks;
    return ok();
}

pusch_status pusch_profile_start(pusch_handle *h, int max_calls) {
    if (!h) return fail(PUSCH_ERR_ARG, "handle is NULL");
    if (max_calls < 0 || max_calls > 1000000) return fail(PUSCH_ERR_ARG, "max_calls out of [0, 1e6]");
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    const int records = max_calls * h->pipeline;
    h->prof_events.assign((size_t)records * (kSlotStages + 1), nullptr);
    for (auto &ev : h->prof_events) {
        cudaError_t e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            h->prof_max_records = h->prof_records = h->prof_calls = 0;
            return cuda_fail(e, "profiling event");
        }
    }
    h->prof_max_records = records;
    h->prof_records = h->prof_calls = 0;
    return ok();
}

pusch_status pusch_profile_read(pusch_handle *h, float *stage_ms, int n_stages, int *n_calls) {
    if (!h) return fail(PUSCH_ERR_ARG, "handle is NULL");
    if (!stage_ms || n_stages < kSlotStages) return fail(PUSCH_ERR_ARG, "stage_ms must hold %d values", kSlotStages);
    for (int k = 0; k < kSlotStages; ++k) stage_ms[k] = 0.f;
    for (int r = 0; r < h->prof_records; ++r) {
        cudaEvent_t *ev = &h->prof_events[(size_t)r * (kSlotStages + 1)];
        cudaError_t e = cudaEventSynchronize(ev[kSlotStages]);
        if (e != cudaSuccess) return cuda_fail(e, "profiling synchronize");
        for (int k = 0; k < kSlotStages; ++k) {
            float ms = 0.f;
            e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
            if (e != cudaSuccess) return cuda_fail(e, "profiling elapsed time");
            stage_ms[k] += ms;
        }
    }
    if (n_calls) *n_calls = h->prof_calls;
    for (cudaEvent_t ev : h->prof_events) cudaEventDestroy(ev);
    h->prof_events.clear();
    h->prof_max_records = h->prof_records = h->prof_calls = 0;
    return ok();
}

pusch_status pusch_slot_host(pusch_handle *h, int n_slots, const void *time_in_host, const void *W,
                             const void *pilots_host, void *x_hat_host, uint8_t *bits_host, uint32_t *status_host,
                             void *stream) {
    pusch_status st = check_handle(h, n_slots);
    if (st != PUSCH_OK) return st;
    if (n_slots == 0) return ok();
    if (!time_in_host || !W || !pilots_host || !x_hat_host || !bits_host)
        return fail(PUSCH_ERR_ARG, "pusch_slot_host: NULL buffer");
    const pusch::Geometry &g = h->geo;
    cudaError_t e;
    if (!h->h_time) {  // staging buffers, sized for max_slots, allocated on first use
        if ((e = cudaMalloc(&h->h_time, time_bytes(g, h->max_slots))) != cudaSuccess) return cuda_fail(e, "staging");
        if ((e = cudaMalloc((void **)&h->h_pilots, pilot_bytes(g, h->max_slots))) != cudaSuccess)
            return cuda_fail(e, "staging");
        if ((e = cudaMalloc((void **)&h->h_xhat, xhat_count(g, h->max_slots) * sizeof(float2))) != cudaSuccess)
            return cuda_fail(e, "staging");
        if ((e = cudaMalloc((void **)&h->h_bits, xhat_count(g, h->max_slots))) != cudaSuccess)
            return cuda_fail(e, "staging");
        if ((e = cudaMalloc((void **)&h->h_status, 4 * sizeof(uint32_t))) != cudaSuccess)
            return cuda_fail(e, "staging");
    }
    cudaStream_t s = (cudaStream_t)stream;
    st = slot_batch(h, n_slots, h->h_time, W, h->h_pilots, h->h_xhat, h->h_bits, h->h_status, s, time_in_host,
                    pilots_host, x_hat_host, bits_host);
    if (st != PUSCH_OK) return st;
    if ((e = pusch::launch_status_fold(h->h_status, h->kernel_err, s)) != cudaSuccess) return cuda_fail(e, "status fold");
    if (status_host &&
        (e = cudaMemcpyAsync(status_host, h->h_status, 4 * sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess)
        return cuda_fail(e, "status copy");
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "stream synchronize");
    return ok();
}

}  // extern "C"

namespace {

// Deterministic stand-in data for pusch_autotune: a hash of the index mapped to [-amp, amp] (as FP16 when fp16),
// or, for W, unit-modulus DFT-like entries / sqrt(n_rx).
__global__ void tune_fill_kernel(void *dst, size_t n, float amp, int fp16, uint32_t seed) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        uint32_t x = (uint32_t)i * 2654435761u ^ seed;
        x ^= x >> 15;
        x *= 2246822519u;
        x ^= x >> 13;
        const float v = amp * ((float)(x & 0xffffu) / 32768.f - 1.f);
        if (fp16)
            static_cast<__half *>(dst)[i] = __float2half_rn(v);
        else
            static_cast<float *>(dst)[i] = v;
    }
}

pusch_status tune_fill(void *dst, size_t n, float amp, int fp16, uint32_t seed, cudaStream_t s) {
    tune_fill_kernel<<<256, 256, 0, s>>>(dst, n, amp, fp16, seed);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "autotune fill");
}

}  // namespace

extern "C" pusch_status pusch_autotune(pusch_handle *h, const char *cache_path, void *stream, int *n_timed) {
    using namespace pusch::tune;
    if (!h) return fail(PUSCH_ERR_ARG, "handle is NULL");
    if (n_timed) *n_timed = 0;
    pusch::Geometry &g = h->geo;
    const int n = h->max_slots;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    std::map<std::string, std::string> cache = read_cache(cache_path);
    std::vector<std::string> lines;
    int timed = 0;
    const int reps = 10;
    char key[192], buf[320];

    // stand-in inputs and outputs of one batch of max_slots slots
    void *time_in = nullptr, *W = nullptr, *pil = nullptr, *xh = nullptr;
    uint8_t *bits = nullptr;
    const size_t t_elems = (size_t)n * pusch::time_elems_per_slot(g) * 2;
    cudaError_t e = cudaMalloc(&time_in, time_bytes(g, n));
    if (e == cudaSuccess) e = cudaMalloc(&W, (size_t)g.n_rx * g.n_beams * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc(&pil, pilot_bytes(g, n));
    if (e == cudaSuccess) e = cudaMalloc(&xh, xhat_count(g, n) * sizeof(float2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&bits, xhat_count(g, n));
    pusch_status st = e == cudaSuccess ? PUSCH_OK : cuda_fail(e, "autotune buffers");
    if (st == PUSCH_OK) st = tune_fill(time_in, t_elems, 0.03f, g.in_fp16, 1u, s);
    if (st == PUSCH_OK) st = tune_fill(W, (size_t)g.n_rx * g.n_beams * 2, 1.f / sqrtf((float)g.n_rx), 0, 2u, s);
    if (st == PUSCH_OK) st = tune_fill(pil, pilot_bytes(g, n) / sizeof(float), 0.7071f, 0, 3u, s);
    const int pipeline0 = h->pipeline;
    auto chain = [&]() { return slot_batch(h, n, time_in, W, pil, xh, bits, h->status_sink, s, nullptr, nullptr,
                                           nullptr, nullptr); };
    if (st == PUSCH_OK) {
        h->pipeline = 1;
        st = chain();   // FFT output, beams and estimate for the per-stage candidates below
    }
    if (st == PUSCH_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "autotune first pass");

    // 1. FFT CTAs per SM (0 = the kernel's own choice, then fewer)
    if (st == PUSCH_OK) {
        snprintf(key, sizeof key, "slot-fft form=%d n_fft=%d in_fp16=%d n_rx=%d slots=%d", g.form, g.n_fft, g.in_fp16,
                 g.n_rx, n);
        auto it = cache.find(key);
        if (it != cache.end()) {
            g.fft_cap = value_of(it->second, "cap", 0);
        } else {
            const int caps[4] = {0, 3, 2, 1};
            float best = 1e30f;
            int best_cap = 0;
            for (int c : caps) {
                g.fft_cap = c;
                const float ms = time_ms(s, reps, [&] {
                    pusch::launch_fft(g, n, time_in, h->freq, h->twiddle, h->kernel_err, s);
                }, &e);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "autotune FFT");
                    break;
                }
                if (ms < best) best = ms, best_cap = c;
            }
            g.fft_cap = best_cap;
            ++timed;
            snprintf(buf, sizeof buf, "%s | cap=%d ms=%.5f", key, best_cap, best);
            lines.push_back(buf);
        }
    }
    // 2. tensor-core GEMM: K rows per pipeline stage and the output path
    if (st == PUSCH_OK && g.form != PUSCH_FORM_FP32) {
        snprintf(key, sizeof key, "slot-bf form=%d n_rx=%d n_beams=%d n_sc=%d slots=%d", g.form, g.n_rx, g.n_beams,
                 g.n_sc, n);
        auto it = cache.find(key);
        if (it != cache.end()) {
            h->bf_tune.chunk_rows = value_of(it->second, "chunk", 0);
            h->bf_tune.staged = value_of(it->second, "staged", 0);
        } else {
            pusch::TcTune cand[8];
            const int nc = pusch::bf_tc_candidates(g, cand, 8);
            float best = 1e30f;
            pusch::TcTune bt;
            for (int i = 0; i < nc && st == PUSCH_OK; ++i) {
                const float ms = time_ms(s, reps, [&] {
                    pusch::launch_beamform(g, n, h->freq, static_cast<const float2 *>(W), h->beam, h->kernel_err, s,
                                           &cand[i]);
                }, &e);
                if (e != cudaSuccess) st = cuda_fail(e, "autotune beamforming");
                else if (ms < best) best = ms, bt = cand[i];
            }
            h->bf_tune = bt;
            ++timed;
            snprintf(buf, sizeof buf, "%s | chunk=%d staged=%d ms=%.5f", key, bt.chunk_rows, bt.staged, best);
            lines.push_back(buf);
        }
    }
    // 3. detector warps per CTA (the 12-data-symbol kernels of one estimate per slot)
    if (st == PUSCH_OK && g.chol_every == 0 && g.n_data == 12) {
        snprintf(key, sizeof key, "slot-det form=%d n_layers=%d n_beams=%d n_sc=%d slots=%d", g.form, g.n_layers,
                 g.n_beams, g.n_sc, n);
        auto it = cache.find(key);
        if (it != cache.end()) {
            g.det_warps = value_of(it->second, "warps", 0);
        } else {
            int ws[4];
            const int nw = pusch::mmse_warp_choices_for(g.n_layers, g.n_beams, ws);
            float best = 1e30f;
            int bw = ws[0];
            const float *sg2 = h->cfg.noise_var == PUSCH_NOISE_ESTIMATE ? h->sigma2 : nullptr;
            const bool fused = pusch::mmse_interp_supported(g, h->beam, h->ls);   // as the chain runs it
            for (int wi = 0; wi < nw; ++wi) {
                const int w = ws[wi];
                g.det_warps = w;
                const float ms = time_ms(s, reps, [&] {
                    pusch::launch_mmse(g, n, h->H, h->beam, static_cast<float2 *>(xh), bits, h->status_sink, s, sg2,
                                       false, fused ? h->ls : nullptr);
                }, &e);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "autotune detection");
                    break;
                }
                if (ms < best) best = ms, bw = w;
            }
            g.det_warps = bw;
            ++timed;
            snprintf(buf, sizeof buf, "%s | warps=%d ms=%.5f", key, bw, best);
            lines.push_back(buf);
        }
    }
    // 4. chunk runs of pusch_slot over the two pipeline streams
    if (st == PUSCH_OK) {
        snprintf(key, sizeof key, "slot-pipe form=%d n_rx=%d n_fft=%d n_sc=%d n_beams=%d n_layers=%d slots=%d", g.form,
                 g.n_rx, g.n_fft, g.n_sc, g.n_beams, g.n_layers, n);
        auto it = cache.find(key);
        int best_k = pipeline0;
        if (it != cache.end()) {
            best_k = value_of(it->second, "chunks", pipeline0);
        } else {
            float best = 1e30f;
            for (int k : {1, 2, 4}) {
                if (k > n) break;
                if (k > 1 && (st = pusch_set_pipeline(h, k)) != PUSCH_OK) break;
                h->pipeline = k;
                pusch_status cst = PUSCH_OK;
                const float ms = time_ms(s, reps, [&] {
                    if (cst == PUSCH_OK) cst = chain();
                }, &e);
                if (cst != PUSCH_OK) {
                    st = cst;
                    break;
                }
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "autotune pipeline");
                    break;
                }
                if (ms < best) best = ms, best_k = k;
            }
            ++timed;
            snprintf(buf, sizeof buf, "%s | chunks=%d ms=%.5f", key, best_k, best);
            lines.push_back(buf);
        }
        h->pipeline = pipeline0;
        if (st == PUSCH_OK) st = pusch_set_pipeline(h, best_k);
    } else {
        h->pipeline = pipeline0;
    }
    cudaStreamSynchronize(s);
    cudaFree(time_in);
    cudaFree(W);
    cudaFree(pil);
    cudaFree(xh);
    cudaFree(bits);
    if (st != PUSCH_OK) return st;
    if (!append_cache(cache_path, lines)) return fail(PUSCH_ERR_ARG, "cannot append to the autotune cache file");
    if (n_timed) *n_timed = timed;
    return ok();
}
