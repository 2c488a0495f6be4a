// Internal declarations shared by the CUDA translation units of libpusch (not part of the C ABI).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <cuda_bf16.h>

#include <vector>

#include "../../include/pusch.h"

namespace pusch {

// ------------------------------------------------------------------------------------ complex helpers
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
    return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
// acc += a * b
__device__ __forceinline__ void cfma(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}
// acc += conj(a) * b
__device__ __forceinline__ void cfmac(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc.y));
}
// acc -= a * b
__device__ __forceinline__ void cfms(float2 &acc, float2 a, float2 b) {
    acc.x = fmaf(-a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(-a.x, b.y, fmaf(-a.y, b.x, acc.y));
}

// ---------------------------------------------------------------------------------- derived geometry
struct Geometry {
    int n_rx, n_fft, n_sc, n_beams, n_layers, comb, qam_bits, in_fp16, form, n_sym;
    int dmrs0, dmrs1;
    int n_data;
    int sc_pitch;                 // mixed / FP8 FFT output: elements between the re and im planes of a row
    float noise_var, loading;
    int port[32];
    int data_sym[16];             // data symbol indices in increasing order
    int chol_every;               // 0, or the data-symbol group size (pusch_cell_cfg.chol_every)
    int n_groups;                 // detection groups (1 when chol_every == 0)
    float group_t[16];            // per group: mean (s - dmrs0) / (dmrs1 - dmrs0) of its data symbols
    int cp;                       // 1: time input is one stream per antenna with NR normal cyclic prefixes
    int cp0, cp1;                 // prefix samples of symbol 0 and of the other symbols (cp == 1)
    long long slot_len;           // samples of one antenna's slot (cp == 1)
    int shift;                    // 1: undo the 7.5 kHz shift before the FFT
    int dmrs_type;                // 1: 3GPP type-1 DMRS; comb / port then give the CDM pair centres (4, 1 + group)
    // launch shapes (pusch_autotune; 0 = the built-in choice)
    int fft_cap;                  // FFT CTAs per SM at most
    int det_warps;                // warps per CTA of the 12-data-symbol detector (0 = the class default)
};

// Complex time samples of one slot's input.
inline long long time_elems_per_slot(const Geometry &g) {
    return g.cp ? (long long)g.n_rx * g.slot_len : (long long)g.n_sym * g.n_rx * g.n_fft;
}

// FFT twiddle table entries: exp(-2 pi i q / n_fft) for q < n_fft, then exp(-2 pi i q / (4 n_fft)) for
// q < n_fft (the derotation of the 7.5 kHz shift).
inline int fft_twiddle_count(int n_fft) { return 2 * n_fft; }
inline std::vector<float2> fft_twiddle_table(int n_fft) {
    std::vector<float2> tw(2 * n_fft);
    for (int q = 0; q < 2 * n_fft; ++q) {
        const double ang = -2.0 * 3.14159265358979323846 * (double)(q % n_fft) / (double)(q < n_fft ? n_fft : 4 * n_fft);
        tw[q] = make_float2((float)cos(ang), (float)sin(ang));
    }
    return tw;
}

// Elements between the re and im planes of an FFT output row (mixed and FP8 forms): every plane starts on a
// 128-byte boundary (one L2 line), because the tensor-core beamforming reads 128-byte rows of the planes.
inline int sc_pitch_of(int form, int n_sc) {
    return form == PUSCH_FORM_FP8 ? (n_sc + 127) & ~127 : (n_sc + 63) & ~63;
}

Geometry make_geometry(const pusch_cell_cfg &c);

// Bytes of the FFT output (pusch_ofdm_fft's freq_out) for n_slots slots of a geometry. FP8 form: the E4M3
// planes [rows][2][sc_pitch] followed, at fp8_scale_offset, by the float block scales
// [n_slots * n_sym][n_blk][n_rx], n_blk = ceil(n_sc / 128).
inline size_t fp8_scale_offset(const Geometry &g, int n_slots) {
    const size_t planes = (size_t)n_slots * g.n_sym * g.n_rx * 2 * g.sc_pitch;
    return (planes + 255) & ~(size_t)255;
}
inline float *fp8_scales(const Geometry &g, int n_slots, void *freq) {
    return reinterpret_cast<float *>(static_cast<uint8_t *>(freq) + fp8_scale_offset(g, n_slots));
}
inline size_t freq_bytes_of(const Geometry &g, int n_slots) {
    const size_t rows = (size_t)n_slots * g.n_sym * g.n_rx;
    if (g.form == PUSCH_FORM_MIXED) return rows * 2 * g.sc_pitch * sizeof(__half);
    if (g.form == PUSCH_FORM_FP8)
        return fp8_scale_offset(g, n_slots) + (size_t)n_slots * g.n_sym * ((g.n_sc + 127) / 128) * g.n_rx * 4;
    return rows * g.n_sc * sizeof(float2);
}

// Sets the thread's pusch_last_error() message.
void set_last_error(const char *msg);

// Bits of a kernel error word (one uint32 on the device per handle, batch or no-alloc call): a bounded wait
// (bounded_wait.cuh) expired in a tensor-core kernel, in the FFT's copy ring, or in the wait self-test.
constexpr uint32_t kErrTensorWait = 1u, kErrFftWait = 2u, kErrSelftest = 4u;
// One thread, ordered on st after the kernels that may set err: when *err != 0, status[0] |=
// PUSCH_STATUS_TIMEOUT and status[3] |= *err, then *err = 0.
cudaError_t launch_status_fold(uint32_t *status, uint32_t *err, cudaStream_t st);

// ------------------------------------------------------------------------------------------ launchers
// Each returns cudaSuccess or the launch error. All pointers are device pointers.
// err (device, one uint32): bit 1 is set if a bounded wait of the FFT kernel expired.
cudaError_t launch_fft(const Geometry &g, int n_slots, const void *time_in, void *freq_out, const float2 *twiddle,
                       uint32_t *err, cudaStream_t st);
// Mixed form, 4096-point FFTs of FP16 samples without prefixes or shift: the tensor-core FFT (fft_tc.cu).
bool fft_tc_supported(const Geometry &g);
cudaError_t launch_fft_tc(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                          uint32_t *err, cudaStream_t st);
cudaError_t launch_beamform_fp32(const Geometry &g, int n_slots, const float2 *freq, const float2 *W, float2 *beam,
                                 cudaStream_t st);
// The full LS estimate (pilot table into ls_scratch, then interpolation); ls_scratch holds
// n_slots * n_layers * ls_pilots_per_layer(g) * n_beams float2.
cudaError_t launch_chest_ls(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *H,
                            float2 *ls_scratch, cudaStream_t st);
// Time-varying estimates of the detection groups (chol_every > 0): ls_scratch holds two tables.
cudaError_t launch_chest_time(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *H,
                              float2 *ls_scratch, cudaStream_t st);
// sigma2 (optional, device, one float per slot): per-slot noise variance replacing g.noise_var.
// time_groups: H holds g.n_groups estimates (launch_chest_time) and each group of g.chol_every data symbols
// is detected with its own.
// The 12-data-symbol kernels run g.det_warps warps per CTA when it is one of mmse_warp_choices_for(n_layers,
// n_beams), else the layer class's default.
cudaError_t launch_mmse(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, float2 *x_hat,
                        uint8_t *bits, uint32_t *status, cudaStream_t st, const float *sigma2 = nullptr,
                        bool time_groups = false, const float2 *ls = nullptr);
// Whether launch_mmse can take the LS table at the pilots (ls) instead of the interpolated estimate H and
// interpolate while staging (16- and 32-layer classes, 32 or 64 beams, one estimate per slot, 16-byte aligned
// beam and table); H is then not read.
bool mmse_interp_supported(const Geometry &g, const float2 *beam, const float2 *ls);
// The warps per CTA the 12-data-symbol detector of n_layers layers and n_beams beams may run (out: at most 4;
// the first is the default); returns their count.
int mmse_warp_choices_for(int n_layers, int n_beams, int *out);
// LS values at the pilot subcarriers: ls[slot][l][k][b] for pilot q = port[l] + k * comb, k < kmax.
int ls_pilots_per_layer(const Geometry &g);
// sym = -1: the mean of the two DMRS symbols; 0 / 1: that DMRS symbol alone.
cudaError_t launch_ls_pilots(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *ls,
                             cudaStream_t st, int sym = -1);
size_t ls_table_elems(const Geometry &g, int n_slots);
// The full estimate H [slots][n_sc][n_layers][n_beams] interpolated from the LS pilot table.
// time_groups: ls holds the two DMRS symbols' tables back to back and H receives g.n_groups estimates
// (group q at g.group_t[q]), each n_slots * n_sc * n_layers * n_beams values.
cudaError_t launch_chest_interp(const Geometry &g, int n_slots, const float2 *ls, float2 *H, cudaStream_t st,
                                bool time_groups = false);
// Noise-variance estimate per slot from the pilot residuals (Section II "NE"): partial needs
// n_slots * kNoiseParts float2 of scratch; sigma2 receives one float per slot.
constexpr int kNoiseParts = 64;
cudaError_t launch_noise_est(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots,
                             float2 *partial, float *sigma2, cudaStream_t st);
// Launch shape of the tensor-core beamforming kernel: K rows per pipeline stage and whether the epilogue
// writes through shared memory and TMA stores. chunk_rows = 0 lets the kernel choose from its shared-memory
// budget; a shape that does not fit falls back to that choice.
struct TcTune {
    int chunk_rows = 0;
    int staged = 0;
};
// The feasible shapes for g's form (tensor-core forms only); returns how many were written (<= max_out).
int bf_tc_candidates(const Geometry &g, TcTune *out, int max_out);

// Mixed form: the tcgen05 beamforming GEMM. err_word (device, one uint32) gets bit 0 set if a bounded
// wait of the kernel expired.
cudaError_t launch_beamform_tc(const Geometry &g, int n_slots, const __half *freq16, const float2 *W, float2 *beam,
                               uint32_t *err_word, cudaStream_t st, const TcTune *tune = nullptr);
bool bf_tc_supported(const Geometry &g);
// FP8 form: E4M3 codes with power-of-two block scales (layout of freq_bytes_of), same kernel family.
cudaError_t launch_beamform_fp8(const Geometry &g, int n_slots, const uint8_t *freq8, const float *scales,
                                const float2 *W, float2 *beam, uint32_t *err_word, cudaStream_t st,
                                const TcTune *tune = nullptr);
bool bf_fp8_supported(const Geometry &g);
// FP32 form on the tensor cores with three TF32 products per FP32 product (beamform_tf32.cu): n_sc even,
// n_rx a multiple of 16, n_beams a multiple of 8 up to 64, W's operands within shared memory.
bool bf_tf32_supported(const Geometry &g);
cudaError_t launch_beamform_tf32(const Geometry &g, int n_slots, const float2 *freq, const float2 *W, float2 *beam,
                                 uint32_t *err_word, cudaStream_t st);
// Beamforming of the FFT output in the geometry's form (FP32: 3xTF32 tensor cores where supported and the
// pointers are 16-byte aligned, else SIMT; FP16 or FP8 tensor cores).
inline cudaError_t launch_beamform(const Geometry &g, int n_slots, const void *freq, const float2 *W, float2 *beam,
                                   uint32_t *err_word, cudaStream_t st, const TcTune *tune = nullptr) {
    if (g.form == PUSCH_FORM_MIXED)
        return launch_beamform_tc(g, n_slots, static_cast<const __half *>(freq), W, beam, err_word, st, tune);
    if (g.form == PUSCH_FORM_FP8)
        return launch_beamform_fp8(g, n_slots, static_cast<const uint8_t *>(freq),
                                   fp8_scales(g, n_slots, const_cast<void *>(freq)), W, beam, err_word, st, tune);
    if (bf_tf32_supported(g) && reinterpret_cast<uintptr_t>(freq) % 16 == 0 && reinterpret_cast<uintptr_t>(beam) % 16 == 0)
        return launch_beamform_tf32(g, n_slots, static_cast<const float2 *>(freq), W, beam, err_word, st);
    return launch_beamform_fp32(g, n_slots, static_cast<const float2 *>(freq), W, beam, st);
}

// Learned channel-estimate denoiser (cnn.cu). Parameters packed per layer as W[co][ci][3][3], b[co].
int cnn_param_count();
// acts rows of ld elements (0 = w); err (optional): error word of the tensor-core layers' bounded waits.
cudaError_t cnn_forward(int n, int w, const __nv_bfloat16 *x, const __nv_bfloat16 *P, float *y, __nv_bfloat16 *acts,
                        cudaStream_t st, int ld = 0, uint32_t *err = nullptr);
// The 32 -> 32 convolution with ReLU on the tensor cores: in, out [n][32][2][ld] bf16 (ld % 8 == 0, dil % 8 == 0).
bool conv32_tc_supported(int ld, int dil);
cudaError_t launch_conv32_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *W, const __nv_bfloat16 *b,
                             __nv_bfloat16 *out, int n, int w, int ld, int dil, uint32_t *err, cudaStream_t st);
cudaError_t cnn_backward(int n, int w, const __nv_bfloat16 *x, const __nv_bfloat16 *acts, const __nv_bfloat16 *P,
                         const float *y, const float *target, float *grad, float *loss, float *work,
                         __nv_bfloat16 *wflip, cudaStream_t st);
cudaError_t cnn_adam(int step, float lr, float b1, float b2, float eps, float *p, __nv_bfloat16 *pb, const float *g,
                     float *m, float *v, cudaStream_t st);
cudaError_t launch_ls_grid(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots,
                           __nv_bfloat16 *grid, float *scale, cudaStream_t st);
cudaError_t launch_cnn_to_h(const Geometry &g, int n_slots, float kappa, const float *y, const float *scale,
                            const float2 *beam, const float2 *pilots, float2 *H, float *resid, uint8_t *fallback,
                            cudaStream_t st);

}  // namespace pusch

struct pusch_handle {
    pusch_cell_cfg cfg;
    pusch::Geometry geo;
    int max_slots = 0;
    int device = 0;
    float2 *twiddle = nullptr;      // FFT twiddle table (fft_twiddle_table)
    uint32_t *kernel_err = nullptr;   // error word (kErr* bits) of the handle's kernels, folded into the status
    void *freq = nullptr;           // workspace: FFT output
    float2 *beam = nullptr;         // workspace: beamformed grid
    float2 *ls = nullptr;           // workspace: LS values at the pilot subcarriers
    float2 *H = nullptr;            // workspace: the interpolated estimate (pusch_slot)
    uint32_t *status_sink = nullptr;  // status words used when the caller passes NULL
    float2 *ne_partial = nullptr;     // noise estimation: per (slot, part) partial sums
    float *sigma2 = nullptr;          // noise estimation: per-slot estimate (read by the detector in estimate mode)
    // staging for pusch_slot_host (allocated on first use)
    void *h_time = nullptr;
    float2 *h_pilots = nullptr;
    float2 *h_xhat = nullptr;
    uint8_t *h_bits = nullptr;
    uint32_t *h_status = nullptr;
    // pipelined pusch_slot (pusch_set_pipeline): the batch runs as `pipeline` chunks of slots alternating over
    // two streams, forked from and joined to the caller's stream by events
    int pipeline = 1;
    cudaStream_t pipe[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr;
    cudaEvent_t ev_join[2] = {nullptr, nullptr};
    // per-stage timing of pusch_slot (pusch_profile_start / pusch_profile_read): one record of
    // kSlotStages + 1 events per chunk run
    std::vector<cudaEvent_t> prof_events;  // [max_records][kSlotStages + 1]
    int prof_max_records = 0;
    int prof_records = 0;
    int prof_calls = 0;
    // learned-estimator workspace (pusch_chest_cnn; allocated on first use, sized for max_slots)
    void *cnn_grid = nullptr;       // [grids][2][2][n_sc] bf16
    float *cnn_scale = nullptr;     // [grids]
    void *cnn_acts = nullptr;       // [3][grids][32][2][n_sc] bf16
    float *cnn_y = nullptr;         // [grids][2][2][n_sc]
    // launch shapes chosen by pusch_autotune (the FFT cap and detector warps live in geo)
    pusch::TcTune bf_tune;
};
