/*
 * pusch.h -- C ABI of the GB300 (sm_103a) PUSCH receive hot path.
 *
 * The path is the lower-PHY PUSCH receive chain of "Efficient Parallelization of 5G-PUSCH on a Scalable
 * RISC-V Many-core Processor" (arXiv 2210.09196), Section II and Fig. 1:
 *   OFDM demodulation (one FFT per antenna and symbol) -> beamforming (y = W^H x per subcarrier)
 *   -> LS channel estimation on the DMRS symbols -> MMSE MIMO detection (Eq. 2) by Gram matrix,
 *   Cholesky factorisation (Section V-C) and two triangular solves -> hard decisions.
 *
 * Conventions shared by every entry point
 *   - Complex numbers are interleaved (re, im). "c64" = two floats (torch.complex64); "c16" = two IEEE
 *     binary16 values (torch.complex32 / half2).
 *   - Every data pointer is a DEVICE pointer owned by the caller, except in pusch_slot_host, which takes
 *     host pointers. The library never frees caller memory. `stream` is a cudaStream_t (NULL = legacy
 *     default stream). Calls are asynchronous on that stream; outputs are valid once it reaches them.
 *   - A batch of n_slots slots of the same cell is processed by one call; arrays carry a leading
 *     [n_slots] dimension that is not repeated in the layouts below.
 *   - Arguments are validated on the host before any launch; an invalid call returns PUSCH_ERR_ARG (or
 *     PUSCH_ERR_UNSUPPORTED for a shape outside the supported range) and launches nothing.
 *     pusch_last_error() then returns a message (thread-local, valid until the next call on the thread).
 *   - Numeric failures inside a kernel (a non-positive Cholesky pivot, a non-finite value) do not change
 *     the return value; they are reported through the caller's device status words (see PUSCH_STATUS_*).
 *   - No C++ exception crosses this interface.
 *
 * Supported shapes: n_fft a power of two in [64, 4096]; 1 <= n_sc <= n_fft; 1 <= n_beams <= 64;
 * mixed form: n_rx a multiple of 8 and n_beams a multiple of 8; FP8 form: n_rx a multiple of 16 up to 512
 * and n_beams a multiple of 8; in both, W's FP16 image (4 n_rx n_beams FP16 values) must fit in shared
 * memory with the operand ring (up to 256 antennas at 64 beams);
 * 1 <= n_layers <= 32 and n_layers <= n_beams; 1 <= comb <= n_sc; n_sym = 14 with two distinct DMRS
 * symbols; 1 <= n_rx <= 1024; qam_bits 2 (QPSK) or 4 (16-QAM).
 */
#ifndef PUSCH_H
#define PUSCH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PUSCH_OK = 0,
    PUSCH_ERR_ARG = -1,         /* invalid argument (null pointer, size out of range, bad config)   */
    PUSCH_ERR_CUDA = -2,        /* a CUDA runtime call failed; the message names it                 */
    PUSCH_ERR_NUMERIC = -3,     /* only from pusch_status_check: the status words report a failure  */
    PUSCH_ERR_TIMEOUT = -4,     /* only from pusch_status_check: a bounded device wait expired      */
    PUSCH_ERR_UNSUPPORTED = -5  /* valid but outside the shapes this build implements               */
} pusch_status;

/* Arithmetic form of the chain. */
typedef enum {
    PUSCH_FORM_FP32 = 0,   /* plain: FFT and beamforming in FP32, intermediates stored as c64           */
    PUSCH_FORM_MIXED = 1,  /* FFT output stored as FP16 (4096-point rows of FP16 samples on the tcgen05
                              tensor cores with FP16 operands and FP32 accumulation, other shapes in FP32
                              registers); beamforming on the tensor cores with FP16 operands and FP32
                              accumulation.                                                              */
    PUSCH_FORM_FP8 = 2     /* FFT output stored as FP8 E4M3 with one power-of-two scale per 128
                              subcarriers of each (symbol, antenna) row; W quantised to E4M3 with one
                              power-of-two scale per (beam, 128 antennas); beamforming is the
                              block-scaled product of the two quantised operands, on the tcgen05 tensor
                              cores with FP32 accumulation (the codes enter the MMA as their exact FP16
                              values). Channel estimation and detection keep FP32 accuracy in every
                              form: FP32 arithmetic, except that the 16- and 32-layer detectors form the
                              Gram matrix and the right-hand sides on the tensor cores from TF32 operands
                              split in two parts (three products each, FP32 accumulation).              */
} pusch_form;

/* Device status words written by the detection kernels (uint32_t status[4]):
 *   status[0] bit field of PUSCH_STATUS_* flags
 *   status[1] number of (slot, subcarrier) factorisations whose pivot was not a positive finite number
 *             (with chol_every > 0, counted per detection group)
 *   status[2] smallest failing (slot * n_sc + subcarrier) index, 0xFFFFFFFF if none
 *   status[3] the kernel error bits behind PUSCH_STATUS_TIMEOUT: 1 a wait of a tensor-core kernel, 2 a wait
 *             of the FFT's copy ring, 4 the wait self-test (pusch_selftest_wait); 0 if none
 * The entry points that take `status` reset it to {0, 0, 0xFFFFFFFF, 0} on the stream first.
 * Every kernel that waits on asynchronous copies or MMAs gives up after 2 s and sets a bit in an error word
 * of its handle (or batch, or no-alloc call) instead of hanging; pusch_slot, pusch_slot_host,
 * pusch_mmse_detect, pusch_batch_run and pusch_slot_noalloc move that word into status[0] / status[3] at
 * their end (pusch_mmse_detect also reports expiries of the handle's earlier stage calls) and clear it. */
#define PUSCH_STATUS_PIVOT 0x1u     /* Cholesky met a non-positive or non-finite pivot            */
#define PUSCH_STATUS_NONFINITE 0x2u /* a detected symbol came out non-finite                      */
#define PUSCH_STATUS_TIMEOUT 0x4u   /* a bounded device wait expired: the call's outputs are not valid */

typedef struct {
    int n_rx;          /* N_R receive antennas                                                   */
    int n_fft;         /* N_F FFT size                                                           */
    int n_sc;          /* N_SC active subcarriers; subcarrier a is FFT bin (a - n_sc/2) mod n_fft */
    int n_beams;       /* N_B beams                                                              */
    int n_layers;      /* N_L layers (single-layer users) detected jointly on every subcarrier   */
    int comb;          /* DMRS comb size: layer l has pilots on subcarriers a, a % comb == port[l] */
    int port[32];      /* comb offset of each layer, 0 <= port[l] < comb                          */
    int qam_bits;      /* 2 = QPSK, 4 = 16-QAM (Gray, 3GPP TS 38.211 5.1.3/5.1.4)                 */
    int in_fp16;       /* 1: time samples are c16; 0: c64                                        */
    int form;          /* pusch_form                                                             */
    int n_sym;         /* OFDM symbols per slot, 14                                              */
    int dmrs_sym[2];   /* the two DMRS (pilot) symbols, e.g. {2, 11}                             */
    float noise_var;   /* sigma^2 of Eq. 2, or PUSCH_NOISE_ESTIMATE: estimated per slot from the pilots  */
    float loading;     /* extra diagonal loading added to sigma^2 (0 = the plain Eq. 2)          */
    int chol_every;    /* 0: one estimate per slot (mean of the two DMRS symbols), one factorisation per
                          subcarrier. K in [1, n_sym - 2] (pusch_slot only): the estimate of each DMRS
                          symbol is kept apart and interpolated linearly in time, the data symbols are
                          taken in increasing order in groups of K, and each group is detected with the
                          estimate at its mean symbol time and one factorisation per subcarrier (K = 1:
                          one per data symbol, Section VI's schedule; K = n_sym - 2 gives the 0 result
                          up to rounding)                                                          */
    int cp;            /* 0: time samples [n_sym][n_rx][n_fft] per slot (prefixes already removed).
                          1: NR normal cyclic prefixes (TS 38.211 5.3.1, 30 kHz): per slot one stream per
                          antenna, [n_rx][slot_len] with slot_len = n_sym * n_fft + cp0 + (n_sym - 1) * cp1,
                          cp0 = 352 * n_fft / 4096 (symbol 0), cp1 = 288 * n_fft / 4096 (other symbols);
                          symbol s's useful part starts at s * (n_fft + cp1) + cp0. Needs n_fft >= 512.
                          Not in the ragged batch (nor shift_7p5khz).                                */
    int shift_7p5khz;  /* 1: the transmitter shifted the spectrum up by 7.5 kHz (a quarter of the 30 kHz
                          spacing) with the phase reference at the start of each useful part (TS 38.211
                          5.4): sample n of the useful part is multiplied by exp(-2 pi i n / (4 n_fft))
                          before the FFT. 0: no shift.                                               */
    int dmrs_type;     /* 0: the comb pilot model above (layer l on subcarriers a % comb == port[l]).
                          1: 3GPP type-1 single-symbol DMRS (TS 38.211 6.4.1.1.3): port[l] in {0..3}
                          (antenna ports 1000..1003, distinct), n_layers <= 4, n_sc % 4 == 0; port p
                          sends w_f(k') r(2n + k') on subcarriers 4n + 2k' + p / 2 (w_f = (+1, -1) for odd
                          p), so two ports share each comb-2 CDM group. pilots holds those values
                          (pusch_dmrs_type1_pilots). The LS estimate despreads each pair of a group,
                          1/2 (y(k0) / p(k0) + y(k0 + 2) / p(k0 + 2)), placed at k0 + 1, then interpolates
                          between the pair centres as above; the noise estimate fits each CDM group's
                          ports to the pair's 4 observations and divides the residual energy by its
                          4 - m degrees of freedom (m ports in the group). comb is ignored. Not in the
                          ragged batch or the learned estimator.                                      */
} pusch_cell_cfg;

/* noise_var value that makes the chain estimate sigma^2 per slot (pusch_noise_estimate) instead of using a
 * given value: pusch_slot estimates after the LS stage; pusch_mmse_detect uses the estimates of the handle's
 * last pusch_noise_estimate call. Not accepted by pusch_batch_create. */
#define PUSCH_NOISE_ESTIMATE (-1.0f)

typedef struct pusch_handle pusch_handle;   /* opaque: owns the twiddle table and workspace   */

/* Creates a handle for one cell configuration and batches of up to max_slots slots. Allocates device
 * memory for the FFT twiddle table, the beam-matrix operand and the chain's intermediates (see
 * pusch_workspace_size) on the current device. Synchronous. */
pusch_status pusch_create(pusch_handle **h, const pusch_cell_cfg *cfg, int max_slots);

/* Frees everything the handle owns. Synchronises the device first. NULL is accepted. */
pusch_status pusch_destroy(pusch_handle *h);

/* Bytes of device workspace pusch_create allocates for (cfg, max_slots). */
pusch_status pusch_workspace_size(const pusch_cell_cfg *cfg, int max_slots, size_t *bytes);

/* Number of elements between the re and im planes of one FFT output row of the mixed form (binary16 planes:
 * n_sc rounded up to a multiple of 64) or of the FP8 form (byte planes: n_sc rounded up to a multiple of
 * 128), so that every plane starts on a 128-byte boundary (the tensor-core beamforming reads 128-byte rows
 * of the planes, one L2 line each). */
int pusch_sc_pitch(const pusch_cell_cfg *cfg);

/* Bytes of the FFT output buffer (freq_out of pusch_ofdm_fft, freq_in of pusch_beamform) for n_slots slots
 * of cfg's form; 0 for an invalid cfg or n_slots < 0. */
size_t pusch_freq_bytes(const pusch_cell_cfg *cfg, int n_slots);

/*
 * OFDM demodulation (Section II; Table I "OFDM dem."): for every slot, symbol s and antenna r,
 *     X[s][r][a] = sum_n x[s][r][n] exp(-2 pi i k n / N_F),  k = (a - N_SC/2) mod N_F,  a < N_SC.
 * time_in : [n_sym][n_rx][n_fft] c64 (cfg.in_fp16 = 0) or c16 (cfg.in_fp16 = 1).
 * freq_out: FP32 form  -> [n_sym][n_rx][n_sc] c64.
 *           mixed form -> [n_sym][n_rx][2][pitch] binary16: plane 0 = re, plane 1 = im of bins 0..n_sc-1
 *                         (pitch = pusch_sc_pitch(cfg); elements n_sc..pitch-1 are written as 0).
 *           FP8 form   -> E4M3 codes [n_slots][n_sym][n_rx][2][pitch] (planes as above, pads 0) and, at
 *                         byte offset ceil256(n_slots * n_sym * n_rx * 2 * pitch), float block scales
 *                         [n_slots][n_sym][n_blk][n_rx], n_blk = ceil(n_sc / 128): block j of a row holds
 *                         subcarriers 128 j .. 128 j + 127 as code * scale, where scale = 2^e with e the
 *                         smallest integer (>= -126) for which the block's largest |re| or |im| is at most
 *                         448 * 2^e, and code = E4M3(value / scale) rounded to nearest even; a block
 *                         holding a non-finite value gets scale NaN. This leading-n_slots layout is the
 *                         one exception to the per-slot convention; the size is pusch_freq_bytes.
 */
pusch_status pusch_ofdm_fft(pusch_handle *h, int n_slots, const void *time_in, void *freq_out, void *stream);

/*
 * Beamforming (Section II, Table I "BF": a matrix-matrix product with known coefficients):
 *     Y[s][a][b] = sum_r conj(W[r][b]) X[s][r][a]      (y = W^H x per subcarrier and symbol)
 * freq_in : the layout pusch_ofdm_fft writes for cfg.form (and the same n_slots).
 * W       : [n_rx][n_beams] c64. The mixed form rounds it to FP16; the FP8 form quantises it to E4M3 with
 *           one power-of-two scale per (beam, block of 128 antennas), chosen like the sample scales.
 * beam_out: [n_sym][n_sc][n_beams] c64 (all symbols, DMRS included).
 */
pusch_status pusch_beamform(pusch_handle *h, int n_slots, const void *freq_in, const void *W, void *beam_out,
                            void *stream);

/*
 * LS channel estimation (Section II: block-type pilots filling whole OFDM symbols; LS is an element-wise
 * division). For layer l and each of its pilot subcarriers q (q % comb == port[l]):
 *     LS[q][l][b] = 1/2 sum_{j=0,1} Y[dmrs_sym[j]][q][b] / P[l][j][q]
 * and every subcarrier a is linearly interpolated between the neighbouring pilot subcarriers of the
 * layer, holding the first/last pilot's value outside them. With dmrs_type = 1 the values are the despread
 * CDM pairs at the pair centres instead (pusch_cell_cfg.dmrs_type); with chol_every > 0 this stage still
 * returns the two-symbol mean (the time-varying estimates live inside pusch_slot).
 * beam   : [n_sym][n_sc][n_beams] c64 (only the DMRS symbols are read).
 * pilots : [n_layers][2][n_sc] c64 (entries off the layer's comb are not read).
 * H_hat  : [n_sc][n_layers][n_beams] c64.
 */
pusch_status pusch_chest_ls(pusch_handle *h, int n_slots, const void *beam, const void *pilots, void *H_hat,
                            void *stream);

/*
 * Noise-variance estimation (Section II "NE": the autocorrelation of the difference between the received pilot
 * symbols and the output expected from the estimated channel and the pilots). Per slot, over the pilot
 * subcarriers q of every layer l, both DMRS symbols j and all beams b, with LS[q] = 1/2 sum_j y_j[q] / p_j[q]
 * (the channel estimate at the layer's own pilot):
 *     sigma2[slot] = 2 * mean |y_j[q][b] - LS[q][b] p_{l,j}[q]|^2
 * The factor 2 undoes the two-symbol mean (E|.|^2 = sigma^2 / 2 for unit-modulus pilots and a channel that is
 * constant between the DMRS symbols). The sum runs in a fixed order (no float atomics): reruns are
 * bit-identical. beam, pilots: as pusch_chest_ls. sigma2: [n_slots] floats (device; may be NULL). The
 * estimates are also kept in the handle for pusch_mmse_detect in PUSCH_NOISE_ESTIMATE mode.
 */
pusch_status pusch_noise_estimate(pusch_handle *h, int n_slots, const void *beam, const void *pilots, float *sigma2,
                                  void *stream);

/*
 * MMSE detection (Eq. 2 with Section II's Cholesky + two triangular solves), per subcarrier a:
 *     G = H^H H + (noise_var + loading) I,  G = L L^H,  L z = H^H y,  L^H x = z
 * for the 12 data symbols (all symbols other than dmrs_sym, in increasing order); hard decisions by
 * Gray demapping with ties to bit 0. G and L are formed once per subcarrier (the estimate does not change
 * within the slot, so this equals forming them per data symbol).
 * H_hat : [n_sc][n_layers][n_beams] c64;  beam : [n_sym][n_sc][n_beams] c64.
 * x_hat : [n_layers][n_sym-2][n_sc] c64;  bits : [n_layers][n_sym-2][n_sc] uint8 (bit j = b_j).
 * status: uint32_t[4] device status words (may be NULL to skip reporting).
 */
pusch_status pusch_mmse_detect(pusch_handle *h, int n_slots, const void *H_hat, const void *beam, void *x_hat,
                               uint8_t *bits, uint32_t *status, void *stream);

/*
 * The whole chain for n_slots slots (Fig. 1): OFDM FFT -> beamforming -> LS division at the pilot
 * subcarriers -> interpolated estimate (-> noise estimate when noise_var is PUSCH_NOISE_ESTIMATE) -> MMSE
 * detection. The FFT output, the beamformed grid, the LS table and the estimate live in the handle's
 * workspace (n_slots <= max_slots), with the arithmetic of the stage entry points (the result equals
 * pusch_chest_ls + pusch_mmse_detect on the pusch_beamform output, bit for bit). With 9 to 32 layers and 32
 * or 64 beams the detector interpolates the estimate from the LS table while it stages its tiles, so the
 * estimate is not written to memory (the estimate buffer is then unused). With chol_every = K > 0 the
 * estimate varies in time and the detector factorises once per group of K data symbols (pusch_cell_cfg).
 * time_in, W, pilots, x_hat, bits, status: as in the stage entry points. Kernels: a one-thread status reset,
 * then per run FFT, beamforming, LS table (+ noise estimate), estimate (unless the detector interpolates),
 * detection; see pusch_set_pipeline.
 */
pusch_status pusch_slot(pusch_handle *h, int n_slots, const void *time_in, const void *W, const void *pilots,
                        void *x_hat, uint8_t *bits, uint32_t *status, void *stream);

/*
 * 3GPP type-1 DMRS values for dmrs_type = 1 (TS 38.211 5.2.1, 6.4.1.1; not in the paper, whose pilots are a
 * block-type model): for slot i (slot number slot_numbers[i] within the frame, host array, 0..159) and DMRS
 * symbol l = cfg->dmrs_sym[j], the Gold sequence c(n) of c_init = (2^17 (14 slot + l + 1)(2 n_id + 1) + 2 n_id
 * + n_scid) mod 2^31 gives r(m) = ((1 - 2c(2m)) + i (1 - 2c(2m + 1))) / sqrt 2, and layer l's port p gets
 * w_f(k') r(2n + k') on subcarriers k = 4n + 2k' + p / 2 (subcarrier 0 = the band's first), zero elsewhere.
 * pilots: DEVICE [n_slots][n_layers][2][n_sc] c64, written on `stream`. n_id in [0, 65535], n_scid in {0, 1}.
 * PUSCH_ERR_ARG for a cfg that is not dmrs_type 1 or arguments out of range.
 */
pusch_status pusch_dmrs_type1_pilots(const pusch_cell_cfg *cfg, int n_slots, const int *slot_numbers, int n_id,
                                     int n_scid, void *pilots, void *stream);

/*
 * Pipelining of pusch_slot and pusch_slot_host (a GPU scheduling choice; no counterpart in the paper).
 * n_chunks = 1 (the default): the batch runs as one pass of the kernels on the caller's stream.
 * n_chunks in [2, 16]: the batch runs as min(n_chunks, n_slots) passes over contiguous runs of slots (sizes
 * differing by at most one), issued alternately on two streams owned by the handle; they start after the
 * work already queued on the caller's stream and the caller's stream waits for them (events), so the call is
 * still ordered on `stream`. Runs on the two streams overlap on the GPU (one run's FFT beside the other's
 * detector; in pusch_slot_host one run's copies beside another's kernels). With two or more runs of
 * pusch_slot the mixed form's 4096-point tensor-core FFT takes two CTAs per SM instead of four unless
 * pusch_autotune chose a number, so that the other stream's detector finds room beside it. Results are bit-identical for
 * every n_chunks: each slot's arithmetic does not depend on the batch it is in. Each run uses the workspace
 * slice of its own slots. Returns PUSCH_ERR_ARG for n_chunks out of range, PUSCH_ERR_CUDA if the streams
 * cannot be created (the setting is then unchanged).
 */
pusch_status pusch_set_pipeline(pusch_handle *h, int n_chunks);

/*
 * pusch_slot on HOST buffers: copies time_in and pilots host->device into handle-owned staging buffers,
 * runs the chain, copies x_hat, bits and status device->host, then waits for `stream`. Without pipelining
 * everything runs on `stream`; with it each run's copies go on that run's stream (pusch_set_pipeline).
 * W is a DEVICE pointer (it is fixed per cell). Host buffers should be page-locked for full speed.
 */
pusch_status pusch_slot_host(pusch_handle *h, int n_slots, const void *time_in_host, const void *W,
                             const void *pilots_host, void *x_hat_host, uint8_t *bits_host, uint32_t *status_host,
                             void *stream);

/* ------------------------------------------------------------------------------------------------------
 * Learned channel-estimate denoiser (an addition to the paper's LS estimator, which stays the fallback).
 * A 4-layer CNN of 3x3 zero-padded ("same") convolutions 2 -> 32 -> 32 -> 32 -> 2, dilated along the
 * subcarrier axis by 1, 8, 16 and 1 (tap offsets d * {-1, 0, 1}; the 2-row DMRS axis is not dilated), with
 * ReLU after the first three and the input added to the output, run on grids
 * [n][2 channels (re, im)][2 DMRS symbols][w subcarriers].
 * Parameters (pusch_cnn_param_count() = 19682) are packed per layer as W[co][ci][3][3] then b[co]; weights
 * and activations are bfloat16, arithmetic and gradients FP32. All pointers are device pointers.
 */
int pusch_cnn_param_count(void);

/* y [n][2][2][w] (FP32) = CNN(x); acts receives the post-ReLU activations [3][n][32][2][w] (bf16), needed
 * by pusch_cnn_backward. n <= 65535. */
pusch_status pusch_cnn_forward(int n, int w, const void *x_bf16, const void *params_bf16, float *y, void *acts_bf16,
                               void *stream);

/* grad (FP32, param_count values, overwritten) = d/dparams of mean((y - target)^2) for the forward pass
 * that produced y and acts; *loss (if not NULL) = that mean. work: 2 * n * 32 * 2 * w floats of scratch;
 * wflip: param_count bf16 values of scratch. */
pusch_status pusch_cnn_backward(int n, int w, const void *x_bf16, const void *acts_bf16, const void *params_bf16,
                                const float *y, const float *target, float *grad, float *loss, float *work,
                                void *wflip_bf16, void *stream);

/* One Adam step (step >= 1) on the FP32 master parameters; params_bf16 receives their bfloat16 copy. */
pusch_status pusch_cnn_adam(int step, float lr, float beta1, float beta2, float eps, float *params, void *params_bf16,
                            const float *grad, float *m, float *v, void *stream);

/* The denoiser's input: for every (slot, layer l, beam b), grid index (slot * n_layers + l) * n_beams + b,
 * the LS estimate of each DMRS symbol separately (y_j / p_j at the layer's pilots, linearly interpolated
 * as in pusch_chest_ls), divided by its RMS over the grid: grid [grids][2][2][n_sc] bf16, scale [grids]. */
pusch_status pusch_ls_grid(pusch_handle *h, int n_slots, const void *beam, const void *pilots, void *grid_bf16,
                           float *scale, void *stream);

/* Channel estimation with the denoiser: H_hat (layout of pusch_chest_ls) receives, per (slot, layer, beam),
 * the CNN estimate (mean of its two DMRS rows, rescaled), or the plain LS estimate of pusch_chest_ls when
 * the CNN explains the layer's pilots worse than plain interpolation would (fallback). On the pilots q of
 * both DMRS symbols, with LS_j[q] = y_j[q] / p_j[q]: r_cnn = mean |LS_j[q] - estimate_j[q]|^2 and
 * r_ref = max(sigma^2, mean |LS_j[q] - (LS_j[q - comb] + LS_j[q + comb]) / 2|^2) (leave-one-out
 * interpolation over the inner pilots); fallback when r_cnn > kappa * r_ref. resid [grids] (optional)
 * receives r_cnn / r_ref, fallback [grids] (optional) 1 where the LS estimate was kept. The first call
 * allocates the handle's CNN workspace for max_slots (max_slots * n_layers * n_beams <= 65535 grids). */
pusch_status pusch_chest_cnn(pusch_handle *h, int n_slots, const void *beam, const void *pilots,
                             const void *params_bf16, float kappa, void *H_hat, float *resid, uint8_t *fallback,
                             void *stream);

/* ------------------------------------------------------------------------------------------------------
 * Ragged multi-cell batches: several cells of different sizes, each with users on their own contiguous
 * subcarrier ranges (PRB allocations) and layer counts, processed by one CUDA graph launch.
 *
 * Per cell, cells[c] gives n_rx, n_fft, n_sc, n_beams, comb, noise_var, loading (its n_layers, port and
 * qam_bits are not used); in_fp16, form, n_sym and dmrs_sym must be equal for all cells. Cells with cp,
 * shift_7p5khz, dmrs_type 1, chol_every > 0 or PUSCH_NOISE_ESTIMATE are refused (PUSCH_ERR_UNSUPPORTED).
 * Users overlap freely: at every subcarrier, all layers of all users whose range covers it are detected
 * jointly (MU-MIMO, Eq. 2 with N_L = those layers). A user's layer l transmits its pilots on the
 * subcarriers a of its range with a % comb == port0 + l; its estimate is interpolated between those pilots
 * only (held constant outside the first/last one).
 *
 * Buffers (device, caller-owned) are the per-cell / per-user arrays concatenated in cell / user order:
 *   time_in : per cell [n_sym][n_rx][n_fft] c16 (or c64)      W      : per cell [n_rx][n_beams] c64
 *   pilots  : per user [n_layers][2][sc_count] c64 (index 0 = sc_start)
 *   x_hat   : per user [n_layers][n_sym-2][sc_count] c64      bits   : same shape, uint8
 * pusch_batch_sizes returns the element counts of the five buffers.
 * status words as for pusch_mmse_detect; status[2] holds the smallest failing cell * 65536 + subcarrier.
 */
typedef struct {
    int cell;        /* index of the user's cell                                              */
    int sc_start;    /* first subcarrier of its contiguous allocation                         */
    int sc_count;    /* number of subcarriers                                                  */
    int n_layers;    /* layers of the user, 1 .. 32                                            */
    int port0;       /* its layers use DMRS ports port0 .. port0 + n_layers - 1 (< comb)       */
    int qam_bits;    /* 2 = QPSK, 4 = 16-QAM                                                    */
} pusch_user_desc;

typedef struct pusch_batch pusch_batch;   /* opaque: descriptor tables, workspace, captured graph */

/* Validates the cells and users (ranges inside the cell, ports inside the comb, at least one pilot of
 * every port inside its user's range, at most min(32, n_beams) layers overlapping anywhere), builds the
 * constant-user-set segments and the device descriptor tables, and allocates the workspace. */
pusch_status pusch_batch_create(pusch_batch **b, const pusch_cell_cfg *cells, int n_cells,
                                const pusch_user_desc *users, int n_users);
pusch_status pusch_batch_destroy(pusch_batch *b);

/* sizes[0..4] = elements of time_in (complex samples), W, pilots, x_hat (complex), bits. */
pusch_status pusch_batch_sizes(const pusch_batch *b, size_t sizes[5]);

/* Runs the whole chain for the batch on `stream`. The first call (and any call with different buffer
 * pointers) captures the chain into a CUDA graph on an internal stream; later calls replay it with
 * cudaGraphLaunch on `stream`. */
pusch_status pusch_batch_run(pusch_batch *b, const void *time_in, const void *W, const void *pilots, void *x_hat,
                             uint8_t *bits, uint32_t *status, void *stream);

/* Autotuning of the batch's launch shapes (arguments as pusch_batch_run; the buffers must hold a valid
 * slot, whose outputs are overwritten). For each key not found in the cache file it times the candidates on
 * `stream` (synchronising it) and keeps the fastest:
 *   "bf form=F n_rx=R n_beams=B n_sc=S"   tensor-core GEMM: K rows per pipeline stage, staged TMA-store
 *                                         output or direct stores (every shape that fits shared memory);
 *   "det form=F class=NL nbmax=B n_data=D" detector of a layer class: 1, 2 or 4 warps per CTA x CTAs per SM
 *                                         (occupancy limit, 1 or 2);
 *   "graph form=F n_cells=C"              parallel graph branches for the cells' chains: 1, 2, 4 or 8.
 * cache_path may be NULL (nothing read or written); otherwise its lines "<key> | <choice>" are read and the
 * newly timed keys appended. *n_timed (if not NULL) receives the number of keys that were timed. The next
 * pusch_batch_run re-captures its graph with the chosen shapes. Shapes change the order of floating-point
 * accumulation only. */
pusch_status pusch_batch_autotune(pusch_batch *b, const void *time_in, const void *W, const void *pilots,
                                  void *x_hat, uint8_t *bits, uint32_t *status, const char *cache_path, void *stream,
                                  int *n_timed);

/* The batch's current launch shapes: out[0] = graph branches; out[1 + 2c], out[2 + 2c] = warps per CTA and
 * CTA-per-SM cap of layer class c (NL = 2 << c, 0 = occupancy limit); then per cell (chunk rows, staged)
 * of the tensor-core GEMM (0 = chosen by the kernel), as far as n_out allows (n_out >= 11). */
pusch_status pusch_batch_tuning(const pusch_batch *b, int *out, int n_out);

/*
 * Autotuning of a single-cell handle's launch shapes (no counterpart in the paper; pusch_batch_autotune is the
 * ragged batch's). Allocates stand-in inputs for max_slots slots (deterministic values: the timings do not
 * depend on them), runs the chain once, and for each key not found in the cache file times the candidates on
 * `stream` (synchronising it) and keeps the fastest:
 *   "slot-fft ..."   FFT CTAs per SM: the kernel's own choice, or at most 3, 2 or 1
 *   "slot-bf ..."    tensor-core beamforming GEMM (mixed and FP8 forms): K rows per pipeline stage and staged
 *                    or direct output stores (every shape that fits shared memory)
 *   "slot-det ..."   detector warps per CTA: 1, 2, 4 or 8, where the tiles fit in shared memory (one estimate
 *                    per slot, 12 data symbols)
 *   "slot-pipe ..."  pusch_set_pipeline chunk count: 1, 2 or 4 (at most max_slots)
 * The choices apply to the handle's later calls; every choice gives bit-identical results (each subcarrier's and
 * each row's arithmetic is the same whatever the launch shape). cache_path may be NULL (nothing read or written);
 * otherwise its lines "<key> | <choice>" are read and the newly timed keys appended. *n_timed (if not NULL)
 * receives the number of keys that were timed. Allocates and frees device memory: not for use inside a stream
 * capture. PUSCH_ERR_ARG for a NULL handle or a cache file that cannot be appended to.
 */
pusch_status pusch_autotune(pusch_handle *h, const char *cache_path, void *stream, int *n_timed);

/*
 * pusch_slot for callers that cannot allocate device memory.
 * The paper has no counterpart of this entry point; it exists for integration. Some callers must not call
 * cudaMalloc: a real-time receiver thread, where the CUDA allocator can synchronise the device and take
 * an unbounded time within a slot deadline; a plug-in whose host framework owns all device memory and
 * hands the library only its input and output buffers; a stateless callback that cannot create and
 * destroy a handle. pusch_slot_noalloc runs the same chain as pusch_slot without a handle and without
 * allocating: its intermediates, the FFT twiddle table and its spare status words live in one static
 * device buffer of PUSCH_NOALLOC_SCRATCH_BYTES that is part of the library (every GPU that loads the
 * library holds it until the process exits). It calls no cudaMalloc or cudaFree.
 *   - The caller still passes every input and output buffer, with the layouts of pusch_slot.
 *   - A call whose cell and n_slots need more than PUSCH_NOALLOC_SCRATCH_BYTES of intermediates returns
 *     PUSCH_ERR_UNSUPPORTED and launches nothing; pusch_last_error() says how many bytes were needed.
 *     (One 16-antenna, 512-point, 300-subcarrier slot needs about 1.3 MB; a 64-antenna, 4096-point,
 *     3276-subcarrier slot does not fit.)
 *   - Every call looks up the buffer's device address in the current context (cudaGetSymbolAddress); the
 *     first call on a device may load the library's device code there, so make that first call before any
 *     stream capture.
 *   - chol_every > 0 (the time-varying estimate) is refused with PUSCH_ERR_UNSUPPORTED: it needs a handle.
 *   - An expired bounded wait is reported as PUSCH_STATUS_TIMEOUT in `status`, as for pusch_slot.
 *   - All calls share the one buffer, which keeps the last call's contents; each call writes everything
 *     it reads from it. Calls that overlap on the GPU (other streams, other host threads) race on it:
 *     serialise them.
 */
#define PUSCH_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
pusch_status pusch_slot_noalloc(const pusch_cell_cfg *cfg, int n_slots, const void *time_in, const void *W,
                                const void *pilots, void *x_hat, uint8_t *bits, uint32_t *status, void *stream);

/*
 * Per-stage device timing of pusch_slot (measurement aid; no counterpart in the paper).
 * pusch_profile_start arms timing for the next max_calls calls of pusch_slot / pusch_slot_host on this
 * handle (at the pipelining set when it is called): each run of the chain records CUDA events on its own
 * stream before the FFT, after the FFT, after beamforming, after the estimate (LS table, noise estimate,
 * interpolation unless the detector interpolates) and after the detector. pusch_profile_read waits for the recorded events, writes the
 * milliseconds of the four stages summed over all timed runs (FFT, beamforming, estimate, detection) to
 * stage_ms[0..3] (n_stages >= 4) and the number of timed calls to *n_calls, and disarms timing. With
 * pipelining a stage's time is that of its kernels while they share the GPU with the other stream's.
 */
pusch_status pusch_profile_start(pusch_handle *h, int max_calls);
pusch_status pusch_profile_read(pusch_handle *h, float *stage_ms, int n_stages, int *n_calls);

/*
 * Synchronous check of finished work (no counterpart in the paper). Waits for `stream`, then reads the
 * status words `status` (DEVICE, 4 words, may be NULL) and, when h is not NULL, the handle's kernel error
 * word, which it clears. Returns
 *   PUSCH_ERR_TIMEOUT  if a bounded device wait expired (status[0] & PUSCH_STATUS_TIMEOUT, or the handle's
 *                      word: a stage call such as pusch_beamform whose wait expired),
 *   PUSCH_ERR_NUMERIC  else if the status words report a pivot failure or a non-finite detected symbol,
 *   PUSCH_OK           otherwise (PUSCH_ERR_CUDA if the stream or the copies fail);
 * pusch_last_error() then describes the failure (counts, first failing index, error bits).
 */
pusch_status pusch_status_check(pusch_handle *h, const uint32_t *status, void *stream);

/*
 * Health check of the failure-detection path (no counterpart in the paper). Launches on `stream` one
 * single-thread kernel that waits, with the bounded wait every waiting kernel of the library uses but with a
 * limit of limit_us microseconds (1 .. 1000000), on a shared-memory barrier that nothing completes. The wait
 * expires and sets bit 4 of h's kernel error word; the kernel issues no copy, MMA or TMEM allocation, so it
 * ends cleanly. Afterwards pusch_status_check(h, ...) returns PUSCH_ERR_TIMEOUT, and the next pusch_slot or
 * pusch_mmse_detect on h reports PUSCH_STATUS_TIMEOUT in its status words. PUSCH_ERR_ARG for a NULL handle or
 * a limit out of range.
 */
pusch_status pusch_selftest_wait(pusch_handle *h, unsigned limit_us, void *stream);

/* Message of the last non-OK status returned on this thread ("" if none). */
const char *pusch_last_error(void);

/* Library version string. */
const char *pusch_version(void);

#ifdef __cplusplus
}
#endif

#endif /* PUSCH_H */
