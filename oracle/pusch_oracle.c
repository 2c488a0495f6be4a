/*
 * pusch_oracle.c -- plain, slow, FP64 CPU oracle of the PUSCH receive hot path of
 * "Efficient Parallelization of 5G-PUSCH on a Scalable RISC-V Many-core Processor" (arXiv 2210.09196).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load this library. The CUDA path shares no code, header, table or helper with it.
 *
 * Every function writes out the definition it follows, in double precision, with no blocking, fusion or
 * reordering beyond the definition:
 *   orc_dft         Section II "OFDM demodulation ... via a FFT": the DFT definition itself.
 *   orc_fft         textbook recursive radix-2 decimation-in-time FFT (pinned against orc_dft).
 *   orc_ofdm_demod  Section II: one FFT per antenna and OFDM symbol, keep the N_SC active bins.
 *   orc_gold, orc_dmrs_cinit, orc_dmrs_type1_pilots, orc_chest_ls_type1, orc_noise_est_type1  3GPP type-1
 *                   DMRS (TS 38.211 5.2.1,
 *                   6.4.1.1): Gold sequence, pilot mapping with frequency OCC, and the LS estimate with OCC
 *                   despreading over each CDM pair (the paper's element-wise division, then the pair mean).
 *   orc_cp_len, orc_slot_len, orc_ofdm_demod_cp  the same on a slot with NR normal cyclic prefixes and the
 *                   optional 7.5 kHz shift (TS 38.211 5.3.1, 5.4; not in the paper, which starts after them).
 *   orc_beamform    Section II: "a MMM with known coefficients", y = W^H x per subcarrier and symbol.
 *   orc_chest_ls    Section II: LS estimate = element-wise division of the received pilot REs by the
 *                   pilots (block-type pilots on whole OFDM symbols), averaged over the two DMRS
 *                   symbols, then linear interpolation between a layer's pilot subcarriers.
 *   orc_gram        Eq. 2: G = H^H H + sigma^2 I.
 *   orc_cholesky    Section V-C: Cholesky-Crout, L computed column by column, G = L L^H.
 *   orc_mmse        Eq. 2 via Section II's Cholesky + two triangular solves, per data symbol and
 *                   subcarrier (the paper's accounting in Table I).
 *   orc_mmse_active Eq. 2 at each subcarrier over the layers active there (users sharing a subcarrier
 *                   are detected jointly).
 *   orc_demap       Gray hard decisions of 3GPP TS 38.211 5.1.3/5.1.4 (QPSK/16-QAM).
 *   orc_op_counts   Table I complex-MAC model.
 *   orc_noise_est   Section II "NE": noise variance from the pilot residual y - H_hat p.
 *   orc_chest_ls_sym, orc_mmse_tv  the estimate of one DMRS symbol, and Eq. 2 with the estimate interpolated
 *                   in time and factorised every K data symbols (Section VI's schedule).
 *   orc_e4m3_*,     the FP8 precision form of the beamforming step (not in the paper; the form this
 *   orc_beamform_fp8  project adds): E4M3 rounding, power-of-two block scales, and the block-scaled
 *                   product y = W^H x of the dequantised operands.
 *
 * Layouts (complex values interleaved re,im; C99 double complex):
 *   time  [n_sym][n_rx][n_fft]     freq [n_sym][n_rx][n_sc]     beam [n_sym][n_sc][n_beams]
 *   W     [n_rx][n_beams]          pilots [n_layers][2][n_sc]   H [n_sc][n_layers][n_beams]
 *   xhat  [n_layers][n_data][n_sc] bits [n_layers][n_data][n_sc] (bit j of the byte = b_j)
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

static const double ORC_PI = 3.14159265358979323846264338327950288;

/* ---------------------------------------------------------------- FFT ---- */

/* X[k] = sum_n x[n] exp(-2 pi i k n / N): the definition, O(N^2). */
void orc_dft(const cplx *x, int n, cplx *X)
{
    for (int k = 0; k < n; ++k) {
        cplx acc = 0;
        for (int t = 0; t < n; ++t) {
            /* reduce k*t mod n first so the angle stays small and exact in double */
            long long kt = ((long long)k * t) % n;
            acc += x[t] * cexp(-2.0 * I * ORC_PI * (double)kt / (double)n);
        }
        X[k] = acc;
    }
}

/* Textbook recursive radix-2 DIT: X[k] = E[k] + w^k O[k], X[k + N/2] = E[k] - w^k O[k]. */
static void fft_rec(const cplx *x, int stride, int n, cplx *out)
{
    if (n == 1) {
        out[0] = x[0];
        return;
    }
    int h = n / 2;
    fft_rec(x, 2 * stride, h, out);              /* even samples -> out[0, h)  */
    fft_rec(x + stride, 2 * stride, h, out + h); /* odd samples  -> out[h, n)  */
    for (int k = 0; k < h; ++k) {
        cplx e = out[k];
        cplx o = out[k + h] * cexp(-2.0 * I * ORC_PI * (double)k / (double)n);
        out[k] = e + o;
        out[k + h] = e - o;
    }
}

/* Returns 0, or -1 if n is not a power of two. */
int orc_fft(const cplx *x, int n, cplx *X)
{
    if (n <= 0 || (n & (n - 1)) != 0) return -1;
    fft_rec(x, 1, n, X);
    return 0;
}

/* FFT bin of active subcarrier a: (a - n_sc/2) mod n_fft (centred band, DC included). */
static int active_bin(int a, int n_sc, int n_fft)
{
    int b = a - n_sc / 2;
    b %= n_fft;
    if (b < 0) b += n_fft;
    return b;
}

/* One FFT per (symbol, antenna) listed in `pairs` (pairs[2i] = symbol, pairs[2i+1] = antenna), or all
 * n_sym*n_rx pairs when pairs == NULL. Only the listed rows of freq are written. */
int orc_ofdm_demod(const cplx *time, int n_sym, int n_rx, int n_fft, int n_sc,
                   const int *pairs, int n_pairs, cplx *freq)
{
    if (n_sc > n_fft || n_sc < 0) return -1;
    cplx *X = malloc(sizeof(cplx) * (size_t)n_fft);
    if (!X) return -2;
    int total = pairs ? n_pairs : n_sym * n_rx;
    int rc = 0;
    for (int i = 0; i < total && rc == 0; ++i) {
        int s = pairs ? pairs[2 * i] : i / n_rx;
        int r = pairs ? pairs[2 * i + 1] : i % n_rx;
        const cplx *x = time + ((size_t)s * n_rx + r) * n_fft;
        rc = orc_fft(x, n_fft, X);
        cplx *f = freq + ((size_t)s * n_rx + r) * n_sc;
        for (int a = 0; a < n_sc; ++a) f[a] = X[active_bin(a, n_sc, n_fft)];
    }
    free(X);
    return rc;
}

/* Cyclic-prefix length in samples of symbol `sym` of a 14-symbol slot at 30 kHz subcarrier spacing with normal
 * cyclic prefix (TS 38.211 5.3.1, mu = 1): 144 kappa 2^-mu T_c, plus 16 kappa T_c on the first symbol of every
 * half subframe (symbol 0 of each slot), kappa = 64. One sample of an n_fft = 4096 transform lasts 16 T_c, so
 * that is 288 and 352 samples, scaled by n_fft / 4096 (an integer for n_fft >= 128). */
int orc_cp_len(int n_fft, int sym)
{
    return (sym == 0 ? 352 : 288) * n_fft / 4096;
}

/* Samples of one antenna's slot with cyclic prefixes: sum over the symbols of cp + n_fft. */
long long orc_slot_len(int n_sym, int n_fft)
{
    long long t = 0;
    for (int s = 0; s < n_sym; ++s) t += orc_cp_len(n_fft, s) + n_fft;
    return t;
}

/* OFDM demodulation of a slot given as one sample stream per antenna, stream [n_rx][slot_len]: symbol s starts
 * after the earlier symbols (each cp + n_fft samples) and its cp_s prefix samples are dropped. With shift != 0 the
 * transmitter moved the spectrum up by 7.5 kHz, a quarter of the 30 kHz spacing, with the phase reference at the
 * start of each symbol's useful part (TS 38.211 5.4): sample n of the useful part is multiplied by
 * exp(-2 pi i n / (4 n_fft)) before the FFT. Then as orc_ofdm_demod: freq [n_sym][n_rx][n_sc]. */
int orc_ofdm_demod_cp(const cplx *stream, int n_sym, int n_rx, int n_fft, int n_sc, int shift, cplx *freq)
{
    if (n_sc > n_fft || n_sc < 0 || n_fft < 128) return -1;
    const long long slot_len = orc_slot_len(n_sym, n_fft);
    cplx *x = malloc(sizeof(cplx) * (size_t)n_fft);
    cplx *X = malloc(sizeof(cplx) * (size_t)n_fft);
    if (!x || !X) {
        free(x);
        free(X);
        return -2;
    }
    int rc = 0;
    long long start = 0;
    for (int s = 0; s < n_sym && rc == 0; ++s) {
        start += orc_cp_len(n_fft, s);
        for (int r = 0; r < n_rx && rc == 0; ++r) {
            const cplx *u = stream + (size_t)r * slot_len + start;
            for (int n = 0; n < n_fft; ++n)
                x[n] = shift ? u[n] * cexp(-2.0 * I * ORC_PI * (double)n / (4.0 * (double)n_fft)) : u[n];
            rc = orc_fft(x, n_fft, X);
            cplx *f = freq + ((size_t)s * n_rx + r) * n_sc;
            for (int a = 0; a < n_sc; ++a) f[a] = X[active_bin(a, n_sc, n_fft)];
        }
        start += n_fft;
    }
    free(x);
    free(X);
    return rc;
}

/* ------------------------------------------------- 3GPP DMRS (type 1) ---- */

/* Pseudo-random sequence of TS 38.211 5.2.1: c(n) = x1(n + 1600) + x2(n + 1600) mod 2 with
 * x1(n + 31) = x1(n + 3) + x1(n), x2(n + 31) = x2(n + 3) + x2(n + 2) + x2(n + 1) + x2(n) (mod 2),
 * x1(0) = 1, x1(1..30) = 0, and x2(i) = bit i of c_init. Bit by bit, as defined. */
int orc_gold(uint32_t c_init, int len, uint8_t *c)
{
    const int total = 1600 + len + 31;
    uint8_t *x1 = calloc((size_t)total, 1), *x2 = calloc((size_t)total, 1);
    if (!x1 || !x2) {
        free(x1);
        free(x2);
        return -2;
    }
    x1[0] = 1;
    for (int i = 0; i < 31; ++i) x2[i] = (uint8_t)((c_init >> i) & 1u);
    for (int n = 0; n + 31 < total; ++n) {
        x1[n + 31] = x1[n + 3] ^ x1[n];
        x2[n + 31] = x2[n + 3] ^ x2[n + 2] ^ x2[n + 1] ^ x2[n];
    }
    for (int n = 0; n < len; ++n) c[n] = x1[n + 1600] ^ x2[n + 1600];
    free(x1);
    free(x2);
    return 0;
}

/* c_init of the PUSCH DMRS with transform precoding disabled (TS 38.211 6.4.1.1.1.1):
 * (2^17 (14 slot + sym + 1)(2 N_ID + 1) + 2 N_ID + n_SCID) mod 2^31, slot = slot number in the frame. */
uint32_t orc_dmrs_cinit(int n_id, int n_scid, int slot, int sym)
{
    const unsigned long long v = (1ull << 17) * (14ull * (unsigned)slot + (unsigned)sym + 1ull) *
                                     (2ull * (unsigned)n_id + 1ull) + 2ull * (unsigned)n_id + (unsigned)n_scid;
    return (uint32_t)(v % (1ull << 31));
}

/* Type-1 single-symbol DMRS (TS 38.211 6.4.1.1.3): antenna port 1000 + p, p in {0, 1, 2, 3}, uses CDM group
 * Delta = p / 2 on subcarriers k = 4n + 2k' + Delta (k' in {0, 1}) with the value w_f(k') r(2n + k'),
 * w_f = (+1, +1) for p = 0, 2 and (+1, -1) for p = 1, 3, and r(m) = ((1 - 2c(2m)) + i (1 - 2c(2m + 1))) / sqrt 2
 * from the c_init of its OFDM symbol; zero on the other subcarriers. Subcarrier k counts from the first
 * subcarrier of the band. pilots [n_layers][2][n_sc] for the two DMRS symbols dmrs_sym[0..1]. */
int orc_dmrs_type1_pilots(int n_id, int n_scid, int slot, const int *dmrs_sym, int n_layers, const int *ports,
                          int n_sc, cplx *pilots)
{
    uint8_t *c = malloc((size_t)n_sc + 2);
    if (!c) return -2;
    const double a = 1.0 / sqrt(2.0);
    for (int j = 0; j < 2; ++j) {
        int rc = orc_gold(orc_dmrs_cinit(n_id, n_scid, slot, dmrs_sym[j]), n_sc + 2, c);
        if (rc) {
            free(c);
            return rc;
        }
        for (int l = 0; l < n_layers; ++l) {
            const int p = ports[l], delta = p / 2;
            cplx *out = pilots + ((size_t)l * 2 + j) * n_sc;
            for (int k = 0; k < n_sc; ++k) out[k] = 0;
            for (int k = delta; k < n_sc; k += 2) {
                const int kp = ((k - delta) / 2) % 2, m = (k - delta) / 2;  /* k = 4n + 2k' + Delta, m = 2n + k' */
                const double w = (p % 2 == 1 && kp == 1) ? -1.0 : 1.0;
                out[k] = w * a * ((1.0 - 2.0 * c[2 * m]) + I * (1.0 - 2.0 * c[2 * m + 1]));
            }
        }
    }
    free(c);
    return 0;
}

/* LS estimate with type-1 DMRS: for layer l (port p, CDM group Delta = p / 2) and every pair of its group's
 * subcarriers k0 = 4n + Delta, k1 = k0 + 2 inside the band, the despread value 1/2 (y(k0) / p(k0) + y(k1) / p(k1))
 * of each DMRS symbol (the OCC w_f is inside the pilot values, so the other port of the group cancels where the
 * channel is equal on k0 and k1), averaged over the two DMRS symbols and placed at the pair centre k0 + 1; then
 * linear interpolation between the centres and the value held outside the first and last. H [n_sc][n_layers][n_beams]. */
static int chest_ls_type1_weighted(const cplx *beam, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                                   const int *ports, const cplx *pilots, const double *wj, cplx *H);

int orc_chest_ls_type1(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                       const int *ports, const cplx *pilots, cplx *H)
{
    (void)n_sym;
    const double w[2] = {0.5, 0.5};
    return chest_ls_type1_weighted(beam, n_sc, n_beams, dmrs_sym, n_layers, ports, pilots, w, H);
}

/* The same estimate from DMRS symbol j alone (the despread pairs of that symbol, interpolated). */
int orc_chest_ls_type1_sym(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                           const int *ports, const cplx *pilots, int j, cplx *H)
{
    (void)n_sym;
    const double w[2] = {j == 0 ? 1.0 : 0.0, j == 0 ? 0.0 : 1.0};
    return chest_ls_type1_weighted(beam, n_sc, n_beams, dmrs_sym, n_layers, ports, pilots, w, H);
}

/* Despread pairs weighted by wj over the DMRS symbols, then interpolation between the pair centres. */
static int chest_ls_type1_weighted(const cplx *beam, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                                   const int *ports, const cplx *pilots, const double *wj, cplx *H)
{
    for (int l = 0; l < n_layers; ++l) {
        const int delta = ports[l] / 2;
        const int n_pairs = (n_sc - delta - 2) >= 0 ? (n_sc - delta - 2) / 4 + 1 : 0;
        if (n_pairs < 1) return -(l + 1);
        cplx *ls = malloc(sizeof(cplx) * (size_t)n_pairs * n_beams);
        if (!ls) return -2;
        for (int n = 0; n < n_pairs; ++n) {
            const int k0 = 4 * n + delta, k1 = k0 + 2;
            for (int b = 0; b < n_beams; ++b) {
                cplx v = 0;
                for (int j = 0; j < 2; ++j) {
                    const cplx *y = beam + (size_t)dmrs_sym[j] * n_sc * n_beams;
                    const cplx *p = pilots + ((size_t)l * 2 + j) * n_sc;
                    v += wj[j] * 0.5 * (y[(size_t)k0 * n_beams + b] / p[k0] + y[(size_t)k1 * n_beams + b] / p[k1]);
                }
                ls[(size_t)n * n_beams + b] = v;
            }
        }
        const int first = delta + 1, last = 4 * (n_pairs - 1) + delta + 1;
        for (int a = 0; a < n_sc; ++a) {
            int lo, hi;
            if (a <= first) {
                lo = hi = 0;
            } else if (a >= last) {
                lo = hi = n_pairs - 1;
            } else {
                lo = (a - first) / 4;
                hi = lo + 1;
            }
            const int c_lo = first + 4 * lo;
            for (int b = 0; b < n_beams; ++b) {
                cplx h = ls[(size_t)lo * n_beams + b];
                if (hi != lo)
                    h += ((double)(a - c_lo) / 4.0) * (ls[(size_t)hi * n_beams + b] - ls[(size_t)lo * n_beams + b]);
                H[((size_t)a * n_layers + l) * n_beams + b] = h;
            }
        }
        free(ls);
    }
    return 0;
}

/* Noise variance with type-1 DMRS: the two ports of a CDM group share its REs, so on every pair (k0, k0 + 2)
 * of a group with m of the layers' ports (m = 1 or 2) the 4 observations y_j(k) (2 REs x 2 DMRS symbols, per
 * beam) are fitted by the m despread estimates h_l = 1/4 sum_{j,k} y_j(k) / p_{l,j}(k) -- the least-squares fit,
 * the pilot vectors of a group being orthogonal and of unit modulus -- and the residual
 * r_j(k) = y_j(k) - sum_l h_l p_{l,j}(k) keeps 4 - m degrees of freedom:
 *     sigma2 = sum |r|^2 / sum (4 - m)      over groups, pairs and beams (unbiased for white noise). */
double orc_noise_est_type1(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                           const int *ports, const cplx *pilots)
{
    (void)n_sym;
    double sum = 0.0, dof = 0.0;
    for (int delta = 0; delta < 2; ++delta) {
        int ls[4], m = 0;
        for (int l = 0; l < n_layers; ++l)
            if (ports[l] / 2 == delta) ls[m++] = l;
        if (m == 0) continue;
        for (int k0 = delta; k0 + 2 < n_sc; k0 += 4) {
            const int kk[2] = {k0, k0 + 2};
            for (int b = 0; b < n_beams; ++b) {
                cplx h[4];
                for (int u = 0; u < m; ++u) {
                    h[u] = 0;
                    for (int j = 0; j < 2; ++j)
                        for (int t = 0; t < 2; ++t)
                            h[u] += beam[((size_t)dmrs_sym[j] * n_sc + kk[t]) * n_beams + b] /
                                    pilots[((size_t)ls[u] * 2 + j) * n_sc + kk[t]];
                    h[u] *= 0.25;
                }
                for (int j = 0; j < 2; ++j)
                    for (int t = 0; t < 2; ++t) {
                        cplx e = beam[((size_t)dmrs_sym[j] * n_sc + kk[t]) * n_beams + b];
                        for (int u = 0; u < m; ++u) e -= h[u] * pilots[((size_t)ls[u] * 2 + j) * n_sc + kk[t]];
                        sum += creal(e) * creal(e) + cimag(e) * cimag(e);
                    }
                dof += 4 - m;
            }
        }
    }
    return dof > 0 ? sum / dof : -1.0;
}

/* ---------------------------------------------------------- beamforming ---- */

/* beam[s][a][b] = sum_r conj(W[r][b]) * freq[s][r][a]   (y = W^H x, a triple loop). */
void orc_beamform(const cplx *freq, const cplx *W, int n_sym, int n_rx, int n_sc, int n_beams,
                  cplx *beam)
{
    for (int s = 0; s < n_sym; ++s)
        for (int a = 0; a < n_sc; ++a)
            for (int b = 0; b < n_beams; ++b) {
                cplx acc = 0;
                for (int r = 0; r < n_rx; ++r)
                    acc += conj(W[(size_t)r * n_beams + b]) * freq[((size_t)s * n_rx + r) * n_sc + a];
                beam[((size_t)s * n_sc + a) * n_beams + b] = acc;
            }
}

/* ------------------------------------------------------ LS channel estimate ---- */

/*
 * Layer l occupies subcarriers [sc_start[l], sc_start[l] + sc_count[l]) and carries its pilots on the
 * subcarriers a of that range with a % comb == port[l]. For each of those pilot subcarriers q:
 *     LS[q][b] = 1/2 * sum_{j in {0,1}} beam[dmrs_sym[j]][q][b] / pilots[l][j][q]
 * and for each subcarrier a of the range:
 *     a at or before the first pilot   -> LS[first]
 *     a at or after the last pilot     -> LS[last]
 *     otherwise, with lo <= a < hi the neighbouring pilots:
 *         H = LS[lo] + (a - lo) / (hi - lo) * (LS[hi] - LS[lo])
 * Subcarriers outside the range are left untouched.
 * Returns 0, or -(l+1) when layer l has no pilot in its range.
 */
/* LS estimate with DMRS-symbol weights wj[2]: at a pilot q, sum_j wj[j] y_j[q] / p_j[q], then frequency
 * interpolation. wj = {1/2, 1/2} is the two-symbol mean (orc_chest_ls); {1, 0} and {0, 1} are the estimates of
 * one DMRS symbol alone (orc_chest_ls_sym). */
static int chest_ls_weighted(const cplx *beam, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                             const cplx *pilots, const int *port, int comb, const int *sc_start, const int *sc_count,
                             const double *wj, cplx *H)
{
    for (int l = 0; l < n_layers; ++l) {
        int a0 = sc_start[l], a1 = sc_start[l] + sc_count[l];
        int first = -1, last = -1;
        for (int a = a0; a < a1; ++a)
            if (a % comb == port[l]) {
                if (first < 0) first = a;
                last = a;
            }
        if (first < 0) return -(l + 1);
        for (int a = a0; a < a1; ++a) {
            int lo, hi;
            if (a <= first) {
                lo = hi = first;
            } else if (a >= last) {
                lo = hi = last;
            } else {
                lo = a;
                while (lo % comb != port[l]) --lo;
                hi = lo + comb;
                if (lo == a) hi = lo;
            }
            for (int b = 0; b < n_beams; ++b) {
                cplx ls_lo = 0, ls_hi = 0;
                for (int j = 0; j < 2; ++j) {
                    const cplx *y = beam + (size_t)dmrs_sym[j] * n_sc * n_beams;
                    const cplx *p = pilots + ((size_t)l * 2 + j) * n_sc;
                    ls_lo += wj[j] * y[(size_t)lo * n_beams + b] / p[lo];
                    ls_hi += wj[j] * y[(size_t)hi * n_beams + b] / p[hi];
                }
                cplx h = ls_lo;
                if (hi != lo) h = ls_lo + ((double)(a - lo) / (double)(hi - lo)) * (ls_hi - ls_lo);
                H[((size_t)a * n_layers + l) * n_beams + b] = h;
            }
        }
    }
    return 0;
}

int orc_chest_ls(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym,
                 int n_layers, const cplx *pilots, const int *port, int comb,
                 const int *sc_start, const int *sc_count, cplx *H)
{
    (void)n_sym;
    const double w[2] = {0.5, 0.5};
    return chest_ls_weighted(beam, n_sc, n_beams, dmrs_sym, n_layers, pilots, port, comb, sc_start, sc_count, w, H);
}

/* The LS estimate of DMRS symbol j (0 or 1) alone: y_j[q] / p_j[q] at the pilots, frequency interpolation. */
int orc_chest_ls_sym(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                     const cplx *pilots, const int *port, int comb, int j, cplx *H)
{
    (void)n_sym;
    const double w[2] = {j == 0 ? 1.0 : 0.0, j == 0 ? 0.0 : 1.0};
    int *st = malloc(sizeof(int) * (size_t)n_layers), *ct = malloc(sizeof(int) * (size_t)n_layers);
    for (int l = 0; l < n_layers; ++l) {
        st[l] = 0;
        ct[l] = n_sc;
    }
    int rc = chest_ls_weighted(beam, n_sc, n_beams, dmrs_sym, n_layers, pilots, port, comb, st, ct, w, H);
    free(st);
    free(ct);
    return rc;
}

/* Noise-variance estimate, Section II "NE": the autocorrelation (mean squared magnitude) of the difference
 * between the received pilot symbols and the output expected from the estimated channel and the pilots.
 * At every subcarrier q that carries a pilot of some layer (q % comb == port[l]) and each DMRS symbol j:
 *     e_j[q] = y_j[q] - sum over the layers l with a pilot at q of H_hat[q][l] p_{l,j}[q]    (all beams)
 * with H_hat from orc_chest_ls (over the whole band), and
 *     sigma2_hat = 2 * mean |e_j[q][b]|^2 over (j, q, b).
 * The factor 2 undoes the two-symbol average: at its own pilot H_hat = (LS_0 + LS_1) / 2, so
 * e_j = p_j (LS_j - LS_{1-j}) / 2 and E|e_j|^2 = sigma^2 / 2 for unit-modulus pilots and a channel that does
 * not change between the DMRS symbols (distinct ports: one layer per pilot subcarrier). Returns -1 when no
 * subcarrier carries a pilot. */
double orc_noise_est(const cplx *beam, int n_sym, int n_sc, int n_beams, const int *dmrs_sym, int n_layers,
                     const cplx *pilots, const int *port, int comb)
{
    cplx *H = malloc(sizeof(cplx) * (size_t)n_sc * n_layers * n_beams);
    int *st = malloc(sizeof(int) * (size_t)n_layers), *ct = malloc(sizeof(int) * (size_t)n_layers);
    for (int l = 0; l < n_layers; ++l) {
        st[l] = 0;
        ct[l] = n_sc;
    }
    double sum = 0.0;
    long long count = 0;
    if (orc_chest_ls(beam, n_sym, n_sc, n_beams, dmrs_sym, n_layers, pilots, port, comb, st, ct, H) == 0) {
        for (int q = 0; q < n_sc; ++q) {
            int any = 0;
            for (int l = 0; l < n_layers; ++l) any |= (q % comb == port[l]);
            if (!any) continue;
            for (int j = 0; j < 2; ++j) {
                const cplx *y = beam + (size_t)dmrs_sym[j] * n_sc * n_beams;
                for (int b = 0; b < n_beams; ++b) {
                    cplx e = y[(size_t)q * n_beams + b];
                    for (int l = 0; l < n_layers; ++l)
                        if (q % comb == port[l])
                            e -= H[((size_t)q * n_layers + l) * n_beams + b] * pilots[((size_t)l * 2 + j) * n_sc + q];
                    sum += creal(e) * creal(e) + cimag(e) * cimag(e);
                    ++count;
                }
            }
        }
    }
    free(H);
    free(st);
    free(ct);
    return count ? 2.0 * sum / (double)count : -1.0;
}

/* --------------------------------------------------------------- MMSE ---- */

/* G = H^H H + load * I for one subcarrier; Hs is stored [n_layers][n_beams] (row l = column l of H). */
void orc_gram(const cplx *Hs, int n_layers, int n_beams, double load, cplx *G)
{
    for (int i = 0; i < n_layers; ++i)
        for (int j = 0; j < n_layers; ++j) {
            cplx acc = 0;
            for (int b = 0; b < n_beams; ++b)
                acc += conj(Hs[(size_t)i * n_beams + b]) * Hs[(size_t)j * n_beams + b];
            G[(size_t)i * n_layers + j] = acc + (i == j ? load : 0.0);
        }
}

/*
 * Cholesky-Crout, column by column: for j = 0..n-1
 *     L[j][j] = sqrt(G[j][j] - sum_{k<j} |L[j][k]|^2)
 *     L[i][j] = (G[i][j] - sum_{k<j} L[i][k] conj(L[j][k])) / L[j][j],   i > j
 * Only the lower triangle of G is read; the strict upper triangle of L is set to zero.
 * Returns 0, or j+1 when the j-th pivot is not a positive finite number.
 */
int orc_cholesky(const cplx *G, int n, cplx *L)
{
    for (int i = 0; i < n * n; ++i) L[i] = 0;
    for (int j = 0; j < n; ++j) {
        double d = creal(G[(size_t)j * n + j]);
        for (int k = 0; k < j; ++k) {
            cplx v = L[(size_t)j * n + k];
            d -= creal(v) * creal(v) + cimag(v) * cimag(v);
        }
        if (!(d > 0.0) || !isfinite(d)) return j + 1;
        double ljj = sqrt(d);
        L[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            cplx acc = G[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) acc -= L[(size_t)i * n + k] * conj(L[(size_t)j * n + k]);
            L[(size_t)i * n + j] = acc / ljj;
        }
    }
    return 0;
}

/* Solve L z = r (forward) then L^H x = z (back); L lower triangular with real positive diagonal. */
void orc_chol_solve(const cplx *L, int n, const cplx *r, cplx *x)
{
    cplx *z = malloc(sizeof(cplx) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        cplx acc = r[i];
        for (int k = 0; k < i; ++k) acc -= L[(size_t)i * n + k] * z[k];
        z[i] = acc / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
        cplx acc = z[i];
        for (int k = i + 1; k < n; ++k) acc -= conj(L[(size_t)k * n + i]) * x[k];
        x[i] = acc / conj(L[(size_t)i * n + i]);
    }
    free(z);
}

/*
 * Eq. 2 for every listed subcarrier (sc_list, or all when NULL) and every data symbol d:
 *     G = H^H H + (noise_var + loading) I ;  G = L L^H ;  L z = H^H y ;  L^H x = z
 * with y = beam[data_sym[d]][a][:]. The Gram and its factor are formed anew for each data symbol, as the
 * paper counts them (Table I: per subcarrier and per data symbol).
 * xhat[l][d][a] receives x_l. Returns the number of (subcarrier, symbol) pairs whose factorisation failed
 * (their xhat entries are set to 0).
 */
int orc_mmse(const cplx *H, const cplx *beam, int n_sc, int n_beams, int n_layers,
             const int *data_sym, int n_data, double noise_var, double loading,
             const int *sc_list, int n_list, cplx *xhat)
{
    int nl = n_layers;
    cplx *G = malloc(sizeof(cplx) * (size_t)nl * nl);
    cplx *L = malloc(sizeof(cplx) * (size_t)nl * nl);
    cplx *r = malloc(sizeof(cplx) * (size_t)nl);
    cplx *x = malloc(sizeof(cplx) * (size_t)nl);
    int fails = 0;
    int total = sc_list ? n_list : n_sc;
    for (int ii = 0; ii < total; ++ii) {
        int a = sc_list ? sc_list[ii] : ii;
        const cplx *Hs = H + (size_t)a * nl * n_beams;
        for (int d = 0; d < n_data; ++d) {
            const cplx *y = beam + ((size_t)data_sym[d] * n_sc + a) * n_beams;
            orc_gram(Hs, nl, n_beams, noise_var + loading, G);
            int st = orc_cholesky(G, nl, L);
            if (st != 0) {
                ++fails;
                for (int l = 0; l < nl; ++l) xhat[((size_t)l * n_data + d) * n_sc + a] = 0;
                continue;
            }
            for (int i = 0; i < nl; ++i) {
                cplx acc = 0;
                for (int b = 0; b < n_beams; ++b) acc += conj(Hs[(size_t)i * n_beams + b]) * y[b];
                r[i] = acc;
            }
            orc_chol_solve(L, nl, r, x);
            for (int l = 0; l < nl; ++l) xhat[((size_t)l * n_data + d) * n_sc + a] = x[l];
        }
    }
    free(G);
    free(L);
    free(r);
    free(x);
    return fails;
}

/*
 * Eq. 2 with a time-varying estimate and the factorisation scheduled every K data symbols (Section VI: one
 * Cholesky per data symbol in Table I's accounting, or every 4 data symbols). H0, H1: the estimates of the two
 * DMRS symbols s0 = dmrs_sym[0], s1 = dmrs_sym[1] alone (orc_chest_ls_sym). Data symbol s has the estimate
 * H(s) = H0 + (s - s0) / (s1 - s0) (H1 - H0) (linear in time, extrapolated outside [s0, s1]). The data symbols,
 * in increasing order, are taken in groups of K (the last group may be shorter); a group uses H at the mean
 * time of its symbols for all of them, one Gram and one factorisation per subcarrier. K = 1: per data symbol.
 * xhat [n_layers][n_data][n_sc] as orc_mmse; returns the number of failed factorisations.
 */
int orc_mmse_tv(const cplx *H0, const cplx *H1, const cplx *beam, int n_sc, int n_beams, int n_layers,
                const int *dmrs_sym, const int *data_sym, int n_data, double noise_var, double loading, int K,
                cplx *xhat)
{
    size_t nh = (size_t)n_sc * n_layers * n_beams;
    cplx *Hg = malloc(sizeof(cplx) * nh);
    cplx *xg = malloc(sizeof(cplx) * (size_t)n_layers * K * n_sc);
    int fails = 0;
    double span = (double)(dmrs_sym[1] - dmrs_sym[0]);
    for (int g0 = 0; g0 < n_data; g0 += K) {
        int ng = n_data - g0 < K ? n_data - g0 : K;
        double t = 0.0;
        for (int d = g0; d < g0 + ng; ++d) t += (double)(data_sym[d] - dmrs_sym[0]) / span;
        t /= ng;
        for (size_t e = 0; e < nh; ++e) Hg[e] = H0[e] + t * (H1[e] - H0[e]);
        fails += orc_mmse(Hg, beam, n_sc, n_beams, n_layers, data_sym + g0, ng, noise_var, loading, NULL, 0, xg);
        for (int l = 0; l < n_layers; ++l)
            for (int d = 0; d < ng; ++d)
                for (int a = 0; a < n_sc; ++a)
                    xhat[((size_t)l * n_data + g0 + d) * n_sc + a] = xg[((size_t)l * ng + d) * n_sc + a];
    }
    free(Hg);
    free(xg);
    return fails;
}

/*
 * MU-MIMO form of Eq. 2: at every subcarrier a, the layers l with active[a][l] != 0 (all users covering a)
 * are detected jointly, G = H_A^H H_A + (noise_var + loading) I over those layers only, formed and
 * factored anew for each data symbol. xhat[l][d][a] is written for the active layers only.
 * Returns the number of (subcarrier, symbol) pairs whose factorisation failed.
 */
int orc_mmse_active(const cplx *H, const cplx *beam, const uint8_t *active, int n_sc, int n_beams, int n_layers,
                    const int *data_sym, int n_data, double noise_var, double loading, cplx *xhat)
{
    int *idx = malloc(sizeof(int) * (size_t)n_layers);
    cplx *Hs = malloc(sizeof(cplx) * (size_t)n_layers * n_beams);
    cplx *G = malloc(sizeof(cplx) * (size_t)n_layers * n_layers);
    cplx *L = malloc(sizeof(cplx) * (size_t)n_layers * n_layers);
    cplx *r = malloc(sizeof(cplx) * (size_t)n_layers);
    cplx *x = malloc(sizeof(cplx) * (size_t)n_layers);
    int fails = 0;
    for (int a = 0; a < n_sc; ++a) {
        int m = 0;
        for (int l = 0; l < n_layers; ++l)
            if (active[(size_t)a * n_layers + l]) idx[m++] = l;
        if (m == 0) continue;
        for (int j = 0; j < m; ++j)
            for (int b = 0; b < n_beams; ++b)
                Hs[(size_t)j * n_beams + b] = H[((size_t)a * n_layers + idx[j]) * n_beams + b];
        for (int d = 0; d < n_data; ++d) {
            const cplx *y = beam + ((size_t)data_sym[d] * n_sc + a) * n_beams;
            orc_gram(Hs, m, n_beams, noise_var + loading, G);
            if (orc_cholesky(G, m, L) != 0) {
                ++fails;
                for (int j = 0; j < m; ++j) xhat[((size_t)idx[j] * n_data + d) * n_sc + a] = 0;
                continue;
            }
            for (int i = 0; i < m; ++i) {
                cplx acc = 0;
                for (int b = 0; b < n_beams; ++b) acc += conj(Hs[(size_t)i * n_beams + b]) * y[b];
                r[i] = acc;
            }
            orc_chol_solve(L, m, r, x);
            for (int j = 0; j < m; ++j) xhat[((size_t)idx[j] * n_data + d) * n_sc + a] = x[j];
        }
    }
    free(idx);
    free(Hs);
    free(G);
    free(L);
    free(r);
    free(x);
    return fails;
}

/* ------------------------------------------------------------- demapper ---- */

/*
 * Gray hard decisions (3GPP TS 38.211 5.1.3 / 5.1.4), tie -> bit 0:
 *   QPSK : b0 = Re < 0, b1 = Im < 0
 *   16QAM: b0 = Re < 0, b1 = Im < 0, b2 = |Re| > 2/sqrt(10), b3 = |Im| > 2/sqrt(10)
 * With f32 != 0 the comparisons are taken in single precision (component and threshold rounded to
 * float), so that decisions can be compared bit for bit with a single-precision detector.
 */
void orc_demap(const cplx *x, long long n, int qam_bits, int f32, uint8_t *bits)
{
    const double thr = 2.0 / sqrt(10.0);
    const float thr_f = (float)(2.0 / sqrt(10.0));
    for (long long i = 0; i < n; ++i) {
        double re = creal(x[i]), im = cimag(x[i]);
        uint8_t v = 0;
        if (f32) {
            float rf = (float)re, imf = (float)im;
            v |= (uint8_t)(rf < 0.0f) << 0;
            v |= (uint8_t)(imf < 0.0f) << 1;
            if (qam_bits == 4) {
                v |= (uint8_t)(fabsf(rf) > thr_f) << 2;
                v |= (uint8_t)(fabsf(imf) > thr_f) << 3;
            }
        } else {
            v |= (uint8_t)(re < 0.0) << 0;
            v |= (uint8_t)(im < 0.0) << 1;
            if (qam_bits == 4) {
                v |= (uint8_t)(fabs(re) > thr) << 2;
                v |= (uint8_t)(fabs(im) > thr) << 3;
            }
        }
        bits[i] = v;
    }
}

/* --------------------------------------------------------- complexity ---- */

/*
 * Table I complex-MAC counts (log taken base 2; the MIMO entry read as N_L^3/3 + 2 N_L^2):
 *   out[0] OFDM  N_symb * N_R * N_SC * log2(N_SC)
 *   out[1] BF    N_symb * N_SC * N_R * N_B
 *   out[2] MIMO  N_data * N_SC * (N_L^3/3 + 2 N_L^2)
 *   out[3] CHE   N_pilot * N_SC * N_B * N_L
 *   out[4] NE    N_pilot * N_SC * 2 N_B * N_L
 */
void orc_op_counts(int n_symb, int n_pilot, int n_r, int n_sc, int n_b, int n_l, double *out)
{
    int n_data = n_symb - n_pilot;
    out[0] = (double)n_symb * n_r * n_sc * log2((double)n_sc);
    out[1] = (double)n_symb * n_sc * n_r * n_b;
    out[2] = (double)n_data * n_sc * ((double)n_l * n_l * n_l / 3.0 + 2.0 * n_l * n_l);
    out[3] = (double)n_pilot * n_sc * n_b * n_l;
    out[4] = (double)n_pilot * n_sc * 2.0 * n_b * n_l;
}

/* ----------------------------------------------------------- full slot ---- */

/*
 * The chain of Fig. 1 for one slot: OFDM demodulation -> beamforming -> LS channel estimation on the
 * DMRS symbols -> MMSE detection of the data symbols -> hard decisions.
 * Every layer spans the whole band [0, n_sc). Returns the number of failed factorisations, or < 0 on
 * an argument error.
 */
int orc_slot(const cplx *time, int n_sym, int n_rx, int n_fft, int n_sc, const cplx *W, int n_beams,
             const int *dmrs_sym, int n_layers, const cplx *pilots, const int *port, int comb,
             int qam_bits, double noise_var, double loading, cplx *xhat, uint8_t *bits)
{
    int n_data = 0;
    int data_sym[64];
    for (int s = 0; s < n_sym && n_data < 64; ++s)
        if (s != dmrs_sym[0] && s != dmrs_sym[1]) data_sym[n_data++] = s;

    cplx *freq = malloc(sizeof(cplx) * (size_t)n_sym * n_rx * n_sc);
    cplx *beam = malloc(sizeof(cplx) * (size_t)n_sym * n_sc * n_beams);
    cplx *H = malloc(sizeof(cplx) * (size_t)n_sc * n_layers * n_beams);
    int *start = malloc(sizeof(int) * (size_t)n_layers);
    int *count = malloc(sizeof(int) * (size_t)n_layers);
    int rc = 0;
    if (!freq || !beam || !H || !start || !count) {
        rc = -2;
        goto done;
    }
    for (int l = 0; l < n_layers; ++l) {
        start[l] = 0;
        count[l] = n_sc;
    }
    rc = orc_ofdm_demod(time, n_sym, n_rx, n_fft, n_sc, NULL, 0, freq);
    if (rc) goto done;
    orc_beamform(freq, W, n_sym, n_rx, n_sc, n_beams, beam);
    rc = orc_chest_ls(beam, n_sym, n_sc, n_beams, dmrs_sym, n_layers, pilots, port, comb, start, count, H);
    if (rc) goto done;
    rc = orc_mmse(H, beam, n_sc, n_beams, n_layers, data_sym, n_data, noise_var, loading, NULL, 0, xhat);
    orc_demap(xhat, (long long)n_layers * n_data * n_sc, qam_bits, 0, bits);
done:
    free(freq);
    free(beam);
    free(H);
    free(start);
    free(count);
    return rc;
}

/* ------------------------------------------------------ learned denoiser (CNN) ---- */

/*
 * The channel-estimate denoiser: four 3x3 same-padded convolutions 2 -> 32 -> 32 -> 32 -> 2 with ReLU after
 * the first three and the input added to the output (residual). Tensors are [n][c][2][w] (n grids, c
 * channels, the 2 DMRS symbols as rows, w subcarriers); zero padding outside the grid.
 *   conv:  out[n][co][h][x] = b[co] + sum_{ci, dh, dx} W[co][ci][dh][dx] in[n][ci][h + dh - 1][x + (dx - 1) d]
 * with the kernel dilated along the subcarriers by d = 1, 8, 16, 1 for the four layers (receptive field of
 * +-26 subcarriers, several pilot spacings of a comb of 8 or 16).
 * Parameters are packed layer by layer as W (co, ci, 3, 3) then b (co).
 * bf16 != 0 rounds weights, biases, the input and every stored activation to bfloat16 (round to nearest
 * even), at the points where a bfloat16 implementation stores them; arithmetic stays double.
 */
static const int CNN_CH[5] = {2, 32, 32, 32, 2};
static const int CNN_DIL[4] = {1, 8, 16, 1};

int orc_cnn_param_count(void)
{
    int n = 0;
    for (int k = 0; k < 4; ++k) n += CNN_CH[k + 1] * CNN_CH[k] * 9 + CNN_CH[k + 1];
    return n;
}

double orc_round_bf16(double v)
{
    float f = (float)v;
    uint32_t u;
    memcpy(&u, &f, 4);
    if ((u & 0x7f800000u) == 0x7f800000u) return v; /* inf / nan unchanged */
    uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return (double)f;
}

static void cnn_conv(const double *in, int n, int cin, int w, const double *W, const double *b, int cout, int dil,
                     double *out)
{
    for (int s = 0; s < n; ++s)
        for (int co = 0; co < cout; ++co)
            for (int h = 0; h < 2; ++h)
                for (int x = 0; x < w; ++x) {
                    double acc = b[co];
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dh = 0; dh < 3; ++dh) {
                            int hh = h + dh - 1;
                            if (hh < 0 || hh > 1) continue;
                            for (int dx = 0; dx < 3; ++dx) {
                                int xx = x + (dx - 1) * dil;
                                if (xx < 0 || xx >= w) continue;
                                acc += W[((co * cin + ci) * 3 + dh) * 3 + dx] *
                                       in[(((size_t)s * cin + ci) * 2 + hh) * w + xx];
                            }
                        }
                    out[(((size_t)s * cout + co) * 2 + h) * w + x] = acc;
                }
}

/* Forward pass. acts (optional) receives the post-ReLU activations of layers 1..3 ([n][32][2][w] each). */
void orc_cnn_forward(const double *params, const double *x, int n, int w, int bf16, double *y, double *acts)
{
    size_t big = (size_t)n * 32 * 2 * w;
    double *p = malloc(sizeof(double) * (size_t)orc_cnn_param_count());
    double *a = malloc(sizeof(double) * big), *z = malloc(sizeof(double) * big);
    double *x0 = malloc(sizeof(double) * (size_t)n * 2 * 2 * w);
    int np = orc_cnn_param_count();
    for (int i = 0; i < np; ++i) p[i] = bf16 ? orc_round_bf16(params[i]) : params[i];
    for (size_t i = 0; i < (size_t)n * 4 * w; ++i) x0[i] = bf16 ? orc_round_bf16(x[i]) : x[i];
    /* in -> z (pre-activation) -> a (post-activation, next input); buffers swapped by copying */
    double *cur = malloc(sizeof(double) * big);
    memcpy(cur, x0, sizeof(double) * (size_t)n * 4 * w);
    int off = 0;
    for (int k = 0; k < 4; ++k) {
        int cin = CNN_CH[k], cout = CNN_CH[k + 1];
        const double *W = p + off, *b = p + off + cout * cin * 9;
        off += cout * cin * 9 + cout;
        cnn_conv(cur, n, cin, w, W, b, cout, CNN_DIL[k], z);
        size_t m = (size_t)n * cout * 2 * w;
        if (k < 3) {
            for (size_t i = 0; i < m; ++i) {
                double v = z[i] > 0 ? z[i] : 0.0;
                a[i] = bf16 ? orc_round_bf16(v) : v;
            }
            if (acts) memcpy(acts + (size_t)k * big, a, sizeof(double) * m);
            memcpy(cur, a, sizeof(double) * m);
        } else {
            for (size_t i = 0; i < m; ++i) y[i] = z[i] + x0[i];
        }
    }
    free(cur);
    free(p);
    free(a);
    free(z);
    free(x0);
}

/*
 * Loss and gradient: L = mean over all output elements of (y - target)^2. grad (same packing as params)
 * receives dL/dparams. Returns L. Same bf16 convention as orc_cnn_forward (the backward pass itself is
 * exact in double, using the rounded forward activations).
 */
double orc_cnn_loss_grad(const double *params, const double *x, const double *target, int n, int w, int bf16,
                         double *grad)
{
    int np = orc_cnn_param_count();
    size_t big = (size_t)n * 32 * 2 * w, small = (size_t)n * 2 * 2 * w;
    double *acts = malloc(sizeof(double) * 3 * big);
    double *y = malloc(sizeof(double) * small);
    double *p = malloc(sizeof(double) * (size_t)np);
    double *x0 = malloc(sizeof(double) * small);
    double *g = malloc(sizeof(double) * big), *gin = malloc(sizeof(double) * big);
    for (int i = 0; i < np; ++i) p[i] = bf16 ? orc_round_bf16(params[i]) : params[i];
    for (size_t i = 0; i < small; ++i) x0[i] = bf16 ? orc_round_bf16(x[i]) : x[i];
    orc_cnn_forward(params, x, n, w, bf16, y, acts);
    double loss = 0;
    for (size_t i = 0; i < small; ++i) {
        double d = y[i] - target[i];
        loss += d * d;
        g[i] = 2.0 * d / (double)small;
    }
    loss /= (double)small;
    int offs[4];
    int off = 0;
    for (int k = 0; k < 4; ++k) {
        offs[k] = off;
        off += CNN_CH[k + 1] * CNN_CH[k] * 9 + CNN_CH[k + 1];
    }
    for (int i = 0; i < np; ++i) grad[i] = 0;
    for (int k = 3; k >= 0; --k) {
        int cin = CNN_CH[k], cout = CNN_CH[k + 1];
        const double *in = k == 0 ? x0 : acts + (size_t)(k - 1) * big;
        const double *W = p + offs[k];
        double *dW = grad + offs[k], *db = grad + offs[k] + cout * cin * 9;
        for (int s = 0; s < n; ++s)
            for (int co = 0; co < cout; ++co)
                for (int h = 0; h < 2; ++h)
                    for (int x = 0; x < w; ++x) {
                        double go = g[(((size_t)s * cout + co) * 2 + h) * w + x];
                        db[co] += go;
                        for (int ci = 0; ci < cin; ++ci)
                            for (int dh = 0; dh < 3; ++dh) {
                                int hh = h + dh - 1;
                                if (hh < 0 || hh > 1) continue;
                                for (int dx = 0; dx < 3; ++dx) {
                                    int xx = x + (dx - 1) * CNN_DIL[k];
                                    if (xx < 0 || xx >= w) continue;
                                    dW[((co * cin + ci) * 3 + dh) * 3 + dx] +=
                                        go * in[(((size_t)s * cin + ci) * 2 + hh) * w + xx];
                                }
                            }
                    }
        if (k == 0) break;
        /* gradient w.r.t. this layer's input, masked by the ReLU of the previous layer */
        for (size_t i = 0; i < (size_t)n * cin * 2 * w; ++i) gin[i] = 0;
        for (int s = 0; s < n; ++s)
            for (int co = 0; co < cout; ++co)
                for (int h = 0; h < 2; ++h)
                    for (int x = 0; x < w; ++x) {
                        double go = g[(((size_t)s * cout + co) * 2 + h) * w + x];
                        for (int ci = 0; ci < cin; ++ci)
                            for (int dh = 0; dh < 3; ++dh) {
                                int hh = h + dh - 1;
                                if (hh < 0 || hh > 1) continue;
                                for (int dx = 0; dx < 3; ++dx) {
                                    int xx = x + (dx - 1) * CNN_DIL[k];
                                    if (xx < 0 || xx >= w) continue;
                                    gin[(((size_t)s * cin + ci) * 2 + hh) * w + xx] +=
                                        go * W[((co * cin + ci) * 3 + dh) * 3 + dx];
                                }
                            }
                    }
        for (size_t i = 0; i < (size_t)n * cin * 2 * w; ++i) g[i] = in[i] > 0 ? gin[i] : 0.0;
    }
    free(acts);
    free(y);
    free(p);
    free(x0);
    free(g);
    free(gin);
    return loss;
}

/* ------------------------------------------------------------------ FP8 E4M3 form ---- */
/*
 * The FP8 form of the beamforming product (Section II "MMM with known coefficients" in a reduced-precision
 * storage format this project adds; the paper has no FP8). Values are stored as E4M3 codes times
 * power-of-two block scales. E4M3: sign, 4 exponent bits (bias 7), 3 mantissa bits, no infinities;
 * normal values (1 + m/8) 2^(e-7) for e = 1..15 (m <= 6 when e = 15, so the largest is 448), subnormal
 * values (m/8) 2^-6.
 */

/* Nearest E4M3 value, ties to the even mantissa; magnitudes of 448 and above give +-448 (saturation);
 * NaN stays NaN. */
double orc_e4m3_round(double v)
{
    if (isnan(v)) return v;
    double a = fabs(v);
    if (a >= 448.0) return copysign(448.0, v);
    int ex;
    frexp(a, &ex);              /* a in [2^(ex-1), 2^ex) */
    int p = ex - 1;             /* binade of a */
    if (p < -6) p = -6;         /* the subnormals share the spacing of the lowest normal binade */
    double q = ldexp(1.0, p - 3);            /* spacing of the 3-bit mantissa grid */
    return copysign(nearbyint(a / q) * q, v);  /* default rounding mode: nearest, ties to even */
}

void orc_e4m3_round_array(const double *x, long long n, double *y)
{
    for (long long i = 0; i < n; ++i) y[i] = orc_e4m3_round(x[i]);
}

/* Exponent of the power-of-two block scale: the smallest integer e >= -126 with amax <= 448 * 2^e;
 * 128 for a non-finite amax. */
int orc_e4m3_block_exp(double amax)
{
    if (!isfinite(amax)) return 128;
    int e = -126;
    while (amax > 448.0 * ldexp(1.0, e)) ++e;
    return e;
}

/* Block quantisation of rows of complex samples: each block of 128 consecutive entries of a row gets
 * e = orc_e4m3_block_exp(largest |Re|, |Im| of the block) and every component becomes
 * orc_e4m3_round(value / 2^e). codes [rows][n] (the E4M3 values, scale not applied), exps
 * [rows][ceil(n / 128)]; a block with a non-finite component gets e = 128 and NaN codes. */
void orc_e4m3_quant_rows(const cplx *x, long long rows, int n, cplx *codes, int *exps)
{
    int n_blk = (n + 127) / 128;
    for (long long r = 0; r < rows; ++r)
        for (int j = 0; j < n_blk; ++j) {
            double amax = 0.0;
            int bad = 0;
            for (int a = 128 * j; a < n && a < 128 * j + 128; ++a) {
                double re = fabs(creal(x[r * n + a])), im = fabs(cimag(x[r * n + a]));
                if (!isfinite(re) || !isfinite(im)) bad = 1;
                if (re > amax) amax = re;
                if (im > amax) amax = im;
            }
            int e = bad ? 128 : orc_e4m3_block_exp(amax);
            exps[r * n_blk + j] = e;
            for (int a = 128 * j; a < n && a < 128 * j + 128; ++a) {
                cplx v = x[r * n + a];
                codes[r * n + a] = bad ? NAN : orc_e4m3_round(ldexp(creal(v), -e)) + I * orc_e4m3_round(ldexp(cimag(v), -e));
            }
        }
}

/* FP8-form beamforming: the block-scaled product of the two quantised operands, summed exactly.
 *   samples: codes [n_sym][n_rx][n_sc] (E4M3 values) with block exponents exps [n_sym][n_rx][ceil(n_sc / 128)];
 *            sample[s][r][a] = codes[s][r][a] * 2^exps[s][r][a / 128];
 *   weights: W [n_rx][n_beams] quantised per (beam, 128 antennas): ew = orc_e4m3_block_exp(largest |Re|, |Im|
 *            of the block), weight[r][b] = E4M3(W[r][b] / 2^ew) * 2^ew;
 *   beam[s][a][b] = sum_r conj(weight[r][b]) sample[s][r][a]   (Section II's Y = W^H X), in double.
 * A block exponent of 128 (a non-finite block) makes every output that block enters NaN. */
void orc_beamform_fp8(const cplx *codes, const int *exps, const cplx *W, int n_sym, int n_rx, int n_sc, int n_beams,
                      cplx *beam)
{
    int n_blk = (n_sc + 127) / 128;
    cplx *wq = malloc(sizeof(cplx) * (size_t)n_rx * n_beams);
    for (int b = 0; b < n_beams; ++b)
        for (int r0 = 0; r0 < n_rx; r0 += 128) {
            double amax = 0.0;
            int bad = 0;
            for (int r = r0; r < n_rx && r < r0 + 128; ++r) {
                double re = fabs(creal(W[r * n_beams + b])), im = fabs(cimag(W[r * n_beams + b]));
                if (!isfinite(re) || !isfinite(im)) bad = 1;
                if (re > amax) amax = re;
                if (im > amax) amax = im;
            }
            int e = bad ? 128 : orc_e4m3_block_exp(amax);
            for (int r = r0; r < n_rx && r < r0 + 128; ++r) {
                cplx w = W[r * n_beams + b];
                wq[r * n_beams + b] = e >= 128 ? NAN
                    : ldexp(orc_e4m3_round(ldexp(creal(w), -e)), e) + I * ldexp(orc_e4m3_round(ldexp(cimag(w), -e)), e);
            }
        }
    for (int s = 0; s < n_sym; ++s)
        for (int a = 0; a < n_sc; ++a)
            for (int b = 0; b < n_beams; ++b) {
                cplx acc = 0;
                for (int r = 0; r < n_rx; ++r) {
                    int e = exps[((long long)s * n_rx + r) * n_blk + a / 128];
                    cplx x = e >= 128 ? NAN : ldexp(creal(codes[((long long)s * n_rx + r) * n_sc + a]), e)
                                             + I * ldexp(cimag(codes[((long long)s * n_rx + r) * n_sc + a]), e);
                    acc += conj(wq[r * n_beams + b]) * x;
                }
                beam[((long long)s * n_sc + a) * n_beams + b] = acc;
            }
    free(wq);
}
