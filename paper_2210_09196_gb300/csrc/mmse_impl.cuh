// MMSE MIMO detection (Eq. 2), computed as in Section II: Gram G = H^H H + sigma^2 I, Cholesky
// G = L L^H (Section V-C), forward solve L z = H^H y, back solve L^H x = z; then Gray hard decisions.
//
// GB300 mapping: a group of NL lanes owns one subcarrier (NL = layer class 2..32, a power of two), so a
// warp detects 32/NL subcarriers at once; lane i of a group owns layer i.
//   0. The data-symbol vectors y_d of the warp's subcarriers are copied to shared memory with cp.async
//      first, so that their latency overlaps step 1.
//   1. The estimate rows of the warp's subcarriers are copied to shared memory with 16-byte cp.async pieces
//      (rows padded to an even stride), or, in the chain of pusch_slot (16 and 32 lanes, 32 or 64 beams),
//      interpolated there from the LS table at the pilots, so that the estimate never goes through HBM.
//   2. Lane i forms row i of G from 16-byte shared loads, then r_d = H^H y_d for every data symbol d.
//   3. The r_d go to shared memory (over the group's data-symbol rows); Crout Cholesky of G column by column:
//      lane i keeps row i of L in registers, the pivot by one shuffle, and publishes every entry over the (now
//      dead) H tile as a broadcast-ready (-Re, -Re, Im, Im) float4.
//   4. Lane i solves the forward and back systems of data symbols i, i + NL, ... with packed FMAs, one
//      broadcast 16-byte load per complex multiply-add; x returns to lane i (= layer i) through shared memory.
// With one estimate per slot, G and L are formed once per subcarrier, which gives the same result as forming
// them per data symbol. With an estimate that varies in time (chol_every = K > 0) the data symbols are taken
// in groups of K and each group is one launch of this kernel with that group's estimate (Section VI's
// schedule: K = 1 is one factorisation per data symbol); d_first / n_det select the group's symbols. Layers beyond n_layers (up to NL) are padded with identity rows and produce
// nothing.
#pragma once

#include "chest_common.cuh"
#include "bounded_wait.cuh"
#include "detect_core.cuh"
#include "detect_tc.cuh"

namespace pusch {
namespace mmse_detail {

constexpr unsigned kFull = 0xffffffffu;

struct MmseArgs {
    int n_sc, n_beams, n_layers, n_sym, n_data, qam_bits;
    float load;  // sigma^2 + extra loading (sigma2 == nullptr)
    float loading;             // extra loading alone
    const float *sigma2;       // per-slot noise variance (device) or nullptr
    int d_first, n_det;        // this launch detects data symbols d_first .. d_first + n_det - 1 (n_data in all)
    int dmrs_lo, dmrs_hi;      // the two DMRS symbols, dmrs_lo < dmrs_hi
    int warps;                 // warps per CTA of the 12-symbol kernels (mmse_warp_choices; 0 = default)
    // LS table at the pilots (ls[slot][l][k][b], pilot q = port[l] + k comb, k < kmax) or nullptr: when set,
    // the beam-count instances interpolate their estimate rows from it while staging (the same arithmetic as
    // the interpolation kernel) and the H argument is not read
    const float2 *ls;
    int kmax, comb;
    int port[32];
};

// Symbol index of data symbol d: the data symbols are all other symbols of the slot in increasing order.
// (Computed rather than read from a table: one compare per DMRS symbol.)
__device__ __forceinline__ int data_symbol(const MmseArgs &g, int d) {
    int s = d;
    if (s >= g.dmrs_lo) ++s;
    if (s >= g.dmrs_hi) ++s;
    return s;
}

// The estimate rows of the warp's SPW subcarriers (from Hq, one group's estimate) -> the warp's H tile, rows
// padded to stride hs; 16-byte cp.async pieces (two beams) when the beam count is even, 8-byte pieces
// otherwise; rows of absent layers and subcarriers are zeroed. Waits for all of the lane's copies.
template <int NL>
__device__ __forceinline__ void stage_H(float2 *Ht, const float2 *__restrict__ Hq, long long sc0, long long total_sc,
                                        int nl, int nb, int hs, int ht, int lane) {
    constexpr int SPW = 32 / NL;
    const int rows = SPW * NL;
    const bool wide = (nb & 1) == 0;
    const int cpr = wide ? nb >> 1 : nb;  // pieces per row
    int r = lane / cpr, c = lane - (lane / cpr) * cpr;
    const int step_r = 32 / cpr, step_c = 32 - (32 / cpr) * cpr;
    for (; r < rows;) {
        const int gg = r / NL, l = r - gg * NL;  // NL is a power of two
        const int b = wide ? 2 * c : c;
        float2 *dst = Ht + gg * ht + l * hs + b;
        if (l < nl && sc0 + gg < total_sc) {
            const float2 *src = Hq + ((sc0 + gg) * nl + l) * (long long)nb + b;
            if (wide)
                cp_async16(dst, src);
            else
                cp_async8(dst, src);
        } else {
            dst[0] = make_float2(0.f, 0.f);
            if (wide) dst[1] = make_float2(0.f, 0.f);
        }
        r += step_r;
        c += step_c;
        if (c >= cpr) {
            c -= cpr;
            ++r;
        }
    }
    cp_async_wait_all();  // the H tile (and the earlier y group)
}

// The interpolated estimate rows of the warp's SPW subcarriers -> the warp's H tile, from the LS table at the
// pilots (Section II: linear interpolation between the neighbouring pilot subcarriers of each layer, held
// outside the first and last; the arithmetic of the interpolation kernel, so the tile is bit-identical to
// staging its output). Lane r finds the bracket of row r (subcarrier sc0 + r / NL, layer r % NL; SPW NL = 32
// rows); the warp then reads the two table rows of every tile row in 16-byte pieces (NB / 2 per row), issuing
// kB pieces' loads before using any. Rows of absent layers and subcarriers are zeroed.
template <int NL, int NB>
__device__ __forceinline__ void stage_H_interp(float2 *Ht, const MmseArgs &g, long long sc0, long long total_sc,
                                               int ht, int lane) {
    constexpr int kU = NB / 2;            // 16-byte pieces per row
    constexpr int kRows = 32 / kU;        // rows per warp pass (2 for 32 beams, 1 for 64)
    constexpr int kHs = (NB + 3) & ~1;    // row_stride(NB)
    constexpr int kB = 4;                 // passes whose loads are issued together
    long long base = -1;                  // table row of (slot, layer, k = 0), in 16-byte pieces
    int klo = 0, khi = 0;
    float w = 0.f;
    {
        const int gg = lane / NL, l = lane - gg * NL;
        const long long sc = sc0 + gg;
        if (l < g.n_layers && sc < total_sc) {
            const long long sl = sc / g.n_sc;
            const int a = (int)(sc - sl * g.n_sc), p = g.port[l];
            int lo, hi;
            pilot_bracket(a, p, g.comb, g.n_sc, lo, hi);
            klo = (lo - p) / g.comb;
            khi = (hi - p) / g.comb;
            w = interp_weight(a, lo, hi);
            base = (sl * g.n_layers + l) * (long long)g.kmax * kU;
        }
    }
    const float4 *tab = reinterpret_cast<const float4 *>(g.ls);
    const int sub = lane / kU, u = lane - sub * kU;
    // rows of pass t: when a pass covers SPW rows, the same layer of the warp's SPW subcarriers (neighbouring
    // subcarriers mostly share the bracket, so the pass reads each table line once); else kRows consecutive rows
    constexpr int SPW = 32 / NL;
    auto row_of = [&](int t) { return kRows == SPW ? sub * NL + t : t * kRows + sub; };
#pragma unroll 1
    for (int t0 = 0; t0 < 32 / kRows; t0 += kB) {
        float4 lo4[kB], hi4[kB];
        float wr[kB];
        bool on[kB];
#pragma unroll
        for (int q = 0; q < kB; ++q) {
            const int r = row_of(t0 + q);
            const long long b = __shfl_sync(kFull, base, r);
            const int kl = __shfl_sync(kFull, klo, r), kh = __shfl_sync(kFull, khi, r);
            wr[q] = __shfl_sync(kFull, w, r);
            on[q] = b >= 0;
            lo4[q] = hi4[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (on[q]) {
                lo4[q] = __ldg(tab + b + (long long)kl * kU + u);
                hi4[q] = __ldg(tab + b + (long long)kh * kU + u);
            }
        }
#pragma unroll
        for (int q = 0; q < kB; ++q) {
            const int r = row_of(t0 + q);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (on[q]) {
                const float2 h0 = interp(make_float2(lo4[q].x, lo4[q].y), make_float2(hi4[q].x, hi4[q].y), wr[q]);
                const float2 h1 = interp(make_float2(lo4[q].z, lo4[q].w), make_float2(hi4[q].z, hi4[q].w), wr[q]);
                v = make_float4(h0.x, h0.y, h1.x, h1.y);
            }
            *reinterpret_cast<float4 *>(Ht + (r / NL) * ht + (r % NL) * kHs + 2 * u) = v;
        }
    }
}

// Warps per CTA of the 12-data-symbol kernels when not tuned: one (each warp then starts and ends on its own;
// larger CTAs measured slower for 16 layers, their warps waiting for one another at the output rows), four for
// 32 layers (one subcarrier per warp).
template <int NL>
constexpr int mmse_default_warps() {
    return NL == 32 ? 4 : 1;
}
// Register cap: 10 warps per SM up to 8 layers, 14 for 16 layers (128 registers: the shared-memory limit is
// also 14 warps of two subcarriers), none for 32.
template <int NL, int WARPS>
constexpr int mmse_min_ctas() {
    constexpr int w = NL <= 8 ? 10 : (NL == 16 ? 14 : WARPS);
    return (w + WARPS - 1) / WARPS;
}
// One CTA detects SPC = WARPS * 32 / NL consecutive subcarriers (warp w: SPW = 32 / NL of them from
// w * SPW). After every warp has left its x_d in its data-symbol rows, the CTA writes x-hat and the bits row by
// row: the SPC subcarriers of one (slot, layer, data symbol) row are consecutive in both outputs, so each row
// segment is one contiguous run of SPC elements (a warp per subcarrier pair would write 16-byte pieces of 16
// rows).
// NB > 0: compiled for NB beams (every shared-memory offset of the Gram, matched-filter and staging loops is
// then a constant) and staged by bulk copies on one mbarrier per warp; 0: g.n_beams at run time, cp.async.
template <int NL, int ND, int WARPS, int NB>
__global__ void __launch_bounds__(WARPS * 32, mmse_min_ctas<NL, WARPS>())
mmse_kernel(const __grid_constant__ MmseArgs g, long long total_sc, const float2 *__restrict__ H, const float2 *__restrict__ beam,
            float2 *__restrict__ xhat, uint8_t *__restrict__ bits, uint32_t *__restrict__ status) {
    constexpr int SPW = 32 / NL;
    constexpr int SPC = WARPS * SPW;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / NL, i = lane - grp * NL;
    const int src0 = grp * NL;
    const int nl = g.n_layers, nb = NB > 0 ? NB : g.n_beams, n_sc = g.n_sc;
    // nd: the data symbols this launch detects (ND when compiled in, else n_det)
    const int nd = ND > 0 ? ND : g.n_det;
    const int hs = row_stride(nb), ht = htile<NL>(nb), ys = y_stride<NL>(nb);
    const size_t wsb = warp_smem_bytes<NL>(nb, nd);

    unsigned char *wbase = smem_raw + (size_t)warp * wsb;
    float2 *Ht = reinterpret_cast<float2 *>(wbase);  // [SPW][ht]
    float2 *Yt = Ht + SPW * ht;                      // [SPW][nd][ys]

    const long long cta_sc0 = (long long)blockIdx.x * SPC;
    const long long sc0 = cta_sc0 + warp * SPW;  // first (slot*n_sc + a) of warp
    if (sc0 < total_sc) {                        // else the whole warp is idle until the output rows
        const long long my_sc = sc0 + grp;
        const bool valid = my_sc < total_sc;
        const long long slot = my_sc / n_sc;

        const float2 *hr = Ht + grp * ht + i * hs;  // own row
        const float2 *hg = Ht + grp * ht;           // the group's rows
        constexpr int NR = ND > 0 ? ND : 14;
        float2 acc[NR];
        if constexpr (NB > 0) {
            // ---- 0-1. the estimate rows and the data-symbol rows of the warp's subcarriers -> shared memory by
            //           bulk copies (one 8 NB-byte row each, by the copy engine, completing on the warp's
            //           mbarrier); rows of absent layers and subcarriers are zeroed. The launcher uses these
            //           instances only with 16-byte aligned H and beam.
            const uint32_t bar = smem_addr(reinterpret_cast<uint64_t *>(smem_raw + (size_t)WARPS * wsb) + warp);
            constexpr uint32_t kRowB = NB * 8;
            const bool interp_h = g.ls != nullptr;   // estimate rows interpolated from the LS table
            uint32_t my_bytes = 0;
            for (int r = lane; r < SPW * NL && !interp_h; r += 32)
                if (r % NL < nl && sc0 + r / NL < total_sc) my_bytes += kRowB;
            for (int r = lane; r < SPW * nd; r += 32)
                if (sc0 + r / nd < total_sc) my_bytes += kRowB;
            const uint32_t total = __reduce_add_sync(kFull, my_bytes);
            if (lane == 0) {
                bw::mbar_init(bar, 1);
                asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(total) : "memory");
            }
            __syncwarp();
            for (int r = lane; r < SPW * NL && !interp_h; r += 32) {
                const int gg = r / NL, l = r - gg * NL;
                float2 *dst = Ht + gg * ht + l * hs;
                if (l < nl && sc0 + gg < total_sc) {
                    const float2 *src = H + ((sc0 + gg) * nl + l) * (long long)NB;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_addr(dst)),
                        "l"(src), "r"(kRowB), "r"(bar)
                        : "memory");
                } else {
#pragma unroll
                    for (int b = 0; b < NB; b += 2) *reinterpret_cast<float4 *>(dst + b) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            for (int r = lane; r < SPW * nd; r += 32) {
                const int gg = r / nd, d = r - gg * nd;
                const long long sc = sc0 + gg;
                float2 *dst = Yt + (gg * nd + d) * ys;
                if (sc < total_sc) {
                    const long long sl = sc / n_sc, aa = sc - sl * n_sc;
                    const float2 *src = beam + ((sl * g.n_sym + data_symbol(g, g.d_first + d)) * n_sc + aa) * NB;
                    asm volatile(
                        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                            smem_addr(dst)),
                        "l"(src), "r"(kRowB), "r"(bar)
                        : "memory");
                } else {
#pragma unroll
                    for (int b = 0; b < NB; b += 2) *reinterpret_cast<float4 *>(dst + b) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            if (interp_h) stage_H_interp<NL, NB>(Ht, g, sc0, total_sc, ht, lane);   // overlaps the y copies
            // bounded wait (2 s); on expiry the timeout bit is set and the copies are waited for once more
            if (!bw::mbar_wait_for(bar, 0, bw::kWaitNs)) {
                if (lane == 0) atomicOr(&status[0], (unsigned)PUSCH_STATUS_TIMEOUT);
                bw::mbar_wait_for(bar, 0, bw::kWaitNs);
            }
            __syncwarp();
        } else {
        // ---- 0. the data-symbol rows y_d of the warp's subcarriers -> shared memory, asynchronously (cp.async,
        //         16-byte pieces when the beam count is even); waited for just before step 2b.
        {
            const bool wide = (nb & 1) == 0;
            const int cpr = wide ? nb >> 1 : nb;  // pieces per row
            int row = lane / cpr, c = lane - (lane / cpr) * cpr;
            const int step_r = 32 / cpr, step_c = 32 - (32 / cpr) * cpr;
            for (; row < SPW * nd;) {
                const int gg = row / nd, d = row - gg * nd;
                const long long sc = sc0 + gg;
                float2 *dst = Yt + (gg * nd + d) * ys + (wide ? 2 * c : c);
                if (sc < total_sc) {
                    const long long sl = sc / n_sc, aa = sc - sl * n_sc;
                    const float2 *src =
                        beam + ((sl * g.n_sym + data_symbol(g, g.d_first + d)) * n_sc + aa) * nb + (wide ? 2 * c : c);
                    if (wide)
                        cp_async16(dst, src);
                    else
                        cp_async8(dst, src);
                } else {
                    dst[0] = make_float2(0.f, 0.f);
                    if (wide) dst[1] = make_float2(0.f, 0.f);
                }
                row += step_r;
                c += step_c;
                if (c >= cpr) {
                    c -= cpr;
                    ++row;
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // ---- 1. channel estimate rows -> shared memory (waits for both copy groups)
        stage_H<NL>(Ht, H, sc0, total_sc, nl, nb, hs, ht, lane);
        __syncwarp();
        }
        // ---- 2-4. Gram, matched filter, Cholesky and solves, the x_d left in the data-symbol rows (detect_group).
        bool bad;
        if constexpr (NB > 0 && ND == 12 && NL >= 16)   // G and r_d on the tensor cores
            bad = detect_group_tc<NL, NB>(Ht, ht, hs, Yt, ys, nl, g.sigma2 ? g.loading : g.load, grp, i, src0, lane,
                                          acc, g.sigma2, valid ? slot : 0);
        else
            bad = detect_group<NL, ND, NR>(hr, hg, Yt + grp * nd * ys, Ht + grp * ht, hs, nb, nd, nl,
                                           g.sigma2 ? g.loading : g.load, i, src0, acc, g.sigma2, valid ? slot : 0, ys);
        if (valid && bad && i == 0) {
            atomicAdd(&status[1], 1u);
            atomicMin(&status[2], (unsigned)my_sc);
            atomicOr(&status[0], (unsigned)PUSCH_STATUS_PIVOT);
        }
    }
    __syncthreads();

    // ---- 5. x-hat and the Gray decisions, row by row: thread t writes subcarrier cta_sc0 + t % SPC of the rows
    //         (layer l, data symbol d_first + d), l * nd + d = t / SPC, t / SPC + NL, ... (the CTA's WARPS * 32
    //         threads are NL times its SPC subcarriers), reading x_d[l] from that subcarrier's rows.
    bool nonfinite = false;
    {
        const int s = threadIdx.x % SPC;
        const long long sc = cta_sc0 + s;
        if (sc < total_sc) {
            const int w = s / SPW, gg = s - w * SPW;
            const float2 *yt = reinterpret_cast<const float2 *>(smem_raw + (size_t)w * wsb) + SPW * ht + gg * nd * ys;
            const long long sl = sc / n_sc, a = sc - sl * n_sc;
            float2 *xo = xhat + (sl * nl * (long long)g.n_data + g.d_first) * n_sc + a;
            uint8_t *bo = bits + (sl * nl * (long long)g.n_data + g.d_first) * n_sc + a;
            for (int ld = threadIdx.x / SPC; ld < nl * nd; ld += NL) {
                const int l = ld / nd, d = ld - l * nd;
                const float2 x = yt[d * ys + l];
                const long long o = ((long long)l * g.n_data + d) * n_sc;
                xo[o] = x;
                bo[o] = det_demap(x, g.qam_bits);
                if (!isfinite(x.x) || !isfinite(x.y)) nonfinite = true;
            }
        }
    }
    if (__any_sync(kFull, nonfinite) && lane == 0) atomicOr(&status[0], (unsigned)PUSCH_STATUS_NONFINITE);
}

template <int NL, int ND, int WARPS, int NB>
cudaError_t launch_nl(const MmseArgs &a, long long total_sc, const float2 *H, const float2 *beam, float2 *xhat,
                      uint8_t *bits, uint32_t *status, cudaStream_t st) {
    constexpr int SPW = 32 / NL;
    const size_t smem = (size_t)WARPS * warp_smem_bytes<NL>(a.n_beams, ND > 0 ? ND : a.n_det) + (NB > 0 ? 8 * WARPS : 0);
    const long long per_cta = (long long)WARPS * SPW;
    const long long grid = (total_sc + per_cta - 1) / per_cta;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto k = mmse_kernel<NL, ND, WARPS, NB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)grid, WARPS * 32, smem, st>>>(a, total_sc, H, beam, xhat, bits, status);
    return cudaGetLastError();
}

// Shared memory one CTA may hold (opt-in maximum per block).
constexpr size_t kMmseSmemMax = 227 * 1024;

// Compiled-in symbol counts: 12 (one estimate per slot; 1, 2, 4 or 8 warps per CTA, a.warps, if that many
// warps' tiles fit in shared memory, else the default), 4 and 1 (Section VI's schedules, one factorisation per 4
// data symbols or per symbol); anything else at run time. The defaults fit every supported shape (at most 64
// beams and 12 data symbols: 120 KB for a 2-layer warp of 16 subcarriers).
template <int NL, int NB>
cudaError_t launch_w(const MmseArgs &a, long long total_sc, const float2 *H, const float2 *beam, float2 *xhat,
                     uint8_t *bits, uint32_t *status, cudaStream_t st) {
    constexpr int W = mmse_default_warps<NL>();
    const bool fits = (size_t)a.warps * warp_smem_bytes<NL>(a.n_beams, a.n_det) <= kMmseSmemMax;
    if (a.n_det == 12 && fits && a.warps == 1) return launch_nl<NL, 12, 1, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 12 && fits && a.warps == 2) return launch_nl<NL, 12, 2, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 12 && fits && a.warps == 4) return launch_nl<NL, 12, 4, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 12 && fits && a.warps == 8) return launch_nl<NL, 12, 8, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 12) return launch_nl<NL, 12, W, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 4) return launch_nl<NL, 4, W, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    if (a.n_det == 1) return launch_nl<NL, 1, W, NB>(a, total_sc, H, beam, xhat, bits, status, st);
    return launch_nl<NL, 0, W, 0>(a, total_sc, H, beam, xhat, bits, status, st);
}

// The 16- and 32-layer classes are also compiled for 32 and 64 beams.
template <int NL>
cudaError_t launch_nd(const MmseArgs &a, long long total_sc, const float2 *H, const float2 *beam, float2 *xhat,
                      uint8_t *bits, uint32_t *status, cudaStream_t st) {
    if constexpr (NL >= 16) {
        // the beam-count instances stage by bulk copies: 16-byte aligned rows
        const bool aligned = reinterpret_cast<uintptr_t>(H) % 16 == 0 && reinterpret_cast<uintptr_t>(beam) % 16 == 0 &&
                             reinterpret_cast<uintptr_t>(a.ls) % 16 == 0;
        if (aligned && a.n_beams == 32) return launch_w<NL, 32>(a, total_sc, H, beam, xhat, bits, status, st);
        if (aligned && a.n_beams == 64) return launch_w<NL, 64>(a, total_sc, H, beam, xhat, bits, status, st);
    }
    if (a.ls) return cudaErrorNotSupported;   // only the beam-count instances interpolate while staging
    return launch_w<NL, 0>(a, total_sc, H, beam, xhat, bits, status, st);
}

// Warps per CTA that a.warps may select for the 12-symbol kernels of a layer class with n_beams beams (the
// default first, then the other counts of 1, 2, 4 and 8 whose tiles fit); returns their count (at most 4).
template <int NL>
int mmse_warp_choices(int n_beams, int *out) {
    constexpr int W = mmse_default_warps<NL>();
    const size_t wb = warp_smem_bytes<NL>(n_beams, 12);
    int n = 0;
    out[n++] = W;
    for (int w = 1; w <= 8; w *= 2)
        if (w != W && w * wb <= kMmseSmemMax) out[n++] = w;
    return n;
}

}  // namespace mmse_detail

// Launch of one layer class (separate translation units, compiled in parallel): NL = 2, 4 or 8 in
// mmse_small.cu, 16 in mmse_nl16.cu, 32 in mmse_nl32.cu.
cudaError_t mmse_launch_class(int nl_class, const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                              const float2 *beam, float2 *xhat, uint8_t *bits, uint32_t *status, cudaStream_t st);
cudaError_t mmse_launch_class16(const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                                const float2 *beam, float2 *xhat, uint8_t *bits, uint32_t *status, cudaStream_t st);
cudaError_t mmse_launch_class32(const mmse_detail::MmseArgs &a, long long total_sc, const float2 *H,
                                const float2 *beam, float2 *xhat, uint8_t *bits, uint32_t *status, cudaStream_t st);

}  // namespace pusch
