// Beamforming on the 5th-generation tensor cores (tcgen05 + TMEM, operands staged by TMA): the mixed form
// (FP16 operands) and the FP8 form (E4M3 operands with power-of-two block scales), FP32 accumulation.
//
// The per-symbol product Y = W^H X of Section II (Table I "BF") is computed as a real GEMM with the
// complex values embedded:  D[a][2b + c] = sum_k A[a][k] B[2b + c][k],  k = 2r + ri, where
//   A[a][2r + 0] = Re X[r][a],  A[a][2r + 1] = Im X[r][a]                        (the FFT output)
//   B[2b][2r] = Re W[r][b],  B[2b][2r+1] = Im W[r][b],  B[2b+1][2r] = -Im W[r][b],  B[2b+1][2r+1] = Re W[r][b]
// so that D[a][2b] = Re y_b and D[a][2b + 1] = Im y_b: each accumulator row is the c64 output row of
// subcarrier a. The MMA's M dimension is the subcarrier axis (tiles of 128), N = 2 N_B, K = 2 N_R.
//
// A is the FFT output [rows][2 N_R][pitch] (subcarriers contiguous): an MN-major operand, copied by TMA
// in K chunks with 128-byte swizzling into a ring of shared-memory stages. B is built once per CTA from W
// in the no-swizzle K-major core-matrix layout and stays resident. Both operands reach the MMA as FP16.
//
// Warp roles (persistent CTAs, one per SM):
//   warp 0      TMA producer: streams the (tile, K chunk) sequence into the stage ring;
//   warp 1      owns the TMEM allocation; one lane issues the MMAs of each chunk into one of two TMEM
//               accumulators and commits the chunk's stage back to the producer;
//   warps 2-5   epilogue: tcgen05.ld of the finished accumulator (one 32-lane quarter per warp), scaling
//               (FP8 form), stores of the c64 rows; the other accumulator is being filled meanwhile;
//   warps 6-13  FP8 form only: convert each landed chunk of E4M3 codes to FP16 for the MMA (below).
//
// FP8 form. The FFT stores each (symbol, antenna) row as E4M3 codes with one power-of-two scale 2^e per
// 128 subcarriers; W is quantised in the kernel to E4M3 with one power-of-two scale per (beam, 128
// antennas). The product is the block-scaled product of these two quantised operands: every operand keeps
// its own scale, nothing is re-rounded. E4M3 codes move through HBM and the TMA ring (one byte each); the
// convert warps write each landed chunk into a second ring as FP16 values code * 2^(e_r - E), E the
// largest exponent among the tile's antennas, and B holds W's codes as FP16 values code * 2^(e_w - E_b),
// E_b the largest block exponent of beam b. FP16 holds a 4-significant-bit E4M3 code shifted down by up
// to 15 octaves exactly (its smallest step is 2^-24, an E4M3 code's 2^-9 shifted 15 times), so the MMA
// (kind::f16, FP32 accumulation) sums exact products; one accumulator holds D * 2^-(E + E_b) and the
// epilogue multiplies by 2^E * 2^E_b. Blocks more than 15 octaves below the largest of their tile round
// in FP16 (below 2^-15 of the tile's largest sample, well under the FP32 sum's own rounding). A
// non-finite scale (a non-finite sample in the block) makes the tile's output NaN, so detection reports it.
//
// Every wait is bounded (%globaltimer, 2 s); on expiry the CTA records a timeout in err_word bit 0, all
// roles leave their loops, in-flight copies and MMAs are drained (bounded) and TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <float.h>

#include "tc_common.cuh"

namespace pusch {
namespace {

constexpr int kTileM = 128;
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kMaxRxFp8 = 512;   // W block exponents are kept for up to 4 blocks of 128 antennas
constexpr int kConvWarps = 8;     // FP8: warps that convert the landed codes

using namespace tc;

// Exponent of a power-of-two block scale as stored by the FFT (an exact power of two, or NaN for a
// non-finite block): e in [-126, 127], or 128 for NaN/inf.
__device__ __forceinline__ int scale_exp(float s) { return (int)((__float_as_uint(s) >> 23) & 0xFFu) - 127; }

// 2^e as a float for e in [-126, 127]; NaN for e = 128.
__device__ __forceinline__ float exp2_int(int e) {
    return e >= 128 ? __uint_as_float(0x7FC00000u) : __uint_as_float((uint32_t)(e + 127) << 23);
}

// E4M3 conversions (PTX cvt: round to nearest even, saturating to +-448). A pair's low byte / low half is
// the first element.
__device__ __forceinline__ uint32_t h2_from_e4m3x2(uint16_t v) {          // two codes -> f16x2 (exact)
    uint32_t r;
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(r) : "h"(v));
    return r;
}
__device__ __forceinline__ float2 e4m3x2_to_float2(uint16_t v) {
    const uint32_t h = h2_from_e4m3x2(v);
    return __half22float2(*reinterpret_cast<const __half2 *>(&h));
}
__device__ __forceinline__ uint16_t float2_to_e4m3x2(float2 v) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(v.y), "f"(v.x));
    return r;
}

// Smallest e with amax <= 448 * 2^e (the power-of-two E4M3 block scale), clamped below at -126;
// 128 for a non-finite amax. Read from the float's bits: amax = 1.m * 2^(E - 127).
__device__ __forceinline__ int block_exp(float amax) {
    if (!(amax <= FLT_MAX)) return 128;
    const uint32_t u = __float_as_uint(amax);
    const int eb = (int)(u >> 23);
    if (eb == 0) return -126;                      // zero or subnormal
    const int e = eb - 127 - 8 + ((u & 0x7FFFFFu) > 0x600000u ? 1 : 0);   // 448 = 1.75 * 2^8
    return e < -126 ? -126 : e;
}

struct TcArgs {
    int n_rx, n_beams, n_sc, n_mtiles, n_blk;
    int K, N, chunk_rows, n_chunks, n_stages, tmem_cols;
    uint32_t stage_bytes, b_bytes;
    uint32_t land_bytes, land_off;  // FP8: landing stage of E4M3 codes and the landing ring's offset
    int n_land;                     // FP8: landing stages (the TMA ring; the FP16 ring has n_stages)
    int stage_out;             // 1: the epilogue writes through shared memory and TMA tensor stores
    long long total_tiles;
};

struct TcShared {
    uint64_t full[kMaxStages], ready[kMaxStages], empty[kMaxStages], lempty[kMaxStages];
    uint64_t tfull[2], tempty[2], drain;
    uint32_t tmem_base;
    int abort;
    int ew[64 * 4];            // FP8: W block exponents [beam][128-antenna block]
    int wexp[64];              // FP8: E_b, the largest block exponent of beam b
    float wsc[64];             // FP8: 2^E_b
    uint8_t shift[kConvWarps][kMaxRxFp8];  // FP8: per convert warp, the shift E - e_r of each antenna of its tile
};

template <bool FP8>
__global__ void __launch_bounds__(FP8 ? 192 + 32 * kConvWarps : 192, 1)
beamform_tc_kernel(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap omap, TcArgs g,
                   const float2 *__restrict__ W, const float *__restrict__ scales, float2 *__restrict__ beam,
                   uint32_t *__restrict__ err) {
    constexpr int kThreads = FP8 ? 192 + 32 * kConvWarps : 192;
    constexpr int kKStep = 16;                  // K per MMA instruction (32 bytes of FP16)
    extern __shared__ uint8_t smem_raw[];
    __shared__ TcShared sh;

    const int K = g.K, N = g.N;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sA = base;
    const uint32_t sB = base + (uint32_t)g.n_stages * g.stage_bytes;
    uint8_t *gB = gbase + (size_t)g.n_stages * g.stage_bytes;
    // output staging (stage_out): per epilogue warp, 32 rows x N floats as N/16 boxes of 32 x 16 floats with
    // 64-byte swizzling (16-byte chunk c of row r at r * 64 + ((c ^ ((r >> 1) & 3)) << 4)), 2 KB each
    const uint32_t out_off = (uint32_t)g.n_stages * g.stage_bytes + ((g.b_bytes + 1023u) & ~1023u);
    const uint32_t b_sbo = (uint32_t)K * 16;  // bytes between 8-row groups of B

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *abort = &sh.abort;

    // ---------------------------------------------------------------- B operand (resident) from W
    // W [n_rx][n_beams] is staged through the (still unused) FP16 ring in pieces of whole antennas, every
    // 8-byte element copied by cp.async so that a piece costs one round trip; B's 16-byte chunks (beam row n,
    // 8 consecutive k = 4 antennas x (re, im)) are then written whole, element (n, k) at (n/8)*SBO +
    // (k/8)*128 + (n%8)*16 + (k%8)*2. FP8: a first pass over the pieces takes the largest |Re|, |Im| per
    // (beam, 128-antenna block) (shared atomics on the bit patterns: non-negative floats order like their
    // bits; a non-finite component records +inf), the second writes the codes as FP16 values on the beam's
    // scale.
    {
        float2 *Ws = reinterpret_cast<float2 *>(gbase);
        const int nb = g.n_beams;
        int P = (int)(((size_t)g.n_stages * g.stage_bytes) / ((size_t)nb * 8));
        P = (P / 4) * 4;
        if (P > g.n_rx) P = g.n_rx;
        auto stage_piece = [&](int r0, int np) {
            __syncthreads();                                 // the previous piece is consumed
            const float2 *src = W + (size_t)r0 * nb;
            const int cnt = np * nb;
            for (int i2 = tid; i2 < cnt; i2 += kThreads)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(Ws + i2)), "l"(src + i2) : "memory");
            asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
            __syncthreads();
        };
        const int n_kb = (g.n_rx + 127) / 128;
        if constexpr (FP8) {
            uint32_t *wmax = reinterpret_cast<uint32_t *>(sh.ew);
            for (int i2 = tid; i2 < 64 * 4; i2 += kThreads) wmax[i2] = 0u;
            for (int r0 = 0; r0 < g.n_rx; r0 += P) {
                const int np = min(P, g.n_rx - r0);
                stage_piece(r0, np);
                for (int i2 = tid; i2 < np * nb; i2 += kThreads) {
                    const int r = r0 + i2 / nb, b = i2 - (i2 / nb) * nb;
                    const float2 w = Ws[i2];
                    const float ax = fabsf(w.x), ay = fabsf(w.y);
                    const bool bad = !(ax <= FLT_MAX) || !(ay <= FLT_MAX);
                    atomicMax(&wmax[b * 4 + (r >> 7)], bad ? 0x7F800000u : __float_as_uint(fmaxf(ax, ay)));
                }
            }
            __syncthreads();
            for (int i2 = tid; i2 < nb * 4; i2 += kThreads)
                sh.ew[i2] = (i2 & 3) < n_kb ? block_exp(__uint_as_float(wmax[i2])) : -126;
            __syncthreads();
            for (int b = tid; b < nb; b += kThreads) {
                int e = -126;
                for (int kb = 0; kb < n_kb; ++kb) e = max(e, sh.ew[b * 4 + kb]);
                sh.wexp[b] = e;
                sh.wsc[b] = exp2_int(e);
            }
        }
        const bool resident = P >= g.n_rx;                   // W already staged whole (FP8 pass 1)
        for (int r0 = 0; r0 < g.n_rx; r0 += P) {
            const int np = min(P, g.n_rx - r0);
            if (FP8 && resident) __syncthreads();            // pass 1's exponents are visible
            else stage_piece(r0, np);
            const int nchunks = (np / 4) * N;
            for (int c = tid; c < nchunks; c += kThreads) {
                const int kcl = c / N, n = c - kcl * N;
                const int b = n >> 1;
                uint32_t h[4];
#pragma unroll
                for (int a4 = 0; a4 < 4; ++a4) {
                    const float2 w = Ws[(4 * kcl + a4) * nb + b];
                    __half re, im;
                    if constexpr (FP8) {
                        const int r = r0 + 4 * kcl + a4;
                        const int eb = sh.wexp[b], e_blk = sh.ew[b * 4 + (r >> 7)];
                        if (eb >= 128) {                     // the beam's scale is NaN; values unused
                            re = im = __float2half_rn(0.f);
                        } else {
                            const float inv = exp2_int(-e_blk);   // 2^-e_blk, e_blk in [-126, 120]
                            const float2 cq = e4m3x2_to_float2(float2_to_e4m3x2(make_float2(w.x * inv, w.y * inv)));
                            const int d = eb - e_blk;             // shift of this block to the beam exponent
                            const float sh2 = exp2_int(d > 40 ? -40 : -d);
                            re = __float2half_rn(cq.x * sh2);
                            im = __float2half_rn(cq.y * sh2);
                        }
                    } else {
                        re = __float2half_rn(w.x);
                        im = __float2half_rn(w.y);
                    }
                    // row 2b: (Re, Im); row 2b + 1: (-Im, Re)
                    const __half lo = (n & 1) ? __hneg(im) : re, hi = (n & 1) ? re : im;
                    h[a4] = (uint32_t)__half_as_ushort(lo) | ((uint32_t)__half_as_ushort(hi) << 16);
                }
                const int kc = r0 / 4 + kcl;
                *reinterpret_cast<uint4 *>(gB + (size_t)(n >> 3) * b_sbo + (size_t)kc * 128 + (n & 7) * 16) =
                    make_uint4(h[0], h[1], h[2], h[3]);
            }
        }
        __syncthreads();                                     // B complete; the ring is free again
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    if (tid == 0) {
        for (int s = 0; s < kMaxStages; ++s) {   // both rings (FP8: n_land may exceed n_stages)
            mbar_init(smem_u32(&sh.full[s]), 1);
            mbar_init(smem_u32(&sh.ready[s]), kConvWarps);
            mbar_init(smem_u32(&sh.empty[s]), 1);
            mbar_init(smem_u32(&sh.lempty[s]), kConvWarps);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&sh.tfull[b]), 1);
            mbar_init(smem_u32(&sh.tempty[b]), 4);
        }
        mbar_init(smem_u32(&sh.drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sh.abort = 0;
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem_base)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = sh.tmem_base;

    const long long n_my =
        g.total_tiles > blockIdx.x ? (g.total_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int NS = g.n_stages;
    const int NR = FP8 ? g.n_land : NS;   // stages of the TMA ring

    if (warp == 0) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long gch = 0;
            bool ok = true;
            const uint64_t pol = l2_policy_evict_first();   // every FFT output tile is read once
            for (long long i = 0; i < n_my && ok; ++i) {
                const long long t = blockIdx.x + i * gridDim.x;
                const long long row = t / g.n_mtiles;
                const int mt = (int)(t - row * g.n_mtiles);
                for (int c = 0; c < g.n_chunks; ++c, ++gch) {
                    const int s = (int)(gch % NR);
                    const uint32_t ph = (uint32_t)((gch / NR) & 1);
                    // FP8: the landing stage is free once the convert warps have read it; FP16: once the MMAs
                    // of its previous chunk have completed
                    if (!mbar_wait(smem_u32(FP8 ? &sh.lempty[s] : &sh.empty[s]), ph ^ 1u, abort, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bar = smem_u32(&sh.full[s]);
                    const int y = (int)(row * K) + c * g.chunk_rows;
                    if constexpr (FP8) {
                        mbar_expect_tx(bar, g.land_bytes);
                        tma_load_2d_hint(base + g.land_off + (uint32_t)s * g.land_bytes, &tmap, mt * kTileM, y, bar, pol);
                    } else {
                        const uint32_t dst = sA + (uint32_t)s * g.stage_bytes;
                        mbar_expect_tx(bar, g.stage_bytes);
                        tma_load_2d_hint(dst, &tmap, mt * kTileM, y, bar, pol);
                        tma_load_2d_hint(dst + (uint32_t)g.chunk_rows * 128, &tmap, mt * kTileM + 64, y, bar, pol);
                    }
                }
            }
            if (*abort) {
                // drain: the latest copy issued into each stage (bounded)
                for (long long j = gch - 1; j >= 0 && j >= gch - NR; --j)
                    mbar_drain(smem_u32(&sh.full[(int)(j % NR)]), (uint32_t)((j / NR) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = instr_desc(kTileM, N);
            const uint32_t a_lbo = (uint32_t)g.chunk_rows * 128;   // FP16: between the two 64-subcarrier halves
            long long gch = 0;
            bool ok = true;
            for (long long i = 0; i < n_my && ok; ++i) {
                const int buf = (int)(i & 1);
                const uint32_t use = (uint32_t)((i >> 1) & 1);
                if (!mbar_wait(smem_u32(&sh.tempty[buf]), use ^ 1u, abort, err)) break;
                fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(buf * N);
                for (int c = 0; c < g.n_chunks; ++c, ++gch) {
                    const int s = (int)(gch % NS);
                    const uint32_t ph = (uint32_t)((gch / NS) & 1);
                    // FP8: the convert warps have written the chunk's FP16 stage (after its landing)
                    if (!mbar_wait(smem_u32(FP8 ? &sh.ready[s] : &sh.full[s]), ph, abort, err)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const int rows_here = min(g.chunk_rows, K - c * g.chunk_rows);
                    const uint32_t a0 = sA + (uint32_t)s * g.stage_bytes;
                    const int kb0 = c * (g.chunk_rows / kKStep);
                    for (int ks = 0; ks < rows_here / kKStep; ++ks) {
                        const uint64_t ad = smem_desc(a0 + (uint32_t)ks * (kKStep * 128), a_lbo, 1024, 2);
                        const uint64_t bd = smem_desc(sB + (uint32_t)(kb0 + ks) * 256, 128, b_sbo, 0);
                        mma<false>(d, ad, bd, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                    }
                    mma_commit(smem_u32(&sh.empty[s]));
                }
                if (!ok) break;
                mma_commit(smem_u32(&sh.tfull[buf]));
            }
            // every MMA issued by this thread has completed once the drain barrier flips (bounded)
            mma_commit(smem_u32(&sh.drain));
            mbar_drain(smem_u32(&sh.drain), 0);
        }
    } else if (warp < 6) {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3;                         // TMEM lane quarter this warp may access
        for (long long i = 0; i < n_my; ++i) {
            const int buf = (int)(i & 1);
            const long long t = blockIdx.x + i * gridDim.x;
            const long long row = t / g.n_mtiles;
            const int mt = (int)(t - row * g.n_mtiles);
            float p2e = 1.f;
            if constexpr (FP8) {
                const float *sc = scales + ((size_t)row * g.n_blk + mt) * g.n_rx;
                int e = -126;
                for (int r = lane; r < g.n_rx; r += 32) e = max(e, scale_exp(__ldg(&sc[r])));
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xFFFFFFFFu, e, o));
                p2e = exp2_int(e);
            }
            const bool okw = mbar_wait(smem_u32(&sh.tfull[buf]), (uint32_t)((i >> 1) & 1), abort, err);
            if (!__all_sync(0xFFFFFFFFu, okw)) break;     // warp-uniform: tcgen05.ld is warp-collective
            fence_after_sync();
            const int a = mt * kTileM + q * 32 + lane;
            float *dst = reinterpret_cast<float *>(beam + (row * g.n_sc + a) * (long long)g.n_beams);
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * N);
            const uint32_t stg = base + out_off + (uint32_t)(warp - 2) * (uint32_t)(128 * N);
            uint8_t *gstg = gbase + out_off + (size_t)(warp - 2) * (128 * N);
            if (g.stage_out) {
                if (lane == 0) bulk_wait_read0();          // the previous tile's stores have read the staging
                __syncwarp();
            }
            for (int c0 = 0; c0 < N; c0 += 32) {
                uint32_t r[32];
                const int ncol = N - c0 < 32 ? N - c0 : 32;   // N is a multiple of 16
                if (ncol == 32) tmem_ld32(tbase + (uint32_t)c0, r);
                else tmem_ld16(tbase + (uint32_t)c0, r);
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    if (j < ncol) {
                        float4 v = make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]),
                                               __uint_as_float(r[j + 2]), __uint_as_float(r[j + 3]));
                        if constexpr (FP8) {
                            const float s0 = p2e * sh.wsc[(c0 + j) >> 1], s1 = p2e * sh.wsc[(c0 + j + 2) >> 1];
                            v.x *= s0;
                            v.y *= s0;
                            v.z *= s1;
                            v.w *= s1;
                        }
                        if (g.stage_out) {
                            const int col = c0 + j, box = col >> 4, ch = (col >> 2) & 3;
                            *reinterpret_cast<float4 *>(gstg + box * 2048 + lane * 64 + ((ch ^ ((lane >> 1) & 3)) << 4)) = v;
                        } else if (a < g.n_sc) {
                            *reinterpret_cast<float4 *>(dst + c0 + j) = v;
                        }
                    }
                }
            }
            if (g.stage_out) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                const int y0 = mt * kTileM + q * 32;       // rows past n_sc are clipped; a wholly past box is skipped
                if (lane == 0 && y0 < g.n_sc) {
                    for (int box = 0; box < N / 16; ++box)
                        tma_store_3d(&omap, stg + (uint32_t)box * 2048u, box * 16, y0, (int)row);
                    bulk_commit();
                }
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh.tempty[buf]));
        }
        if (g.stage_out && lane == 0) bulk_wait0();        // stores complete before the CTA's shared memory goes
    } else if constexpr (FP8) {
        // ------------------------------------------------------------------ FP8: codes to FP16
        // Each convert warp derives the tile exponent E itself (no cross-warp barrier, so an abort in one warp
        // cannot strand the others) and converts the 16-byte pieces u = 32 w + lane (mod 32 kConvWarps) of
        // each landed chunk.
        const int w4 = warp - 6;
        long long gch = 0;
        bool ok = true;
        for (long long i = 0; i < n_my && ok; ++i) {
            const long long t = blockIdx.x + i * gridDim.x;
            const long long row = t / g.n_mtiles;
            const int mt = (int)(t - row * g.n_mtiles);
            const float *sc = scales + ((size_t)row * g.n_blk + mt) * g.n_rx;
            int E = -126;
            for (int r = lane; r < g.n_rx; r += 32) E = max(E, scale_exp(__ldg(&sc[r])));
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) E = max(E, __shfl_xor_sync(0xFFFFFFFFu, E, o));
            __syncwarp();                                    // this warp's previous tile no longer reads shift[]
            for (int r = lane; r < g.n_rx; r += 32) {
                const int d = E - scale_exp(__ldg(&sc[r]));
                sh.shift[w4][r] = (uint8_t)(d > 25 ? 25 : d);
            }
            __syncwarp();
            for (int c = 0; c < g.n_chunks; ++c, ++gch) {
                const int s = (int)(gch % NS), sl = (int)(gch % NR);
                const uint32_t ph = (uint32_t)((gch / NS) & 1), phl = (uint32_t)((gch / NR) & 1);
                // the chunk has landed, and the MMAs of the FP16 stage's previous chunk have completed
                bool okw = mbar_wait(smem_u32(&sh.full[sl]), phl, abort, err);
                okw = okw && mbar_wait(smem_u32(&sh.empty[s]), ph ^ 1u, abort, err);
                if (!__all_sync(0xFFFFFFFFu, okw)) {
                    ok = false;
                    break;
                }
                const uint8_t *land = gbase + g.land_off + (size_t)sl * g.land_bytes;
                uint8_t *f16s = gbase + (size_t)s * g.stage_bytes;
                const int k0 = c * g.chunk_rows;
                const int rows_here = min(g.chunk_rows, K - k0);
                const uint32_t half_off = (uint32_t)g.chunk_rows * 128;
                // Landed K row k (one antenna's re or im plane over the tile's 128 subcarriers) is 128 bytes
                // with 16-byte piece j (subcarriers 16 j ..) at piece j ^ (k % 8); its FP16 image is two
                // 64-subcarrier halves of 128-byte rows with 16-byte piece q (8 subcarriers) at q ^ (k % 8),
                // the layout a 128-byte-swizzled TMA box of FP16 planes has. Every value of the row takes the
                // factor 2^-d of its antenna (d = E - e_r): exact in binary16 up to d = 15 (see above).
                // Four units per pass, their loads issued together.
                constexpr int kStride = 32 * kConvWarps;
                for (int u0 = w4 * 32 + lane; u0 < rows_here * 8; u0 += 4 * kStride) {
                    uint4 v[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int u = u0 + kStride * q, k = u >> 3, j = u & 7;
                        if (u < rows_here * 8)
                            v[q] = *reinterpret_cast<const uint4 *>(land + (size_t)k * 128 + ((j ^ (k & 7)) << 4));
                    }
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int u = u0 + kStride * q, k = u >> 3, j = u & 7;
                        if (u >= rows_here * 8) continue;
                        const int d = sh.shift[w4][(k0 + k) >> 1];
                        // 2^-d in binary16: normal for d <= 14, subnormal 2^-24 * 2^(24 - d) up to 24, zero beyond
                        __half2_raw fr;
                        fr.x = fr.y = d <= 14 ? (unsigned short)((15 - d) << 10)
                                              : (d <= 24 ? (unsigned short)(1u << (24 - d)) : (unsigned short)0);
                        const __half2 f2 = *reinterpret_cast<const __half2 *>(&fr);
                        const uint32_t in[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
                        uint32_t o[8];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const uint32_t lo = h2_from_e4m3x2((uint16_t)(in[e] & 0xFFFFu));
                            const uint32_t hi = h2_from_e4m3x2((uint16_t)(in[e] >> 16));
                            const __half2 l2 = __hmul2(*reinterpret_cast<const __half2 *>(&lo), f2);
                            const __half2 h2 = __hmul2(*reinterpret_cast<const __half2 *>(&hi), f2);
                            o[2 * e] = *reinterpret_cast<const uint32_t *>(&l2);
                            o[2 * e + 1] = *reinterpret_cast<const uint32_t *>(&h2);
                        }
                        uint8_t *dst = f16s + (size_t)(j >> 2) * half_off + (size_t)k * 128;
                        const int q0 = 2 * (j & 3);
                        *reinterpret_cast<uint4 *>(dst + ((q0 ^ (k & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
                        *reinterpret_cast<uint4 *>(dst + (((q0 + 1) ^ (k & 7)) << 4)) = make_uint4(o[4], o[5], o[6], o[7]);
                    }
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(smem_u32(&sh.ready[s]));
                    mbar_arrive(smem_u32(&sh.lempty[sl]));
                }
            }
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
    }
}

// Launch plan for a geometry: chunk size and stage count so that B, the ring and the static shared state
// fit in 227 KB with at least 3 stages (2 for the largest B).
struct Plan {
    bool ok;
    int chunk_rows, n_chunks, n_stages, tmem_cols, stage_out;
    uint32_t stage_bytes, b_bytes, land_bytes, land_off;
    int n_land;
    size_t smem;
};

// Launch plan for a geometry: chunk size, stage count and whether the output is staged for TMA stores, so
// that B, the output staging, the ring and the static shared state fit in 227 KB. Without a tuning:
// staged output with >= 3 stages, then direct stores with >= 3 stages, halving the chunk down to 64 rows
// (2 stages are accepted at 64 rows). A tuning (chunk rows, staged) is taken when it fits with >= 2 stages.
Plan plan_for(const Geometry &g, bool fp8, int rows, int staged) {
    Plan p{};
    const int K = 2 * g.n_rx, N = 2 * g.n_beams;
    p.b_bytes = (uint32_t)((size_t)N * K * 2);
    const size_t fixed = 1024 + sizeof(TcShared) + 256 + (((size_t)p.b_bytes + 1023) & ~(size_t)1023);
    int cols = 32;
    while (cols < 2 * N) cols *= 2;
    p.tmem_cols = cols;
    const size_t out_b = staged ? (size_t)512 * N : 0;
    const int cr = K < rows ? K : rows;
    const uint32_t sb = (uint32_t)kTileM * 2 * cr;           // FP16 stage
    const uint32_t lb = fp8 ? (uint32_t)kTileM * cr : 0u;    // FP8: E4M3 landing stage
    const long long avail = (long long)kSmemLimit - (long long)(fixed + out_b);
    int ns = 0, nl = 0;
    if (!fp8) {
        ns = avail > 0 ? (int)(avail / sb) : 0;
        if (ns > kMaxStages) ns = kMaxStages;
    } else {
        // two FP16 stages (the convert warps stay ahead of the MMAs); the rest of shared memory lands codes:
        // the landing ring's bytes in flight set the load bandwidth
        ns = 2;
        const long long rest = avail - (long long)ns * sb;
        nl = rest > 0 ? (int)(rest / lb) : 0;
        if (nl > kMaxStages) nl = kMaxStages;
        if (nl < 2) ns = 0;
    }
    p.chunk_rows = cr;
    p.stage_bytes = sb;
    p.land_bytes = lb;
    p.n_stages = ns;
    p.n_land = nl;
    p.stage_out = staged;
    p.n_chunks = (K + cr - 1) / cr;
    p.land_off = (uint32_t)((size_t)ns * sb + (((size_t)p.b_bytes + 1023) & ~(size_t)1023) + out_b);
    p.smem = 1024 + (size_t)ns * sb + (size_t)nl * lb + (((size_t)p.b_bytes + 1023) & ~(size_t)1023) + out_b;
    p.ok = cols <= 256 && ns >= 2;
    return p;
}

Plan make_plan(const Geometry &g, bool fp8, const TcTune *tune = nullptr) {
    if (tune && tune->chunk_rows > 0) {
        const Plan p = plan_for(g, fp8, tune->chunk_rows, tune->staged ? 1 : 0);
        if (p.ok) return p;
    }
    for (int staged = 1; staged >= 0; --staged)
        for (int rows = 128; rows >= 64; rows >>= 1) {
            const Plan p = plan_for(g, fp8, rows, staged);
            if (p.ok && (p.n_stages >= 3 || (!staged && rows == 64))) return p;
        }
    return Plan{};
}

bool shape_ok(const Geometry &g, bool fp8) {
    if (g.n_beams % 8 != 0 || g.n_beams < 8 || g.n_beams > 64) return false;
    if (fp8) {
        if (g.n_rx % 16 != 0 || g.n_rx < 16 || g.n_rx > kMaxRxFp8) return false;
    } else {
        if (g.n_rx % 8 != 0 || g.n_rx < 8 || g.n_rx > 1024) return false;
    }
    return make_plan(g, fp8).ok;
}

template <bool FP8>
cudaError_t launch_tc(const Geometry &g, int n_slots, const void *freq, const float *scales, const float2 *W,
                      float2 *beam, uint32_t *err_word, cudaStream_t st, const TcTune *tune) {
    if (n_slots == 0) return cudaSuccess;
    if (!shape_ok(g, FP8)) return cudaErrorNotSupported;
    if (reinterpret_cast<uintptr_t>(freq) % 16 != 0 || reinterpret_cast<uintptr_t>(beam) % 16 != 0)
        return cudaErrorMisalignedAddress;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const Plan p = make_plan(g, FP8, tune);
    const int K = 2 * g.n_rx;
    const long long rows = (long long)n_slots * g.n_sym;
    const int elem = FP8 ? 1 : 2;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)g.sc_pitch, (cuuint64_t)(rows * K)};
    cuuint64_t strides[1] = {(cuuint64_t)g.sc_pitch * elem};
    cuuint32_t box[2] = {(cuuint32_t)(FP8 ? 128 : 64), (cuuint32_t)p.chunk_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, FP8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
                     const_cast<void *>(freq), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    // output as floats [rows][n_sc][2 n_beams]: boxes of 16 floats x 32 subcarriers, 64-byte swizzle
    CUtensorMap omap;
    {
        cuuint64_t od[3] = {(cuuint64_t)(2 * g.n_beams), (cuuint64_t)g.n_sc, (cuuint64_t)rows};
        cuuint64_t os[2] = {(cuuint64_t)g.n_beams * 8, (cuuint64_t)g.n_sc * g.n_beams * 8};
        cuuint32_t ob[3] = {16, 32, 1};
        cuuint32_t oe[3] = {1, 1, 1};
        r = enc(&omap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, beam, od, os, ob, oe, CU_TENSOR_MAP_INTERLEAVE_NONE,
                CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    }
    TcArgs a;
    a.n_rx = g.n_rx;
    a.n_beams = g.n_beams;
    a.n_sc = g.n_sc;
    a.n_mtiles = (g.n_sc + kTileM - 1) / kTileM;
    a.n_blk = a.n_mtiles;
    a.K = K;
    a.N = 2 * g.n_beams;
    a.chunk_rows = p.chunk_rows;
    a.n_chunks = p.n_chunks;
    a.n_stages = p.n_stages;
    a.tmem_cols = p.tmem_cols;
    a.stage_bytes = p.stage_bytes;
    a.b_bytes = p.b_bytes;
    a.land_bytes = p.land_bytes;
    a.land_off = p.land_off;
    a.n_land = p.n_land;
    a.stage_out = p.stage_out;
    a.total_tiles = rows * a.n_mtiles;
    auto kern = beamform_tc_kernel<FP8>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = sms;
    if (grid > a.total_tiles) grid = a.total_tiles;
    kern<<<(unsigned)grid, FP8 ? 192 + 32 * kConvWarps : 192, p.smem, st>>>(map, omap, a, W, scales, beam, err_word);
    return cudaGetLastError();
}

}  // namespace

bool bf_tc_supported(const Geometry &g) { return shape_ok(g, false); }
bool bf_fp8_supported(const Geometry &g) { return shape_ok(g, true); }

int bf_tc_candidates(const Geometry &g, TcTune *out, int max_out) {
    const bool fp8 = g.form == PUSCH_FORM_FP8;
    if (g.form == PUSCH_FORM_FP32 || !shape_ok(g, fp8)) return 0;
    int n = 0, last_cr = -1, last_st = -1;
    for (int staged = 1; staged >= 0; --staged)
        for (int rows = 128; rows >= 64; rows >>= 1) {
            const Plan p = plan_for(g, fp8, rows, staged);
            if (!p.ok || (p.chunk_rows == last_cr && staged == last_st) || n >= max_out) continue;
            out[n].chunk_rows = p.chunk_rows;
            out[n].staged = staged;
            last_cr = p.chunk_rows;
            last_st = staged;
            ++n;
        }
    return n;
}

cudaError_t launch_beamform_tc(const Geometry &g, int n_slots, const __half *freq16, const float2 *W, float2 *beam,
                               uint32_t *err_word, cudaStream_t st, const TcTune *tune) {
    return launch_tc<false>(g, n_slots, freq16, nullptr, W, beam, err_word, st, tune);
}

cudaError_t launch_beamform_fp8(const Geometry &g, int n_slots, const uint8_t *freq8, const float *scales,
                                const float2 *W, float2 *beam, uint32_t *err_word, cudaStream_t st,
                                const TcTune *tune) {
    if (reinterpret_cast<uintptr_t>(scales) % 16 != 0) return cudaErrorMisalignedAddress;
    return launch_tc<true>(g, n_slots, freq8, scales, W, beam, err_word, st, tune);
}

}  // namespace pusch
