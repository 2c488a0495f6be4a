// OFDM demodulation: batched forward FFTs of N_F = 64..4096 points with active-bin extraction
// (Section II: one FFT per antenna and OFDM symbol; Table I "OFDM dem.").
//
// Design (GB300): one FFT per group of T = N/E threads, each thread holding E = 8 or 16 complex values in
// registers. The transform is a Stockham auto-sort sequence of radix-16/8/4 passes, so that
//   * pass 1 reads its butterfly inputs (element t + T*e) from the shared-memory copy of the input row,
//   * the last pass leaves bin t + T*e in register e, written to global memory in natural order,
//   * the passes in between exchange through shared memory padded by one slot per 16 (conflict-free).
// 4096 = 16*16*16 therefore costs one global read, two shared-memory exchanges and one global write.
// CTAs are persistent: the next input rows arrive by bulk (TMA) copies into a one-stage ring, issued as soon
// as the current rows are in registers, so HBM reads overlap the arithmetic (four CTAs per SM for FP16 input).
// Twiddles come from a table exp(-2 pi i q / N) (computed in double precision).
#pragma once

#include <float.h>

#include "bounded_wait.cuh"
#include "internal.cuh"

namespace pusch {
namespace fft_detail {

enum : int { kOutC64 = 0, kOutF16 = 1, kOutE4M3 = 2 };

constexpr float kC8 = 0.70710678118654752440f;   // cos(pi/4)
constexpr float kC16 = 0.92387953251128675613f;  // cos(pi/8)
constexpr float kS16 = 0.38268343236508977173f;  // sin(pi/8)

// x * exp(-2 pi i q / 16) for a compile-time q in [0, 16)
template <int Q>
__device__ __forceinline__ float2 rot16(float2 x) {
    constexpr int q = Q & 15;
    if constexpr (q == 0) return x;
    else if constexpr (q == 4) return make_float2(x.y, -x.x);
    else if constexpr (q == 8) return make_float2(-x.x, -x.y);
    else if constexpr (q == 12) return make_float2(-x.y, x.x);
    else {
        constexpr float c[16] = {1.f, kC16, kC8, kS16, 0.f, -kS16, -kC8, -kC16,
                                 -1.f, -kC16, -kC8, -kS16, 0.f, kS16, kC8, kC16};
        constexpr float s[16] = {0.f, kS16, kC8, kC16, 1.f, kC16, kC8, kS16,
                                 0.f, -kS16, -kC8, -kC16, -1.f, -kC16, -kC8, -kS16};
        // multiply by (c - i s)
        return make_float2(x.x * c[q] + x.y * s[q], x.y * c[q] - x.x * s[q]);
    }
}

// Complex add / subtract as one packed FP32x2 instruction each (the subtraction as b * (-1) + a, which is
// exact in the product and rounds once, like a - b).
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

__device__ __forceinline__ void dft2(float2 &a, float2 &b) {
    float2 t = a;
    a = padd(t, b);
    b = psub(t, b);
}

// forward 4-point DFT in place
__device__ __forceinline__ void dft4(float2 &x0, float2 &x1, float2 &x2, float2 &x3) {
    const float2 a = padd(x0, x2), b = psub(x0, x2), c = padd(x1, x3), d = psub(x1, x3);
    x0 = padd(a, c);
    x2 = psub(a, c);
    const float2 id = make_float2(d.y, -d.x);  // -i d
    x1 = padd(b, id);                          // b - i d
    x3 = psub(b, id);                          // b + i d
}

// Forward R-point DFT of x[0..R) in natural order, R in {2, 4, 8, 16}.
// R = 8 and 16 are split as R = 4 * (R/4): n = (R/4)*n1 + n2, k = k1 + 4*k2.
template <int R>
__device__ __forceinline__ void dft(float2 (&x)[R]) {
    if constexpr (R == 2) {
        dft2(x[0], x[1]);
    } else if constexpr (R == 4) {
        dft4(x[0], x[1], x[2], x[3]);
    } else if constexpr (R == 8) {
        // inner DFT-4 over n1 for n2 = 0, 1 (stride-2 samples)
        dft4(x[0], x[2], x[4], x[6]);
        dft4(x[1], x[3], x[5], x[7]);
        float2 a1 = rot16<2>(x[3]), a2 = rot16<4>(x[5]), a3 = rot16<6>(x[7]);
        float2 y[8];
        y[0] = padd(x[0], x[1]); y[4] = psub(x[0], x[1]);
        y[1] = padd(x[2], a1);   y[5] = psub(x[2], a1);
        y[2] = padd(x[4], a2);   y[6] = psub(x[4], a2);
        y[3] = padd(x[6], a3);   y[7] = psub(x[6], a3);
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = y[i];
    } else if constexpr (R == 16) {
        // A[n2][k1] = DFT4_{n1}(x[4 n1 + n2]) stored back at x[4 k1 + n2]
        dft4(x[0], x[4], x[8], x[12]);
        dft4(x[1], x[5], x[9], x[13]);
        dft4(x[2], x[6], x[10], x[14]);
        dft4(x[3], x[7], x[11], x[15]);
        // twiddle A[n2][k1] by w16^(n2 k1)
        x[5] = rot16<1>(x[5]);  x[9] = rot16<2>(x[9]);   x[13] = rot16<3>(x[13]);
        x[6] = rot16<2>(x[6]);  x[10] = rot16<4>(x[10]); x[14] = rot16<6>(x[14]);
        x[7] = rot16<3>(x[7]);  x[11] = rot16<6>(x[11]); x[15] = rot16<9>(x[15]);
        // out[k1 + 4 k2] = DFT4_{n2}(A[n2][k1]); A[.][k1] sits at x[4 k1 .. 4 k1 + 3]
        dft4(x[0], x[1], x[2], x[3]);
        dft4(x[4], x[5], x[6], x[7]);
        dft4(x[8], x[9], x[10], x[11]);
        dft4(x[12], x[13], x[14], x[15]);
        float2 y[16];
#pragma unroll
        for (int k1 = 0; k1 < 4; ++k1)
#pragma unroll
            for (int k2 = 0; k2 < 4; ++k2) y[k1 + 4 * k2] = x[4 * k1 + k2];
#pragma unroll
        for (int i = 0; i < 16; ++i) x[i] = y[i];
    }
}

__device__ __forceinline__ int pad16(int p) { return p + (p >> 4); }

// One Stockham radix-R pass over the E register values of thread t (Ls = product of earlier radices).
// Butterfly j = t + u*T takes inputs j + m*N/R (register u + m*E/R) and twiddles input m by
// exp(-2 pi i (j mod Ls) m / (Ls R)).
template <int N, int E, int R, int LS>
__device__ __forceinline__ void fft_pass(float2 (&v)[E], const float2 *__restrict__ tw, int t) {
    constexpr int T = N / E;
    constexpr int NB = E / R;
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + u * T;
        const int k = j & (LS - 1);
        float2 x[R];
#pragma unroll
        for (int m = 0; m < R; ++m) x[m] = v[u + m * NB];
        if constexpr (LS > 1) {
            // w^m, m < R, from the table entries w^1..w^4 and at most two more products (<= 3 roundings)
            constexpr int S = N / (LS * R);
            float2 w[R];
            w[0] = make_float2(1.f, 0.f);
#pragma unroll
            for (int m = 1; m < R && m <= 4; ++m) w[m] = __ldg(&tw[(k * m) * S]);
            if constexpr (R > 5) {
                const float2 w8 = cmul(w[4], w[4]);
                const float2 w12 = cmul(w8, w[4]);
#pragma unroll
                for (int m = 5; m < R; ++m) {
                    const int a4 = m >> 2, b = m & 3;
                    const float2 base = a4 == 1 ? w[4] : (a4 == 2 ? w8 : w12);
                    w[m] = b == 0 ? base : cmul(base, w[b]);
                }
            }
#pragma unroll
            for (int m = 1; m < R; ++m) x[m] = cmul(x[m], w[m]);
        }
        dft<R>(x);
#pragma unroll
        for (int m = 0; m < R; ++m) v[u + m * NB] = x[m];
    }
}

// Stockham output placement of a non-final pass, then gather of the next pass's inputs t + T*e.
template <int N, int E, int R, int LS>
__device__ __forceinline__ void fft_exchange(float2 (&v)[E], float2 *sm, int t) {
    constexpr int T = N / E;
    constexpr int NB = E / R;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
        const int j = t + u * T;
        const int k = j & (LS - 1);
        const int base = (j - k) * R + k;
#pragma unroll
        for (int m = 0; m < R; ++m) sm[pad16(base + m * LS)] = v[u + m * NB];
    }
    __syncthreads();
#pragma unroll
    for (int e = 0; e < E; ++e) v[e] = sm[pad16(t + T * e)];
}

template <int N, int E, int LS, int R, int... Rest>
__device__ __forceinline__ void fft_run(float2 (&v)[E], float2 *sm, const float2 *__restrict__ tw, int t) {
    fft_pass<N, E, R, LS>(v, tw, t);
    if constexpr (sizeof...(Rest) > 0) {
        fft_exchange<N, E, R, LS>(v, sm, t);
        fft_run<N, E, LS * R, Rest...>(v, sm, tw, t);
    }
}

template <int N> struct Plan;
template <> struct Plan<4096> { static constexpr int E = 16; };
template <> struct Plan<2048> { static constexpr int E = 16; };
template <> struct Plan<1024> { static constexpr int E = 16; };
template <> struct Plan<512> { static constexpr int E = 8; };
template <> struct Plan<256> { static constexpr int E = 16; };
template <> struct Plan<128> { static constexpr int E = 16; };
template <> struct Plan<64> { static constexpr int E = 8; };

template <int N>
__device__ __forceinline__ void fft_full(float2 (&v)[Plan<N>::E], float2 *sm, const float2 *__restrict__ tw, int t) {
    constexpr int E = Plan<N>::E;
    if constexpr (N == 4096) fft_run<N, E, 1, 16, 16, 16>(v, sm, tw, t);
    else if constexpr (N == 2048) fft_run<N, E, 1, 16, 16, 8>(v, sm, tw, t);
    else if constexpr (N == 1024) fft_run<N, E, 1, 16, 16, 4>(v, sm, tw, t);
    else if constexpr (N == 512) fft_run<N, E, 1, 8, 8, 8>(v, sm, tw, t);
    else if constexpr (N == 256) fft_run<N, E, 1, 16, 16>(v, sm, tw, t);
    else if constexpr (N == 128) fft_run<N, E, 1, 16, 8>(v, sm, tw, t);
    else if constexpr (N == 64) fft_run<N, E, 1, 8, 8>(v, sm, tw, t);
}

__device__ __forceinline__ float2 to_f2(float2 v) { return v; }
__device__ __forceinline__ float2 to_f2(__half2 v) { return __half22float2(v); }

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

using bw::mbar_init;
using bw::mbar_try_wait;

// Bounded wait (the library's 2 s limit, bounded_wait.cuh); false on expiry.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    return bw::mbar_wait_for(bar, parity, bw::kWaitNs);
}

// Bulk (TMA, non-tensor) copies global -> shared completing on an mbarrier: 16-byte aligned, size % 16 == 0.
// bulk_expect announces the bytes of all copies of one phase, bulk_copy issues one of them.
__device__ __forceinline__ void bulk_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    bulk_expect(bar, bytes);
    bulk_copy(dst, src, bytes, bar);
}

// Where the input rows are. cp == 0: row r (= (slot * n_sym + sym) * n_rx + rx) at r * N. cp == 1: one stream
// of slot_len samples per (slot, antenna) with NR normal cyclic prefixes; the useful part of symbol s starts at
// s * (N + cp1) + cp0. shift == 1: sample n of the useful part is multiplied by exp(-2 pi i n / (4 N)) (table
// entries N + n) to undo the 7.5 kHz shift.
struct FftIn {
    int cp, cp0, cp1, shift, n_sym, n_rx;
    long long slot_len;
};
__device__ __forceinline__ long long fft_row_offset(const FftIn &fi, int N, long long row) {
    if (!fi.cp) return row * N;
    const long long sr = row / fi.n_rx;
    const int rx = (int)(row - sr * fi.n_rx);
    const long long slot = sr / fi.n_sym;
    const int sym = (int)(sr - slot * fi.n_sym);
    return (slot * fi.n_rx + rx) * fi.slot_len + (long long)sym * (N + fi.cp1) + fi.cp0;
}

constexpr int kFftThreads = 256;

template <int N>
constexpr int ffts_per_cta() {
    return (kFftThreads / (N / Plan<N>::E)) > 0 ? kFftThreads / (N / Plan<N>::E) : 1;
}

// One ring stage: the next row's copy is issued as soon as every thread has loaded the current row into
// registers, so it still overlaps the transform, and the smaller footprint fits one more CTA per SM
// (FP16 input: 4 x 51 KB; c64 input: 3 x 67 KB).
template <typename TIn>
constexpr int fft_stages() { return 1; }
template <typename TIn>
constexpr int fft_min_ctas() { return sizeof(TIn) == 4 ? 4 : 3; }

template <int N, typename TIn>
constexpr size_t fft_smem_bytes() {
    return (size_t)fft_stages<TIn>() * ffts_per_cta<N>() * N * sizeof(TIn)        // input ring
           + (size_t)ffts_per_cta<N>() * (N + N / 16) * sizeof(float2)             // exchange buffer
           + 8 * fft_stages<TIn>() + 16;                                           // mbarriers
}

// Two floats to two E4M3 codes, round to nearest even, saturating to +-448: the low byte holds lo.
__device__ __forceinline__ uint32_t e4m3x2_of(float lo, float hi) {
    uint16_t r;
    asm("cvt.rn.satfinite.e4m3x2.f32 %0, %1, %2;" : "=h"(r) : "f"(hi), "f"(lo));
    return r;
}

// Smallest e with amax <= 448 * 2^e (power-of-two E4M3 block scale), clamped below at -126; 128 when
// amax is not finite. From the float's bits: amax = 1.m * 2^(E - 127) and 448 = 1.75 * 2^8.
__device__ __forceinline__ int e4m3_block_exp(float amax) {
    if (!(amax <= FLT_MAX)) return 128;
    const uint32_t u = __float_as_uint(amax);
    const int eb = (int)(u >> 23);
    if (eb == 0) return -126;
    const int e = eb - 135 + ((u & 0x7FFFFFu) > 0x600000u ? 1 : 0);
    return e < -126 ? -126 : e;
}

// Persistent batched FFT. rows = n_slots * n_sym * n_rx transforms; each CTA iterates over blocks of F
// consecutive rows (one contiguous span of F*N input samples). The spans arrive by bulk copies into a
// ring of STAGES shared-memory buffers issued STAGES-1 blocks ahead, so HBM reads overlap the passes.
// OUT = kOutC64: c64 [rows][n_sc]. OUT = kOutF16: binary16 [rows][2][pitch] (re plane, im plane; pads
// zeroed), staged through shared memory for 16-byte stores. OUT = kOutE4M3: E4M3 codes [rows][2][pitch]
// (pads zero) and, per 128-subcarrier block, the power-of-two scale 2^e with e the smallest exponent
// for which the block's largest |re|, |im| is at most 448 * 2^e; codes = round-to-nearest-even E4M3 of
// value * 2^-e. Scales go to scales[(row / n_rx) * n_blk + blk][row % n_rx] (NaN for a block holding a
// non-finite value). Each warp quantises one (FFT, block): 4 subcarriers per lane.
// Four 256-thread CTAs per SM for FP16 input (registers capped at 64, 51 KB of shared memory each), three for
// c64 input: 32 (24) warps hide the exchange barriers while the next row per CTA streams in.
// OPT: the input options (prefixed streams, shift) are compiled in; without them the kernel is the plain
// contiguous-row transform.
template <int N, typename TIn, int OUT, bool OPT>
__global__ void __launch_bounds__(kFftThreads, fft_min_ctas<TIn>())
fft_kernel(const TIn *__restrict__ in, void *__restrict__ out, const float2 *__restrict__ tw, long long rows,
           int n_sc, int pitch, float *__restrict__ scales, int n_rx, int n_blk, uint32_t *__restrict__ err,
           FftIn fi) {
    constexpr int E = Plan<N>::E;
    constexpr int T = N / E;
    constexpr int F = ffts_per_cta<N>();
    constexpr int STAGES = fft_stages<TIn>();
    constexpr uint32_t kSpan = (uint32_t)F * N * sizeof(TIn);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TIn *ring = reinterpret_cast<TIn *>(smem_raw);
    float2 *xbuf = reinterpret_cast<float2 *>(smem_raw + (size_t)STAGES * kSpan);
    const uint32_t bar0 = smem_u32(smem_raw + (size_t)STAGES * kSpan + (size_t)F * (N + N / 16) * sizeof(float2));
    __shared__ int s_abort;

    const int f = threadIdx.x / T;
    const int t = threadIdx.x - f * T;
    float2 *sm = xbuf + f * (N + N / 16);
    const long long n_blocks = (rows + F - 1) / F;
    const long long n_my = n_blocks > blockIdx.x ? (n_blocks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    auto issue = [&](long long it) {
        const long long blk = blockIdx.x + it * gridDim.x;
        const long long r0 = blk * F;
        const long long nr = rows - r0 < F ? rows - r0 : F;
        const int s = (int)(it % STAGES);
        if (!OPT || !fi.cp) {  // the block's rows are one contiguous span
            bulk_load(smem_u32(ring) + s * kSpan, in + r0 * N, (uint32_t)(nr * N * sizeof(TIn)), bar0 + 8 * s);
        } else {       // one copy per row, out of the antennas' streams
            bulk_expect(bar0 + 8 * s, (uint32_t)(nr * N * sizeof(TIn)));
            for (int f = 0; f < (int)nr; ++f)
                bulk_copy(smem_u32(ring) + s * kSpan + (uint32_t)(f * N * sizeof(TIn)), in + fft_row_offset(fi, N, r0 + f),
                          (uint32_t)(N * sizeof(TIn)), bar0 + 8 * s);
        }
    };
    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(bar0 + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        for (long long it = 0; it < (STAGES > 1 ? STAGES - 1 : 1) && it < n_my; ++it) issue(it);

    const int h = n_sc >> 1;
    long long it = 0;
    for (; it < n_my; ++it) {
        const int s = (int)(it % STAGES);
        const bool ok = mbar_wait(bar0 + 8 * s, (uint32_t)((it / STAGES) & 1));
        if (__syncthreads_or(!ok)) {
            if (threadIdx.x == 0) {
                s_abort = 1;
                if (err) atomicOr(err, kErrFftWait);
            }
            break;
        }
        // the ring slot consumed by the previous block is free (all threads passed a barrier since, after the
        // proxy fence that follows their reads of it)
        if (STAGES > 1 && threadIdx.x == 0 && it + STAGES - 1 < n_my) issue(it + STAGES - 1);

        const long long row = (blockIdx.x + it * gridDim.x) * F + f;
        const bool valid = row < rows;
        const TIn *src = ring + (size_t)s * F * N + (size_t)f * N;
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = to_f2(src[t + T * e]);
        if constexpr (STAGES == 1) {
            // every thread holds its row in registers: the single ring slot takes the next block's copy. The
            // proxy fence orders this thread's generic reads of the slot before the bulk copy (async proxy)
            // that overwrites it; without it the copy could land before every read had completed.
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (threadIdx.x == 0 && it + 1 < n_my) issue(it + 1);
        }
        if (OPT && fi.shift) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cmul(v[e], __ldg(&tw[N + t + T * e]));
        }
        fft_full<N>(v, sm, tw, t);

        if constexpr (OUT == kOutC64) {
            if (valid) {
                float2 *dst = static_cast<float2 *>(out) + row * n_sc;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int a = t + T * e + h;
                    if (a >= N) a -= N;
                    if (a < n_sc) dst[a] = v[e];
                }
            }
        } else if constexpr (OUT == kOutF16) {
            // direct 2-byte stores of the two planes: consecutive threads hold consecutive bins, so each warp
            // writes 64 contiguous bytes of each plane per register (no staging, no barrier)
            if (valid) {
                __half *o = static_cast<__half *>(out) + row * 2 * (long long)pitch;
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    int a = t + T * e + h;
                    if (a >= N) a -= N;
                    if (a < n_sc) {
                        const __half2 hv = __floats2half2_rn(v[e].x, v[e].y);
                        o[a] = __low2half(hv);
                        o[pitch + a] = __high2half(hv);
                    }
                }
                for (int a = n_sc + t; a < pitch; a += T) {
                    o[a] = __float2half_rn(0.f);
                    o[pitch + a] = __float2half_rn(0.f);
                }
            }
        } else {
            // stage this FFT's active bins (FP32) in its exchange buffer, then quantise block by block
            __syncthreads();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                int a = t + T * e + h;
                if (a >= N) a -= N;
                if (a < n_sc) sm[a] = v[e];
            }
            __syncthreads();
            const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
            const long long row0 = (blockIdx.x + it * gridDim.x) * F;
            constexpr int kWarps = kFftThreads / 32;
            // one (FFT, 128-subcarrier block) job per warp at a time: block maximum, exponent, codes
            auto quantise = [&](const float2 *sb, unsigned rw32, unsigned srow, unsigned ant, int blk) {
                float2 q[4];
                float m = 0.f;
                bool bad = false;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int a = blk * 128 + lane + 32 * j;          // consecutive lanes, consecutive banks
                    q[j] = a < n_sc ? sb[a] : make_float2(0.f, 0.f);
                    const float ax = fabsf(q[j].x), ay = fabsf(q[j].y);
                    bad |= !(ax <= FLT_MAX) || !(ay <= FLT_MAX);
                    m = fmaxf(m, fmaxf(ax, ay));
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
                const bool anybad = __any_sync(0xFFFFFFFFu, bad);
                const int ex = anybad ? 128 : e4m3_block_exp(m);
                if (lane == 0)
                    scales[((size_t)srow * n_blk + blk) * n_rx + ant] =
                        anybad ? __uint_as_float(0x7FC00000u) : __uint_as_float((uint32_t)(ex + 127) << 23);
                const float inv = anybad ? 1.f : __uint_as_float((uint32_t)(127 - ex) << 23);   // 2^-e
                const float2 inv2 = make_float2(inv, inv);
                uint8_t *o8 = static_cast<uint8_t *>(out) + (size_t)rw32 * 2 * pitch;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int a = blk * 128 + lane + 32 * j;
                    if (a < pitch) {
                        // one conversion per complex value: low byte = re code, high byte = im code
                        const float2 sv = __fmul2_rn(q[j], inv2);
                        const uint32_t c = e4m3x2_of(sv.x, sv.y);
                        o8[a] = (uint8_t)(c & 0xFFu);
                        o8[pitch + a] = (uint8_t)(c >> 8);
                    }
                }
            };
            if constexpr (F == 1) {
                // one FFT per CTA: a warp's blocks warp, warp + 8, ... (at most 4 for 4096 points) are
                // processed together so that their loads, reductions and stores overlap
                if (row0 < rows) {
                    const unsigned rw32 = (unsigned)row0;                // rows < 2^31 (host check)
                    const unsigned srow = rw32 / (unsigned)n_rx, ant = rw32 - srow * (unsigned)n_rx;
                    uint8_t *o8 = static_cast<uint8_t *>(out) + (size_t)rw32 * 2 * pitch;
                    constexpr int kJ = (N / 128 + kWarps - 1) / kWarps > 0 ? (N / 128 + kWarps - 1) / kWarps : 1;
                    float2 q[kJ][4];
                    float m[kJ];
                    bool bad[kJ];
#pragma unroll
                    for (int g4 = 0; g4 < kJ; ++g4) {
                        const int blk = warp + g4 * kWarps;
                        m[g4] = 0.f;
                        bad[g4] = false;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int a = blk * 128 + lane + 32 * j;
                            q[g4][j] = (blk < n_blk && a < n_sc) ? xbuf[a] : make_float2(0.f, 0.f);
                            const float ax = fabsf(q[g4][j].x), ay = fabsf(q[g4][j].y);
                            bad[g4] |= !(ax <= FLT_MAX) || !(ay <= FLT_MAX);
                            m[g4] = fmaxf(m[g4], fmaxf(ax, ay));
                        }
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                        for (int g4 = 0; g4 < kJ; ++g4) m[g4] = fmaxf(m[g4], __shfl_xor_sync(0xFFFFFFFFu, m[g4], o));
#pragma unroll
                    for (int g4 = 0; g4 < kJ; ++g4) {
                        const int blk = warp + g4 * kWarps;
                        const bool anybad = __any_sync(0xFFFFFFFFu, bad[g4]);
                        if (blk >= n_blk) continue;                      // warp-uniform
                        const int ex = anybad ? 128 : e4m3_block_exp(m[g4]);
                        if (lane == 0)
                            scales[((size_t)srow * n_blk + blk) * n_rx + ant] =
                                anybad ? __uint_as_float(0x7FC00000u) : __uint_as_float((uint32_t)(ex + 127) << 23);
                        const float inv = anybad ? 1.f : __uint_as_float((uint32_t)(127 - ex) << 23);   // 2^-e
                        const float2 inv2 = make_float2(inv, inv);
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int a = blk * 128 + lane + 32 * j;
                            if (a < pitch) {
                                const float2 sv = __fmul2_rn(q[g4][j], inv2);
                                const uint32_t c = e4m3x2_of(sv.x, sv.y);    // low byte re, high byte im
                                o8[a] = (uint8_t)(c & 0xFFu);
                                o8[pitch + a] = (uint8_t)(c >> 8);
                            }
                        }
                    }
                }
            } else {
                for (int p = warp; p < F * n_blk; p += kWarps) {
                    const int ff = p / n_blk, blk = p - ff * n_blk;
                    if (row0 + ff >= rows) continue;                     // warp-uniform
                    const unsigned rw32 = (unsigned)(row0 + ff);
                    const unsigned srow = rw32 / (unsigned)n_rx, ant = rw32 - srow * (unsigned)n_rx;
                    quantise(xbuf + ff * (N + N / 16), rw32, srow, ant, blk);
                }
            }
        }
    }
    if (s_abort && threadIdx.x == 0) {
        // drain the copies still in flight (bounded) before the CTA exits
        for (long long j = it; j < it + (STAGES > 1 ? STAGES - 1 : 1) && j < n_my; ++j)
            mbar_wait(bar0 + 8 * (int)(j % STAGES), (uint32_t)((j / STAGES) & 1));
    }
}

template <int N, typename TIn, int OUT>
cudaError_t launch_n(long long rows, const void *in, void *out, const float2 *tw, int n_sc, int pitch, float *scales,
                     int n_rx, int n_blk, uint32_t *err, const FftIn &fi, cudaStream_t st, int cap) {
    constexpr int F = ffts_per_cta<N>();
    constexpr size_t smem = fft_smem_bytes<N, TIn>();
    static_assert(smem <= 227 * 1024, "FFT shared memory");
    auto k = (fi.cp || fi.shift) ? fft_kernel<N, TIn, OUT, true> : fft_kernel<N, TIn, OUT, false>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kFftThreads, smem);
    if (per_sm < 1) per_sm = 1;
    if (cap > 0 && per_sm > cap) per_sm = cap;     // tuned CTAs per SM
    const long long blocks = (rows + F - 1) / F;
    long long grid = (long long)sms * per_sm;
    if (grid > blocks) grid = blocks;
    k<<<(unsigned)grid, kFftThreads, smem, st>>>(static_cast<const TIn *>(in), out, tw, rows, n_sc, pitch, scales,
                                                  n_rx, n_blk, err, fi);
    return cudaGetLastError();
}

// All transform sizes for one input type and output format.
template <typename TIn, int OUT>
cudaError_t launch_out(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw, float *scales,
                       uint32_t *err, cudaStream_t st) {
    const int n_blk = (g.n_sc + 127) / 128;
    FftIn fi;
    fi.cp = g.cp;
    fi.cp0 = g.cp0;
    fi.cp1 = g.cp1;
    fi.shift = g.shift;
    fi.n_sym = g.n_sym;
    fi.n_rx = g.n_rx;
    fi.slot_len = g.slot_len;
    switch (g.n_fft) {
        case 4096: return launch_n<4096, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 2048: return launch_n<2048, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 1024: return launch_n<1024, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 512: return launch_n<512, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 256: return launch_n<256, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 128: return launch_n<128, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        case 64: return launch_n<64, TIn, OUT>(rows, in, out, tw, g.n_sc, g.sc_pitch, scales, g.n_rx, n_blk, err, fi, st, g.fft_cap);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fft_detail

// One entry per output format (separate translation units, compiled in parallel).
cudaError_t launch_fft_c64(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                           float *scales, uint32_t *err, cudaStream_t st);
cudaError_t launch_fft_f16(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                           float *scales, uint32_t *err, cudaStream_t st);
cudaError_t launch_fft_e4m3(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                            float *scales, uint32_t *err, cudaStream_t st);

}  // namespace pusch
