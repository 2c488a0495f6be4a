// Beamforming, plain FP32 form (Section II and Table I "BF": a matrix-matrix product with known
// coefficients, y = W^H x for every subcarrier and OFDM symbol).
//
// Per (slot, symbol) the product is Y[a][b] = sum_r conj(W[r][b]) X[r][a]: M = subcarriers, K = antennas,
// N = beams. Each CTA owns a tile of subcarriers and every beam; K is staged through shared memory in
// chunks of 32 antennas, and every thread accumulates a 2-subcarrier x 8-beam register block
// (16 complex accumulators), reading one 16-byte X pair and four 16-byte W pairs per antenna.
// The output row of a subcarrier (all beams) is contiguous, which is the layout detection reads.
#include "internal.cuh"

namespace pusch {
namespace {

constexpr int kBfThreads = 128;
constexpr int kBB = 8;   // beams per thread
constexpr int kSB = 2;   // subcarriers per thread
constexpr int kKC = 32;  // antennas per shared-memory chunk

template <int GB>  // beam groups of 8: ceil(n_beams / 8)
__global__ void __launch_bounds__(kBfThreads)
beamform_fp32_kernel(const float2 *__restrict__ freq, const float2 *__restrict__ W, float2 *__restrict__ beam,
                     int n_rx, int n_sc, int n_beams) {
    constexpr int TA = (kBfThreads / GB) * kSB;  // subcarriers per CTA
    constexpr int WB = GB * kBB;                 // padded beams
    __shared__ __align__(16) float2 Xs[kKC][TA];
    __shared__ __align__(16) float2 Ws[kKC][WB];

    const long long row = blockIdx.y;  // slot * n_sym + symbol
    const int a_base = blockIdx.x * TA;
    const int tid = threadIdx.x;
    const int bg = tid % GB;
    const int sg = tid / GB;
    const int sc0 = sg * kSB;
    const int b0 = bg * kBB;
    const float2 *X = freq + row * n_rx * (long long)n_sc;

    float2 acc[kSB][kBB];
#pragma unroll
    for (int i = 0; i < kSB; ++i)
#pragma unroll
        for (int j = 0; j < kBB; ++j) acc[i][j] = make_float2(0.f, 0.f);

    for (int r0 = 0; r0 < n_rx; r0 += kKC) {
        for (int idx = tid; idx < kKC * TA; idx += kBfThreads) {
            const int rr = idx / TA, aa = idx - rr * TA;
            const int r = r0 + rr, a = a_base + aa;
            Xs[rr][aa] = (r < n_rx && a < n_sc) ? __ldg(&X[(long long)r * n_sc + a]) : make_float2(0.f, 0.f);
        }
        for (int idx = tid; idx < kKC * WB; idx += kBfThreads) {
            const int rr = idx / WB, bb = idx - rr * WB;
            const int r = r0 + rr;
            Ws[rr][bb] = (r < n_rx && bb < n_beams) ? __ldg(&W[(long long)r * n_beams + bb]) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kKC; ++rr) {
            const float4 xv = *reinterpret_cast<const float4 *>(&Xs[rr][sc0]);
            const float2 x[2] = {make_float2(xv.x, xv.y), make_float2(xv.z, xv.w)};
            float2 w[kBB];
#pragma unroll
            for (int j = 0; j < kBB; j += 2) {
                const float4 wv = *reinterpret_cast<const float4 *>(&Ws[rr][b0 + j]);
                w[j] = make_float2(wv.x, wv.y);
                w[j + 1] = make_float2(wv.z, wv.w);
            }
#pragma unroll
            for (int i = 0; i < kSB; ++i)
#pragma unroll
                for (int j = 0; j < kBB; ++j) cfmac(acc[i][j], w[j], x[i]);
        }
        __syncthreads();
    }

    float2 *Y = beam + row * (long long)n_sc * n_beams;
#pragma unroll
    for (int i = 0; i < kSB; ++i) {
        const int a = a_base + sc0 + i;
        if (a >= n_sc) continue;
        float2 *dst = Y + (long long)a * n_beams;
        if (b0 + kBB <= n_beams && (n_beams % 2) == 0) {
#pragma unroll
            for (int j = 0; j < kBB; j += 2)
                *reinterpret_cast<float4 *>(dst + b0 + j) =
                    make_float4(acc[i][j].x, acc[i][j].y, acc[i][j + 1].x, acc[i][j + 1].y);
        } else {
#pragma unroll
            for (int j = 0; j < kBB; ++j)
                if (b0 + j < n_beams) dst[b0 + j] = acc[i][j];
        }
    }
}

template <int GB>
cudaError_t launch_gb(const Geometry &g, int n_slots, const float2 *freq, const float2 *W, float2 *beam,
                      cudaStream_t st) {
    constexpr int TA = (kBfThreads / GB) * kSB;
    const long long rows = (long long)n_slots * g.n_sym;
    if (rows > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((g.n_sc + TA - 1) / TA, (unsigned)rows);
    beamform_fp32_kernel<GB><<<grid, kBfThreads, 0, st>>>(freq, W, beam, g.n_rx, g.n_sc, g.n_beams);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_beamform_fp32(const Geometry &g, int n_slots, const float2 *freq, const float2 *W, float2 *beam,
                                 cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    const int gb = (g.n_beams + kBB - 1) / kBB;
    switch (gb) {
        case 1: return launch_gb<1>(g, n_slots, freq, W, beam, st);
        case 2: return launch_gb<2>(g, n_slots, freq, W, beam, st);
        case 3:
        case 4: return launch_gb<4>(g, n_slots, freq, W, beam, st);
        case 5:
        case 6:
        case 7:
        case 8: return launch_gb<8>(g, n_slots, freq, W, beam, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pusch
