// MMSE MIMO detection (Eq. 2), computed as in Section II: Gram G = H^H H + sigma^2 I, Cholesky
// G = L L^H (Section V-C), forward solve L z = H^H y, back solve L^H x = z; then Gray hard decisions.
//
// GB300 mapping: a group of NL lanes owns one subcarrier (NL = layer class 2..32, a power of two), so a
// warp detects 32/NL subcarriers at once. Lane i of a group owns row i of G, then row i of L, in
// registers. The factorisation is right-looking: at column j, lane j's pivot is broadcast with a warp
// shuffle, the lanes below scale their entry, and the trailing rows are updated with the column entries
// broadcast from their owner lanes. The solves run the same way, one shuffle per unknown. L's columns
// (needed by the back solve) are transposed once through shared memory. The estimate H of the warp's
// subcarriers is staged in shared memory (rows padded by one element against bank conflicts) and reused
// for the Gram and for H^H y of all 12 data symbols: G and L are formed once per subcarrier, which gives
// the same result as forming them per data symbol because the estimate is constant over the slot.
// Layers beyond n_layers (up to NL) are padded with identity rows and produce nothing.
#include "internal.cuh"

namespace pusch {
namespace {

constexpr int kMmseWarps = 4;
constexpr unsigned kFull = 0xffffffffu;

struct MmseArgs {
    int n_sc, n_beams, n_layers, n_sym, n_data, qam_bits;
    float load;  // sigma^2 + extra loading
    int data_sym[16];
};

__device__ __forceinline__ float2 shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(kFull, v.x, src), __shfl_sync(kFull, v.y, src));
}

__device__ __forceinline__ uint8_t demap(float2 x, int q) {
    const float thr = 0.63245553203367586640f;  // 2 / sqrt(10), rounded to float
    uint8_t v = (uint8_t)(x.x < 0.f) | (uint8_t)((x.y < 0.f) << 1);
    if (q == 4) v |= (uint8_t)((fabsf(x.x) > thr) << 2) | (uint8_t)((fabsf(x.y) > thr) << 3);
    return v;
}

template <int NL>
__host__ __device__ constexpr int mmse_warp_floats2(int nb) {
    // H rows (padded), L transpose tile, one y vector per subcarrier
    return (32 / NL) * NL * (nb + 1) + (32 / NL) * NL * (NL + 1) + (32 / NL) * nb;
}

template <int NL>
__global__ void __launch_bounds__(kMmseWarps * 32)
mmse_kernel(MmseArgs g, long long total_sc, const float2 *__restrict__ H, const float2 *__restrict__ beam,
            float2 *__restrict__ xhat, uint8_t *__restrict__ bits, uint32_t *__restrict__ status) {
    constexpr int SPW = 32 / NL;
    extern __shared__ float2 smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / NL, i = lane - grp * NL;
    const int src0 = grp * NL;
    const int nl = g.n_layers, nb = g.n_beams, n_sc = g.n_sc;
    const int hs = nb + 1;

    float2 *Hsm = smem + (size_t)warp * mmse_warp_floats2<NL>(nb);
    float2 *Lsm = Hsm + SPW * NL * hs;
    float2 *ysm = Lsm + SPW * NL * (NL + 1);

    const long long sc0 = ((long long)blockIdx.x * kMmseWarps + warp) * SPW;  // first (slot*n_sc + a) of warp
    if (sc0 >= total_sc) return;                                              // whole warp idle
    const long long my_sc = sc0 + grp;
    const bool valid = my_sc < total_sc;
    const long long slot = my_sc / n_sc;
    const int a = (int)(my_sc - slot * n_sc);

    // ---- stage H of the warp's subcarriers: [SPW][NL][nb] (zero rows beyond n_layers / total_sc)
    const int per_sc = nl * nb;
    for (int idx = lane; idx < SPW * NL * nb; idx += 32) {
        const int gg = idx / (NL * nb);
        const int rem = idx - gg * NL * nb;
        const int l = rem / nb, b = rem - l * nb;
        float2 v = make_float2(0.f, 0.f);
        if (l < nl && sc0 + gg < total_sc) v = __ldg(&H[(sc0 + gg) * per_sc + (long long)l * nb + b]);
        Hsm[(gg * NL + l) * hs + b] = v;
    }
    __syncwarp();

    const float2 *hrow = Hsm + (grp * NL + i) * hs;
    const float2 *hgrp = Hsm + (grp * NL) * hs;

    // ---- Gram row i: G[j] = sum_b conj(H[i][b]) H[j][b]
    float2 G[NL];
#pragma unroll
    for (int j = 0; j < NL; ++j) G[j] = make_float2(0.f, 0.f);
    for (int b = 0; b < nb; ++b) {
        const float2 hi = hrow[b];
#pragma unroll
        for (int j = 0; j < NL; ++j) cfmac(G[j], hi, hgrp[j * hs + b]);
    }
#pragma unroll
    for (int j = 0; j < NL; ++j)
        if (j == i) G[j] = (i < nl) ? make_float2(G[j].x + g.load, 0.f) : make_float2(1.f, 0.f);

    // ---- Cholesky, right-looking, row i of L replaces row i of G
    bool bad = false;
    float dinv = 1.f;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        float d = __shfl_sync(kFull, G[j].x, src0 + j);
        if (!(d > 0.f) || !isfinite(d)) {
            bad = true;
            d = 1.f;
        }
        const float ljj = sqrtf(d);
        const float inv = 1.f / ljj;
        if (i > j) G[j] = cscale(G[j], inv);
        else if (i == j) G[j] = make_float2(ljj, 0.f);
        else G[j] = make_float2(0.f, 0.f);
        if (i == j) dinv = inv;
#pragma unroll
        for (int k = j + 1; k < NL; ++k) {
            const float2 lkj = shfl2(G[j], src0 + k);
            if (i >= k) {
                // G[i][k] -= L[i][j] conj(L[k][j])
                G[k].x -= G[j].x * lkj.x + G[j].y * lkj.y;
                G[k].y -= G[j].y * lkj.x - G[j].x * lkj.y;
            }
        }
    }

    // ---- transpose: Lc[k] = L[k][i] (k > i) for the back solve
    float2 *lt = Lsm + grp * NL * (NL + 1);
#pragma unroll
    for (int k = 0; k < NL; ++k) lt[i * (NL + 1) + k] = G[k];
    __syncwarp();
    float2 Lc[NL];
#pragma unroll
    for (int k = 0; k < NL; ++k) Lc[k] = lt[k * (NL + 1) + i];

    if (valid && bad && i == 0) {
        atomicAdd(&status[1], 1u);
        atomicMin(&status[2], (unsigned)my_sc);
        atomicOr(&status[0], (unsigned)PUSCH_STATUS_PIVOT);
    }

    const int n_data = g.n_data;
    bool nonfinite = false;
    for (int d = 0; d < n_data; ++d) {
        const int s = g.data_sym[d];
        __syncwarp();
        for (int idx = lane; idx < SPW * nb; idx += 32) {
            const int gg = idx / nb, b = idx - gg * nb;
            const long long sc = sc0 + gg;
            float2 v = make_float2(0.f, 0.f);
            if (sc < total_sc) {
                const long long sl = sc / n_sc;
                const long long aa = sc - sl * n_sc;
                v = __ldg(&beam[((sl * g.n_sym + s) * n_sc + aa) * nb + b]);
            }
            ysm[gg * nb + b] = v;
        }
        __syncwarp();
        const float2 *y = ysm + grp * nb;
        float2 acc = make_float2(0.f, 0.f);
        for (int b = 0; b < nb; ++b) cfmac(acc, hrow[b], y[b]);

        // forward: L z = r
        float2 zi = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const float2 zk = shfl2(cscale(acc, dinv), src0 + k);
            if (i == k) zi = zk;
            if (i > k) cfms(acc, G[k], zk);
        }
        // back: L^H x = z
        acc = zi;
        float2 xi = make_float2(0.f, 0.f);
#pragma unroll
        for (int k = NL - 1; k >= 0; --k) {
            const float2 xk = shfl2(cscale(acc, dinv), src0 + k);
            if (i == k) xi = xk;
            if (i < k) {
                // acc -= conj(L[k][i]) x_k
                acc.x -= Lc[k].x * xk.x + Lc[k].y * xk.y;
                acc.y -= Lc[k].x * xk.y - Lc[k].y * xk.x;
            }
        }
        if (valid && i < nl) {
            const long long o = ((slot * nl + i) * n_data + d) * (long long)n_sc + a;
            xhat[o] = xi;
            bits[o] = demap(xi, g.qam_bits);
            if (!isfinite(xi.x) || !isfinite(xi.y)) nonfinite = true;
        }
    }
    if (__any_sync(kFull, nonfinite) && lane == 0) atomicOr(&status[0], (unsigned)PUSCH_STATUS_NONFINITE);
}

template <int NL>
cudaError_t launch_nl(const MmseArgs &a, long long total_sc, const float2 *H, const float2 *beam, float2 *xhat,
                      uint8_t *bits, uint32_t *status, cudaStream_t st) {
    constexpr int SPW = 32 / NL;
    const size_t smem = (size_t)kMmseWarps * mmse_warp_floats2<NL>(a.n_beams) * sizeof(float2);
    const long long per_cta = (long long)kMmseWarps * SPW;
    const long long grid = (total_sc + per_cta - 1) / per_cta;
    if (grid > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    auto k = mmse_kernel<NL>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<(unsigned)grid, kMmseWarps * 32, smem, st>>>(a, total_sc, H, beam, xhat, bits, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mmse(const Geometry &g, int n_slots, const float2 *H, const float2 *beam, float2 *x_hat,
                        uint8_t *bits, uint32_t *status, cudaStream_t st) {
    MmseArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.n_sym = g.n_sym;
    a.n_data = g.n_data;
    a.qam_bits = g.qam_bits;
    a.load = g.noise_var + g.loading;
    for (int d = 0; d < 16; ++d) a.data_sym[d] = g.data_sym[d];
    const long long total_sc = (long long)n_slots * g.n_sc;
    if (total_sc == 0) return cudaSuccess;
    const int nl = g.n_layers;
    if (nl <= 2) return launch_nl<2>(a, total_sc, H, beam, x_hat, bits, status, st);
    if (nl <= 4) return launch_nl<4>(a, total_sc, H, beam, x_hat, bits, status, st);
    if (nl <= 8) return launch_nl<8>(a, total_sc, H, beam, x_hat, bits, status, st);
    if (nl <= 16) return launch_nl<16>(a, total_sc, H, beam, x_hat, bits, status, st);
    return launch_nl<32>(a, total_sc, H, beam, x_hat, bits, status, st);
}

}  // namespace pusch
