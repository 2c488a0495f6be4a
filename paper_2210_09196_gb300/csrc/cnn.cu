// Learned channel-estimate denoiser: four 3x3 same-padded convolutions 2 -> 32 -> 32 -> 32 -> 2, ReLU after
// the first three, the input added to the output; the kernels are dilated along the subcarriers by 1, 8, 16, 1
// (receptive field +-26 subcarriers, several pilot spacings). Grids are [n][c][2][w]: n grids (one per slot, layer and
// beam), c channels (re, im of the estimate at the input and output), the two DMRS symbols as rows and w
// subcarriers. Weights and activations are stored as bfloat16, arithmetic and gradients are FP32, the
// optimiser keeps FP32 master weights. Parameters are packed per layer as W[co][ci][3][3] then b[co].
//
// Kernels: conv3x3 (forward with ReLU or residual epilogue; also the input-gradient pass as a convolution
// with transposed, flipped weights and a ReLU-mask epilogue), conv3x3_wgrad (weight and bias gradients,
// persistent CTAs reducing in registers, one atomic add per weight per CTA), MSE loss gradient, Adam, and
// for the receive chain: the per-DMRS-symbol LS grid builder and the estimate writer with the
// pilot-residual fallback to the plain LS estimate.
#include <cuda_bf16.h>

#include "chest_common.cuh"

namespace pusch {
namespace {

constexpr int kConvThreads = 128;
constexpr int kCh[5] = {2, 32, 32, 32, 2};
constexpr int kDil[4] = {1, 8, 16, 1};   // kernel dilation along the subcarriers, per layer
constexpr int kMaxDil = 16;

__device__ __forceinline__ float ldv(const __nv_bfloat16 *p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldv(const float *p) { return *p; }

enum ConvOut { kOutReluBf16 = 0, kOutResidF32 = 1, kOutMaskF32 = 2 };

template <int CIN, int COUT>
struct ConvGeom {
    static constexpr int CPT = COUT < 8 ? COUT : 8;   // output channels per thread
    static constexpr int COG = COUT / CPT;             // channel groups
    static constexpr int CGS = kConvThreads / COG;     // column groups
    static constexpr int WPT = COUT >= 8 ? 4 : 1;      // output columns per thread (tiles of 128 columns)
    static constexpr int TW = CGS * WPT;               // tile width
    static size_t smem(int dil) { return (size_t)(COUT * CIN * 9 + CIN * 2 * (TW + 2 * dil)) * sizeof(float); }
};

// out[s][co][h][x] = b[co] + sum_{ci, kh, kw} W[co][ci][kh][kw] in[s][ci][h + kh - 1][x + (kw - 1) dil]
//   kOutReluBf16: out (bf16) = relu(.)
//   kOutResidF32: out (f32)  = . + aux[s][co][h][x]          (aux: the CNN input, bf16)
//   kOutMaskF32 : out (f32)  = aux[s][co][h][x] > 0 ? . : 0   (aux: an activation, bf16; b is NULL)
// in has rows of in_ld elements, out and aux rows of out_ld (the grid width w <= both).
template <int CIN, int COUT, typename TIn, int MODE>
__global__ void __launch_bounds__(kConvThreads)
conv3x3_kernel(const TIn *__restrict__ in, const __nv_bfloat16 *__restrict__ W, const __nv_bfloat16 *__restrict__ b,
               void *__restrict__ out, const __nv_bfloat16 *__restrict__ aux, int w, int dil, int in_ld, int out_ld) {
    using G = ConvGeom<CIN, COUT>;
    constexpr int CPT = G::CPT, COG = G::COG, TW = G::TW, kWPT = G::WPT;
    extern __shared__ float sm[];
    const int TP = TW + 2 * dil;         // tile with halo
    float *sW = sm;                      // [COUT][CIN][9]
    float *sX = sm + COUT * CIN * 9;     // [CIN][2][TP], column c <-> x = x0 + c - dil
    const long long s = blockIdx.y;
    const int x0 = blockIdx.x * TW;
    for (int i = threadIdx.x; i < COUT * CIN * 9; i += kConvThreads) sW[i] = __bfloat162float(W[i]);
    for (int i = threadIdx.x; i < CIN * 2 * TP; i += kConvThreads) {
        const int ci = i / (2 * TP);
        const int rem = i - ci * 2 * TP;
        const int h = rem / TP;
        const int xx = rem - h * TP + x0 - dil;
        sX[i] = (xx >= 0 && xx < w) ? ldv(in + ((s * CIN + ci) * 2 + h) * (long long)in_ld + xx) : 0.f;
    }
    __syncthreads();
    const int cg = threadIdx.x % COG;
    const int xl = (threadIdx.x / COG) * kWPT;
    const int co0 = cg * CPT;
    float acc[2][kWPT][CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const float bv = b ? __bfloat162float(b[co0 + c]) : 0.f;
#pragma unroll
        for (int j = 0; j < kWPT; ++j) acc[0][j][c] = acc[1][j][c] = bv;
    }
    for (int ci = 0; ci < CIN; ++ci) {
        float xv[2][3][kWPT];  // [row][tap][column]
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int kw = 0; kw < 3; ++kw)
#pragma unroll
                for (int j = 0; j < kWPT; ++j) xv[h][kw][j] = sX[(ci * 2 + h) * TP + xl + j + kw * dil];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const float *wp = sW + ((co0 + c) * CIN + ci) * 9;
            float wv[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) wv[k] = wp[k];
#pragma unroll
            for (int j = 0; j < kWPT; ++j)
#pragma unroll
                for (int kw = 0; kw < 3; ++kw) {
                    // output row 0 reads input rows 0 (kh = 1) and 1 (kh = 2); row 1 reads 0 (kh = 0) and 1 (kh = 1)
                    acc[0][j][c] = fmaf(wv[3 + kw], xv[0][kw][j], fmaf(wv[6 + kw], xv[1][kw][j], acc[0][j][c]));
                    acc[1][j][c] = fmaf(wv[0 + kw], xv[0][kw][j], fmaf(wv[3 + kw], xv[1][kw][j], acc[1][j][c]));
                }
        }
    }
#pragma unroll
    for (int j = 0; j < kWPT; ++j) {
        const int x = x0 + xl + j;
        if (x >= w) continue;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long long idx = ((s * COUT + co0 + c) * 2 + h) * (long long)out_ld + x;
                const float v = acc[h][j][c];
                if constexpr (MODE == kOutReluBf16) {
                    static_cast<__nv_bfloat16 *>(out)[idx] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
                } else if constexpr (MODE == kOutResidF32) {
                    static_cast<float *>(out)[idx] = v + __bfloat162float(aux[idx]);
                } else {
                    static_cast<float *>(out)[idx] = __bfloat162float(aux[idx]) > 0.f ? v : 0.f;
                }
            }
    }
}

template <int CIN, int COUT, typename TIn, int MODE>
cudaError_t launch_conv(const TIn *in, const __nv_bfloat16 *W, const __nv_bfloat16 *b, void *out,
                        const __nv_bfloat16 *aux, int n, int w, int dil, cudaStream_t st, int in_ld = 0,
                        int out_ld = 0) {
    if (in_ld <= 0) in_ld = w;
    if (out_ld <= 0) out_ld = w;
    using G = ConvGeom<CIN, COUT>;
    auto k = conv3x3_kernel<CIN, COUT, TIn, MODE>;
    const size_t smem = G::smem(dil);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem(kMaxDil));
        if (e != cudaSuccess) return e;
    }
    if (n > 65535) return cudaErrorInvalidConfiguration;
    dim3 grid((w + G::TW - 1) / G::TW, n);
    k<<<grid, kConvThreads, smem, st>>>(in, W, b, out, aux, w, dil, in_ld, out_ld);
    return cudaGetLastError();
}

// dW[co][ci][kh][kw] += sum_{s, h, x} g[s][co][h][x] in[s][ci][h + kh - 1][x + (kw - 1) dil];  db[co] += sum g.
// Persistent CTAs over (grid, 64-column tile) pairs; thread t owns input channel ci = t % CIN and COPT
// consecutive output channels, accumulating 9 taps each in registers; one atomic add per weight per CTA.
constexpr int kWgThreads = 256;
constexpr int kWgTW = 64;

template <int CIN, int COUT, typename TIn>
__global__ void __launch_bounds__(kWgThreads)
conv3x3_wgrad_kernel(const float *__restrict__ g, const TIn *__restrict__ in, float *__restrict__ dW,
                     float *__restrict__ db, int n, int w, int dil) {
    constexpr int PAIRS = COUT * CIN;
    constexpr int COPT = PAIRS >= 4 * kWgThreads ? 4 : 1;
    constexpr int ACTIVE = PAIRS / COPT;
    __shared__ float sG[COUT][2][kWgTW];
    __shared__ float sI[CIN][2][kWgTW + 2 * kMaxDil];  // column c <-> x = x0 + c - dil
    const int t = threadIdx.x;
    const bool act = t < ACTIVE;
    const int ci = t % CIN;
    const int cq = t / CIN;
    float acc[COPT][9];
    float accb[COPT];
#pragma unroll
    for (int c = 0; c < COPT; ++c) {
        accb[c] = 0.f;
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[c][k] = 0.f;
    }
    const int tiles_w = (w + kWgTW - 1) / kWgTW;
    const long long tiles = (long long)n * tiles_w;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const long long s = tile / tiles_w;
        const int x0 = (int)(tile - s * tiles_w) * kWgTW;
        __syncthreads();
        for (int i = t; i < COUT * 2 * kWgTW; i += kWgThreads) {
            const int co = i / (2 * kWgTW), rem = i - co * 2 * kWgTW, h = rem / kWgTW, x = rem - h * kWgTW + x0;
            sG[co][h][rem - h * kWgTW] = x < w ? g[((s * COUT + co) * 2 + h) * (long long)w + x] : 0.f;
        }
        const int TP = kWgTW + 2 * dil;
        for (int i = t; i < CIN * 2 * TP; i += kWgThreads) {
            const int c = i / (2 * TP), rem = i - c * 2 * TP, h = rem / TP;
            const int x = rem - h * TP + x0 - dil;
            sI[c][h][rem - h * TP] = (x >= 0 && x < w) ? ldv(in + ((s * CIN + c) * 2 + h) * (long long)w + x) : 0.f;
        }
        __syncthreads();
        if (act) {
            for (int x = 0; x < kWgTW; ++x) {
                float iv[2][3];
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int kw = 0; kw < 3; ++kw) iv[h][kw] = sI[ci][h][x + kw * dil];
#pragma unroll
                for (int c = 0; c < COPT; ++c) {
                    const int co = cq * COPT + c;
                    const float g0 = sG[co][0][x], g1 = sG[co][1][x];
                    if (ci == 0) accb[c] += g0 + g1;
#pragma unroll
                    for (int kw = 0; kw < 3; ++kw) {
                        // row 0 of g meets input rows 0 (kh = 1) and 1 (kh = 2); row 1 meets rows 0 (kh = 0), 1 (kh = 1)
                        acc[c][3 + kw] = fmaf(g0, iv[0][kw], acc[c][3 + kw]);
                        acc[c][6 + kw] = fmaf(g0, iv[1][kw], acc[c][6 + kw]);
                        acc[c][0 + kw] = fmaf(g1, iv[0][kw], acc[c][0 + kw]);
                        acc[c][3 + kw] = fmaf(g1, iv[1][kw], acc[c][3 + kw]);
                    }
                }
            }
        }
    }
    if (act) {
#pragma unroll
        for (int c = 0; c < COPT; ++c) {
            const int co = cq * COPT + c;
#pragma unroll
            for (int k = 0; k < 9; ++k) atomicAdd(&dW[(co * CIN + ci) * 9 + k], acc[c][k]);
            if (ci == 0) atomicAdd(&db[co], accb[c]);
        }
    }
}

template <int CIN, int COUT, typename TIn>
cudaError_t launch_wgrad(const float *g, const TIn *in, float *dW, float *db, int n, int w, int dil, cudaStream_t st) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long tiles = (long long)n * ((w + kWgTW - 1) / kWgTW);
    long long grid = 2LL * sms;
    if (grid > tiles) grid = tiles;
    if (grid < 1) return cudaSuccess;
    conv3x3_wgrad_kernel<CIN, COUT, TIn><<<(unsigned)grid, kWgThreads, 0, st>>>(g, in, dW, db, n, w, dil);
    return cudaGetLastError();
}

// W'[ci][co][2 - kh][2 - kw] = W[co][ci][kh][kw]: the input-gradient pass as a forward convolution.
__global__ void flip_weights_kernel(const __nv_bfloat16 *__restrict__ W, __nv_bfloat16 *__restrict__ Wf, int cin,
                                    int cout) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cin * cout * 9) return;
    const int co = i / (cin * 9), rem = i - co * cin * 9, ci = rem / 9, k = rem - ci * 9;
    const int kh = k / 3, kw = k - kh * 3;
    Wf[((ci * cout + co) * 3 + (2 - kh)) * 3 + (2 - kw)] = W[i];
}

// g = 2 (y - t) / count; *loss += sum (y - t)^2 / count
__global__ void mse_grad_kernel(const float *__restrict__ y, const float *__restrict__ tgt, float *__restrict__ g,
                                long long count, float *__restrict__ loss) {
    float part = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float d = y[i] - tgt[i];
        g[i] = 2.f * d / (float)count;
        part += d * d;
    }
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, part / (float)count);
}

__global__ void adam_kernel(int n, float lr, float b1, float b2, float eps, float c1, float c2, float *__restrict__ p,
                            __nv_bfloat16 *__restrict__ pb, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

int param_offset(int layer) {
    int off = 0;
    for (int k = 0; k < layer; ++k) off += kCh[k + 1] * kCh[k] * 9 + kCh[k + 1];
    return off;
}

}  // namespace

int cnn_param_count() { return param_offset(4); }

// Forward pass of n grids of width w. acts: [3][n][32][2][ld] bf16 (post-ReLU activations, rows of ld >= w
// elements), x: [n][2][2][w] bf16, y: [n][2][2][w] f32. The two 32 -> 32 layers run on the tensor cores
// (cnn_tc.cu) when ld is a multiple of 8 (16-byte rows for the copy engine), on the FP32 pipes otherwise.
cudaError_t cnn_forward(int n, int w, const __nv_bfloat16 *x, const __nv_bfloat16 *P, float *y, __nv_bfloat16 *acts,
                        cudaStream_t st, int ld, uint32_t *err) {
    if (ld <= 0) ld = w;
    const size_t big = (size_t)n * 32 * 2 * ld;
    const __nv_bfloat16 *W0 = P + param_offset(0), *W1 = P + param_offset(1), *W2 = P + param_offset(2),
                        *W3 = P + param_offset(3);
    cudaError_t e;
    if ((e = launch_conv<2, 32, __nv_bfloat16, kOutReluBf16>(x, W0, W0 + 32 * 2 * 9, acts, nullptr, n, w, kDil[0],
                                                             st, w, ld)) != cudaSuccess)
        return e;
    for (int k = 1; k <= 2; ++k) {
        const __nv_bfloat16 *Wk = k == 1 ? W1 : W2;
        const __nv_bfloat16 *in = acts + (k - 1) * big;
        __nv_bfloat16 *out = acts + k * big;
        if (conv32_tc_supported(ld, kDil[k]))
            e = launch_conv32_tc(in, Wk, Wk + 32 * 32 * 9, out, n, w, ld, kDil[k], err, st);
        else
            e = launch_conv<32, 32, __nv_bfloat16, kOutReluBf16>(in, Wk, Wk + 32 * 32 * 9, out, nullptr, n, w, kDil[k],
                                                                 st, ld, ld);
        if (e != cudaSuccess) return e;
    }
    return launch_conv<32, 2, __nv_bfloat16, kOutResidF32>(acts + 2 * big, W3, W3 + 2 * 32 * 9, y, x, n, w, kDil[3],
                                                           st, ld, w);
}

// Backward pass: grad (zeroed here) = d mean((y - target)^2) / d params; *loss = that mean (if loss != NULL).
// work: 2 * n * 32 * 2 * w floats; wflip: cnn_param_count() bf16 scratch.
cudaError_t cnn_backward(int n, int w, const __nv_bfloat16 *x, const __nv_bfloat16 *acts, const __nv_bfloat16 *P,
                         const float *y, const float *target, float *grad, float *loss, float *work,
                         __nv_bfloat16 *wflip, cudaStream_t st) {
    const size_t big = (size_t)n * 32 * 2 * w;
    float *ga = work, *gb = work + big;
    cudaError_t e;
    if ((e = cudaMemsetAsync(grad, 0, sizeof(float) * cnn_param_count(), st)) != cudaSuccess) return e;
    if (loss && (e = cudaMemsetAsync(loss, 0, sizeof(float), st)) != cudaSuccess) return e;
    const long long cnt = (long long)n * 2 * 2 * w;
    mse_grad_kernel<<<(unsigned)((cnt + 255) / 256 < 4096 ? (cnt + 255) / 256 : 4096), 256, 0, st>>>(y, target, ga, cnt,
                                                                                                      loss);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    for (int k = 0; k < 4; ++k) {
        const int cin = kCh[k], cout = kCh[k + 1];
        flip_weights_kernel<<<(cin * cout * 9 + 255) / 256, 256, 0, st>>>(P + param_offset(k), wflip + param_offset(k),
                                                                           cin, cout);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    float *G3 = grad + param_offset(3), *G2 = grad + param_offset(2), *G1 = grad + param_offset(1),
          *G0 = grad + param_offset(0);
    // layer 4 (32 -> 2): weights from a3, input gradient into a3's channels, masked by a3 > 0
    if ((e = launch_wgrad<32, 2, __nv_bfloat16>(ga, acts + 2 * big, G3, G3 + 2 * 32 * 9, n, w, kDil[3], st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_conv<2, 32, float, kOutMaskF32>(ga, wflip + param_offset(3), nullptr, gb, acts + 2 * big, n, w,
                                                    kDil[3], st)) != cudaSuccess)
        return e;
    // layer 3 (32 -> 32)
    if ((e = launch_wgrad<32, 32, __nv_bfloat16>(gb, acts + big, G2, G2 + 32 * 32 * 9, n, w, kDil[2], st)) !=
        cudaSuccess)
        return e;
    if ((e = launch_conv<32, 32, float, kOutMaskF32>(gb, wflip + param_offset(2), nullptr, ga, acts + big, n, w,
                                                     kDil[2], st)) != cudaSuccess)
        return e;
    // layer 2 (32 -> 32)
    if ((e = launch_wgrad<32, 32, __nv_bfloat16>(ga, acts, G1, G1 + 32 * 32 * 9, n, w, kDil[1], st)) != cudaSuccess)
        return e;
    if ((e = launch_conv<32, 32, float, kOutMaskF32>(ga, wflip + param_offset(1), nullptr, gb, acts, n, w, kDil[1],
                                                     st)) != cudaSuccess)
        return e;
    // layer 1 (2 -> 32): weights only
    return launch_wgrad<2, 32, __nv_bfloat16>(gb, x, G0, G0 + 32 * 2 * 9, n, w, kDil[0], st);
}

cudaError_t cnn_adam(int step, float lr, float b1, float b2, float eps, float *p, __nv_bfloat16 *pb, const float *g,
                     float *m, float *v, cudaStream_t st) {
    const int n = cnn_param_count();
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    adam_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, lr, b1, b2, eps, c1, c2, p, pb, g, m, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------- receive-chain glue

namespace {

struct GridArgs {
    int n_sc, n_beams, n_layers, comb, n_sym, dmrs0, dmrs1;
    int port[32];
};

// Per-DMRS-symbol LS estimate of one (slot, layer, beam) grid, interpolated over the subcarriers:
// v_j[a] = interp(y_j[q] / p_j[q]) between the layer's pilot subcarriers (held outside them).
__device__ __forceinline__ float2 grid_value(const GridArgs &g, const float2 *y, const float2 *p, int a, int port) {
    int lo, hi;
    pilot_bracket(a, port, g.comb, g.n_sc, lo, hi);
    const float2 vlo = cmul(__ldg(&y[(long long)lo * g.n_beams]), pilot_inverse(__ldg(&p[lo])));
    if (hi == lo) return vlo;
    const float2 vhi = cmul(__ldg(&y[(long long)hi * g.n_beams]), pilot_inverse(__ldg(&p[hi])));
    return interp(vlo, vhi, interp_weight(a, lo, hi));
}

__device__ __forceinline__ float block_sum(float v, float *red) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
        for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
        if (threadIdx.x == 0) red[0] = s;
    }
    __syncthreads();
    s = red[0];
    __syncthreads();
    return s;
}

// grid[gi][ch][j][a] (bf16) = v_j[a] / scale with scale = rms over the grid; gi = (slot * L + l) * B + b.
__global__ void __launch_bounds__(256)
ls_grid_kernel(GridArgs g, const float2 *__restrict__ beam, const float2 *__restrict__ pilots,
               __nv_bfloat16 *__restrict__ grid, float *__restrict__ scale) {
    __shared__ float red[32];
    const long long gi = blockIdx.x;
    const int b = (int)(gi % g.n_beams);
    const long long sl_l = gi / g.n_beams;
    const int l = (int)(sl_l % g.n_layers);
    const long long slot = sl_l / g.n_layers;
    const float2 *y0 = beam + ((slot * g.n_sym + g.dmrs0) * g.n_sc) * (long long)g.n_beams + b;
    const float2 *y1 = beam + ((slot * g.n_sym + g.dmrs1) * g.n_sc) * (long long)g.n_beams + b;
    const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
    const float2 *p1 = p0 + g.n_sc;
    const int port = g.port[l];
    float ss = 0.f;
    for (int a = threadIdx.x; a < g.n_sc; a += blockDim.x) {
        const float2 v0 = grid_value(g, y0, p0, a, port), v1 = grid_value(g, y1, p1, a, port);
        ss += v0.x * v0.x + v0.y * v0.y + v1.x * v1.x + v1.y * v1.y;
    }
    const float tot = block_sum(ss, red);
    const float sc = sqrtf(tot / (2.f * g.n_sc)) + 1e-30f;
    const float inv = 1.f / sc;
    if (threadIdx.x == 0) scale[gi] = sc;
    __nv_bfloat16 *o = grid + gi * 4LL * g.n_sc;  // [2 ch][2 rows][n_sc]
    for (int a = threadIdx.x; a < g.n_sc; a += blockDim.x) {
        const float2 v0 = grid_value(g, y0, p0, a, port), v1 = grid_value(g, y1, p1, a, port);
        o[0 * g.n_sc + a] = __float2bfloat16_rn(v0.x * inv);
        o[1 * g.n_sc + a] = __float2bfloat16_rn(v1.x * inv);
        o[2 * g.n_sc + a] = __float2bfloat16_rn(v0.y * inv);
        o[3 * g.n_sc + a] = __float2bfloat16_rn(v1.y * inv);
    }
}

// Denoised estimate of grid gi: H = scale * (y_row0 + y_row1) / 2.
// Fallback test on the layer's pilots q (both DMRS symbols j, LS_j[q] = y_j[q] / p_j[q]):
//   r_cnn = mean |LS_j[q] - scale * y_row_j[q]|^2                 (how well the estimate explains the pilots)
//   r_ref = mean |LS_j[q] - (LS_j[q - comb] + LS_j[q + comb]) / 2|^2 over the inner pilots
//           (how well plain linear interpolation predicts a pilot from its neighbours), floored at sigma^2.
// r_cnn <= kappa * r_ref: the CNN estimate replaces the plain LS estimate in H_hat; otherwise the plain LS
// estimate already written there is kept (fallback). resid[gi] = r_cnn / r_ref.
__global__ void __launch_bounds__(256)
cnn_to_h_kernel(GridArgs g, float noise_var, float kappa, const float *__restrict__ y, const float *__restrict__ scale,
                const float2 *__restrict__ beam, const float2 *__restrict__ pilots, float2 *__restrict__ H,
                float *__restrict__ resid, uint8_t *__restrict__ fallback) {
    __shared__ float red[32];
    const long long gi = blockIdx.x;
    const int b = (int)(gi % g.n_beams);
    const long long sl_l = gi / g.n_beams;
    const int l = (int)(sl_l % g.n_layers);
    const long long slot = sl_l / g.n_layers;
    const float2 *y0 = beam + ((slot * g.n_sym + g.dmrs0) * g.n_sc) * (long long)g.n_beams + b;
    const float2 *y1 = beam + ((slot * g.n_sym + g.dmrs1) * g.n_sc) * (long long)g.n_beams + b;
    const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
    const float2 *p1 = p0 + g.n_sc;
    const float *yo = y + gi * 4LL * g.n_sc;
    const float sc = scale[gi];
    const int port = g.port[l];
    const int npil = (g.n_sc - 1 - port) / g.comb + 1;
    auto ls = [&](const float2 *yy, const float2 *pp, int q) {
        return cmul(__ldg(&yy[(long long)q * g.n_beams]), pilot_inverse(__ldg(&pp[q])));
    };
    float rc = 0.f, rr = 0.f;
    for (int k = threadIdx.x; k < npil; k += blockDim.x) {
        const int q = port + k * g.comb;
        const float2 l0 = ls(y0, p0, q), l1 = ls(y1, p1, q);
        const float d0x = l0.x - sc * yo[0 * g.n_sc + q], d0y = l0.y - sc * yo[2 * g.n_sc + q];
        const float d1x = l1.x - sc * yo[1 * g.n_sc + q], d1y = l1.y - sc * yo[3 * g.n_sc + q];
        rc += d0x * d0x + d0y * d0y + d1x * d1x + d1y * d1y;
        if (k > 0 && k + 1 < npil) {
            const float2 a0 = ls(y0, p0, q - g.comb), b0 = ls(y0, p0, q + g.comb);
            const float2 a1 = ls(y1, p1, q - g.comb), b1 = ls(y1, p1, q + g.comb);
            const float e0x = l0.x - 0.5f * (a0.x + b0.x), e0y = l0.y - 0.5f * (a0.y + b0.y);
            const float e1x = l1.x - 0.5f * (a1.x + b1.x), e1y = l1.y - 0.5f * (a1.y + b1.y);
            rr += e0x * e0x + e0y * e0y + e1x * e1x + e1y * e1y;
        }
    }
    const float r_cnn = block_sum(rc, red) / (2.f * npil);
    const float r_loo = npil > 2 ? block_sum(rr, red) / (2.f * (npil - 2)) : 0.f;
    const float r_ref = fmaxf(r_loo, noise_var > 0.f ? noise_var : 1e-30f);
    const bool use_cnn = r_cnn <= kappa * r_ref;
    if (threadIdx.x == 0) {
        if (resid) resid[gi] = r_cnn / r_ref;
        if (fallback) fallback[gi] = use_cnn ? 0 : 1;
    }
    if (!use_cnn) return;
    for (int a = threadIdx.x; a < g.n_sc; a += blockDim.x) {
        const float2 h = make_float2(0.5f * sc * (yo[0 * g.n_sc + a] + yo[1 * g.n_sc + a]),
                                     0.5f * sc * (yo[2 * g.n_sc + a] + yo[3 * g.n_sc + a]));
        H[((slot * g.n_sc + a) * g.n_layers + l) * (long long)g.n_beams + b] = h;
    }
}

GridArgs grid_args(const Geometry &g) {
    GridArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.comb = g.comb;
    a.n_sym = g.n_sym;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    return a;
}

}  // namespace

cudaError_t launch_ls_grid(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots,
                           __nv_bfloat16 *grid, float *scale, cudaStream_t st) {
    const long long grids = (long long)n_slots * g.n_layers * g.n_beams;
    if (grids == 0) return cudaSuccess;
    if (grids > 0x7fffffffLL) return cudaErrorInvalidConfiguration;
    ls_grid_kernel<<<(unsigned)grids, 256, 0, st>>>(grid_args(g), beam, pilots, grid, scale);
    return cudaGetLastError();
}

cudaError_t launch_cnn_to_h(const Geometry &g, int n_slots, float kappa, const float *y, const float *scale,
                            const float2 *beam, const float2 *pilots, float2 *H, float *resid, uint8_t *fallback,
                            cudaStream_t st) {
    const long long grids = (long long)n_slots * g.n_layers * g.n_beams;
    if (grids == 0) return cudaSuccess;
    cnn_to_h_kernel<<<(unsigned)grids, 256, 0, st>>>(grid_args(g), g.noise_var + g.loading, kappa, y, scale, beam,
                                                     pilots, H, resid, fallback);
    return cudaGetLastError();
}

}  // namespace pusch
