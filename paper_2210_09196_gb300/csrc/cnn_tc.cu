// The learned estimator's two 32 -> 32 convolutions (layers 2 and 3: 3x3 kernels dilated along the subcarriers
// by 8 and 16, ReLU) on the 5th-generation tensor cores, as an implicit GEMM with BF16 operands and FP32
// accumulation in TMEM. They carry 94 % of the network's multiply-adds.
//
// For one output row h of one grid and a tile of 128 subcarriers x0 .. x0 + 127:
//     out[co][h][x] = relu(b[co] + sum_{kh, kw, ci} W[co][ci][kh][kw] in[ci][h + kh - 1][x + (kw - 1) dil])
// is D[x][co] = sum_{tap, ci} A_tap[x][ci] B_tap[co][ci] over the taps (kh, kw) whose input row h + kh - 1 lies
// in the grid (two of the three kh, so six taps; the third row is the zero padding). A_tap is the input row
// h + kh - 1 of all 32 channels shifted by (kw - 1) dil subcarriers: one TMA box of [32 ci][64 x] BF16 per 64
// subcarriers, read as an MN-major operand (x contiguous) with 128-byte swizzling; the shift keeps the box start
// on a 16-byte boundary because dil is a multiple of 8, and subcarriers outside the grid (negative, or past w)
// are filled with zeros by the copy engine, which is the "same" padding. B_tap = W[.][.][kh][kw] as [32 co][32
// ci], K-major, resident. M = 128, N = 32, K = 16 per MMA: 12 MMAs per tile.
//
// Warp roles (persistent CTAs, one per SM): warp 0 streams the taps of each tile into a three-stage ring (12
// boxes of 4 KB per tile), warp 1 owns the TMEM allocation and issues the MMAs into one of two accumulators,
// warps 2-5 add the bias, apply the ReLU and store the BF16 rows (TMEM lane = subcarrier, column = channel).
// Every wait is bounded (2 s); on expiry the CTA leaves, drains its copies and MMAs (bounded) and frees TMEM.
#include "tc_common.cuh"

namespace pusch {
namespace {

using namespace tc;

constexpr int kStages = 3;
constexpr int kTapBytes = 8192;                  // two [32 ci][64 x] BF16 boxes
constexpr int kStageBytes = 6 * kTapBytes;       // the six taps of one tile
constexpr int kBBytes = 9 * 2048;                // [9 taps][32 co][32 ci] BF16, K-major
constexpr int kThreads = 192;
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + kBBytes;

struct ConvTcArgs {
    long long tiles;     // n grids x 2 rows x ntx tiles of 128 subcarriers
    int ntx, w, ld, dil;
};

// Instruction descriptor of kind::f16 with BF16 A and B (format code 1 at [7,10) and [10,13)), F32 accumulator,
// A MN-major, B K-major, M = 128, N = 32.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | ((uint32_t)(32 >> 3) << 17) |
                            ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(acc));
}

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int x, int y, int z, int w4,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(w4), "r"(bar)
        : "memory");
}

struct ConvShared {
    uint64_t full[kStages], empty[kStages], tfull[2], tempty[2], drain;
    uint32_t tmem_base;
    int abort;
    float bias[32];
};

__global__ void __launch_bounds__(kThreads, 1)
conv32_tc_kernel(const __grid_constant__ CUtensorMap tin, ConvTcArgs g, const __nv_bfloat16 *__restrict__ W,
                 const __nv_bfloat16 *__restrict__ bias, __nv_bfloat16 *__restrict__ out, uint32_t *err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ ConvShared sh;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sB = base + (uint32_t)kStages * kStageBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *abort = &sh.abort;

    // B_tap[co][ci] = W[co][ci][kh][kw], tap = 3 kh + kw: element (co, ci) at tap * 2048 + (co / 8) * 512 +
    // (ci / 8) * 128 + (co % 8) * 16 + (ci % 8) * 2
    for (int e = tid; e < 9 * 32 * 32; e += kThreads) {
        const int tap = e >> 10, co = (e >> 5) & 31, ci = e & 31;
        const __nv_bfloat16 v = W[(co * 32 + ci) * 9 + tap];
        *reinterpret_cast<__nv_bfloat16 *>(gbase + kStages * kStageBytes + tap * 2048 + (co >> 3) * 512 + (ci >> 3) * 128 +
                                           (co & 7) * 16 + (ci & 7) * 2) = v;
    }
    if (tid < 32) sh.bias[tid] = __bfloat162float(bias[tid]);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(smem_u32(&sh.full[s]), 1);
            mbar_init(smem_u32(&sh.empty[s]), 1);
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
                     "r"(64));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = sh.tmem_base;
    const long long n_my = g.tiles > blockIdx.x ? (g.tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (warp == 0) {
        // ---------------------------------------------------------------- TMA producer
        if (lane == 0) {
            long long i = 0;
            for (; i < n_my; ++i) {
                const int s = (int)(i % kStages);
                if (!mbar_wait(smem_u32(&sh.empty[s]), (uint32_t)(((i / kStages) & 1) ^ 1), abort, err)) break;
                const long long t = blockIdx.x + i * gridDim.x;
                const long long grid_row = t / g.ntx;
                const int xt = (int)(t - grid_row * g.ntx), h = (int)(grid_row & 1);
                const int gi = (int)(grid_row >> 1);
                const uint32_t bar = smem_u32(&sh.full[s]);
                mbar_expect_tx(bar, kStageBytes);
                const uint32_t dst = base + (uint32_t)s * kStageBytes;
                for (int r = 0; r < 2; ++r)          // input row r = h + kh - 1 (kh = 1 - h + r)
                    for (int kw = 0; kw < 3; ++kw)
                        for (int half = 0; half < 2; ++half)
                            tma_load_4d(dst + (uint32_t)((r * 3 + kw) * kTapBytes + half * 4096), &tin,
                                        xt * 128 + (kw - 1) * g.dil + 64 * half, r, 0, gi, bar);
                (void)h;
            }
            if (*abort)
                for (long long j = i - 1; j >= 0 && j >= i - kStages; --j)
                    mbar_drain(smem_u32(&sh.full[(int)(j % kStages)]), (uint32_t)((j / kStages) & 1));
        }
    } else if (warp == 1) {
        // ---------------------------------------------------------------- MMA issuer
        if (lane == 0) {
            for (long long i = 0; i < n_my; ++i) {
                const int s = (int)(i % kStages), buf = (int)(i & 1);
                if (!mbar_wait(smem_u32(&sh.tempty[buf]), (uint32_t)(((i >> 1) & 1) ^ 1), abort, err)) break;
                if (!mbar_wait(smem_u32(&sh.full[s]), (uint32_t)((i / kStages) & 1), abort, err)) break;
                fence_after_sync();
                const long long t = blockIdx.x + i * gridDim.x;
                const int h = (int)((t / g.ntx) & 1);
                const uint32_t a0 = base + (uint32_t)s * kStageBytes;
                int k = 0;
                for (int r = 0; r < 2; ++r)
                    for (int kw = 0; kw < 3; ++kw) {
                        const int tapw = (1 - h + r) * 3 + kw;       // weight tap (kh, kw)
                        for (int ks = 0; ks < 2; ++ks, ++k)
                            mma_bf16(tmem + (uint32_t)(buf * 32),
                                     smem_desc(a0 + (uint32_t)((r * 3 + kw) * kTapBytes + ks * 2048), 4096, 1024, 2),
                                     smem_desc(sB + (uint32_t)(tapw * 2048 + ks * 256), 128, 512, 0), k > 0 ? 1u : 0u);
                    }
                mma_commit(smem_u32(&sh.empty[s]));
                mma_commit(smem_u32(&sh.tfull[buf]));
            }
            mma_commit(smem_u32(&sh.drain));
            mbar_drain(smem_u32(&sh.drain), 0);
        }
    } else {
        // ---------------------------------------------------------------- epilogue: bias, ReLU, BF16 rows
        const int q = warp & 3;
        for (long long i = 0; i < n_my; ++i) {
            const int buf = (int)(i & 1);
            bool ok = true;
            if (lane == 0) ok = mbar_wait_sleep(smem_u32(&sh.tfull[buf]), (uint32_t)((i >> 1) & 1), abort, err, 32);
            if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) break;
            fence_after_sync();
            const long long t = blockIdx.x + i * gridDim.x;
            const long long grid_row = t / g.ntx;
            const int xt = (int)(t - grid_row * g.ntx), h = (int)(grid_row & 1);
            const long long gi = grid_row >> 1;
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(buf * 32), r);
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh.tempty[buf]));
            const int x = xt * 128 + 32 * q + lane;
            if (x < g.w) {
                __nv_bfloat16 *o = out + (gi * 64 + h) * (long long)g.ld + x;   // channel co at o + co * 2 ld
#pragma unroll
                for (int co = 0; co < 32; ++co) {
                    const float v = __uint_as_float(r[co]) + sh.bias[co];
                    o[(long long)co * 2 * g.ld] = __float2bfloat16_rn(v > 0.f ? v : 0.f);
                }
            }
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
    }
}

}  // namespace

bool conv32_tc_supported(int ld, int dil) { return ld % 8 == 0 && dil % 8 == 0 && dil > 0 && dil <= 64; }

cudaError_t launch_conv32_tc(const __nv_bfloat16 *in, const __nv_bfloat16 *W, const __nv_bfloat16 *b,
                             __nv_bfloat16 *out, int n, int w, int ld, int dil, uint32_t *err, cudaStream_t st) {
    if (!conv32_tc_supported(ld, dil) || w > ld) return cudaErrorNotSupported;
    if (n == 0 || w == 0) return cudaSuccess;
    if (reinterpret_cast<uintptr_t>(in) % 16 != 0) return cudaErrorMisalignedAddress;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    // the activations [n][32 ci][2 rows][ld] BF16 as a 4-D tensor of logical width w: x beyond w reads as zero
    CUtensorMap map;
    cuuint64_t dims[4] = {(cuuint64_t)w, 2, 32, (cuuint64_t)n};
    cuuint64_t strides[3] = {(cuuint64_t)ld * 2, (cuuint64_t)ld * 4, (cuuint64_t)ld * 128};
    cuuint32_t box[4] = {64, 1, 32, 1};
    cuuint32_t estr[4] = {1, 1, 1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<__nv_bfloat16 *>(in), dims, strides, box,
                     estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(conv32_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    ConvTcArgs a;
    a.ntx = (w + 127) / 128;
    a.tiles = (long long)n * 2 * a.ntx;
    a.w = w;
    a.ld = ld;
    a.dil = dil;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = sms;
    if (grid > a.tiles) grid = a.tiles;
    conv32_tc_kernel<<<(unsigned)grid, kThreads, kSmemBytes, st>>>(map, a, W, b, out, err);
    return cudaGetLastError();
}

}  // namespace pusch
