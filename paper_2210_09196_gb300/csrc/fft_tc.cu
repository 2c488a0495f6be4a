// OFDM demodulation on the 5th-generation tensor cores (Section II: one FFT per antenna and OFDM symbol;
// Table I "OFDM dem."): the mixed form's 4096-point FFTs of FP16 time samples, written as three radix-16
// stages, each a tcgen05 matrix product with a 16-point DFT matrix (FP16 operands, FP32 accumulation in
// TMEM), with the twiddles between the stages applied in FP32 by the threads that read the accumulators.
//
// The transform. With n = 256 a + m (m = 16 b + c) and k = k0 + 16 k1 + 256 k2 (all digits in [0, 16)):
//   stage 1  Y1[m][k0]      = sum_a x[256 a + m] w16^(a k0),            then * W^(m k0)
//   stage 2  Y2[k0][c][k1]  = sum_b Y1[16 b + c][k0] w16^(b k1),        then * W^(16 c k1)
//   stage 3  X[k0 + 16 k1 + 256 k2] = sum_c Y2[k0][c][k1] w16^(c k2)
// with W = exp(-2 pi i / 4096), w16 = W^256. Each stage is D[M][N] = A[M][K] B[N][K]^T with M the
// independent vectors (tiles of 128 TMEM lanes), K the 16 inputs of a radix-16 butterfly, N its 16 outputs.
//
// Operands (shared memory, no global round trip between the stages):
//   stage 1  A = the time samples as loaded by TMA: the row of 4096 interleaved complex values read as a
//            [16 a][512 mu] FP16 matrix, mu = 2 m + (re, im), so M = mu (512 real rows), K = a (16), MN-major
//            with 128-byte swizzling; B1 = [cos | -sin] of the DFT angles (N = 32: k0 x (re, im)). A real row
//            gives sum_a Re(x) w^(a k0) or sum_a Im(x) w^(a k0); the two lanes of a subcarrier pair combine
//            them (Y1 = P_re + i P_im) with one exchange of eight values.
//   stage 2  A2 = Y1 written by the threads, M = c + 16 k0, K = (b, re/im) (32), MN-major, 128-byte swizzle,
//            2-byte stores ordered so that a warp's 32 stores hit distinct banks; B2 = the real embedding of the
//            complex DFT matrix ([[C, S], [-S, C]] per entry).
//   stage 3  A3 = Y2 written by the threads, M = k0 + 16 k1, K = (c, re/im), K-major without swizzle with the
//            core-matrix strides padded (160 B along K, 608 B along M) so that the 4-byte complex stores of a
//            warp are conflict-free; B = B2. The accumulator row of lane M holds bins M + 256 k2, so
//            consecutive lanes write consecutive bins of the FP16 output planes.
//
// Each CTA (8 warps, three per SM, 128 TMEM columns) transforms its rows one after another; the rows arrive by
// TMA into a two-stage ring, one MMA-issuing thread drives the stages, and all eight warps read the
// accumulators (warp w owns TMEM lane quarter w % 4). Every wait is bounded (2 s); on expiry the CTA sets the
// tensor-core bit (kErrTensorWait) of the error word, drains its copies and MMAs (bounded) and frees its TMEM.
//
// Error: the operands of every stage are FP16 (the input exactly, the two intermediates and the DFT matrices
// rounded to nearest), so the output carries about 2^-11 relative error per stage (-60 dB or better against
// the exact transform; measured against the FP64 oracle in the tests), well under the chain's -40 dB gate.
#include "tc_common.cuh"

namespace pusch {
namespace {

using namespace tc;

constexpr int kN = 4096;
constexpr int kThreads = 256;
constexpr int kCtasPerSm = 3;
constexpr int kTmemCols = 128;
constexpr int kStages = 2;

constexpr uint32_t kRowBytes = kN * 4;                      // one row of FP16 complex samples: 16 KB
constexpr uint32_t kOffIn = 0;                              // input ring (stage-1 A operands)
constexpr uint32_t kOffA2 = kOffIn + kStages * kRowBytes;   // 16 KB, 1024-aligned
constexpr uint32_t kA3Lbo = 160, kA3Sbo = 608;              // padded K-major strides of A3
constexpr uint32_t kOffA3 = kOffA2 + 16384;                 // 32 row groups x 608 B
constexpr uint32_t kOffB1 = kOffA3 + 32 * kA3Sbo;           // [32][16] FP16, K-major
constexpr uint32_t kOffB2 = kOffB1 + 1024;                  // [32][32] FP16, K-major
constexpr uint32_t kSmemUsed = kOffB2 + 2048;
constexpr size_t kSmemBytes = kSmemUsed + 1024;             // + alignment of the base to 1024 B

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

// K-major, no swizzle: element (n, k) of an operand with `sbo` bytes per 8-row group and `lbo` bytes between
// the core matrices (8 rows x 8 FP16) along K.
__device__ __forceinline__ uint32_t kmajor_off(int n, int k, uint32_t lbo, uint32_t sbo) {
    return (uint32_t)(n >> 3) * sbo + (uint32_t)(k >> 3) * lbo + (uint32_t)(n & 7) * 16u + (uint32_t)(k & 7) * 2u;
}

// A2 (MN-major, 128-byte swizzle, 1024-aligned atoms): element (row M, K row kr), the 64-row halves 4 KB apart.
__device__ __forceinline__ uint32_t a2_off(int M, int kr) {
    return (uint32_t)(M >> 6) * 4096u + (uint32_t)kr * 128u + ((uint32_t)(((M & 63) >> 3) ^ (kr & 7)) << 4) +
           (uint32_t)(M & 7) * 2u;
}

// p[i] = w^i for i < 8 (p[0] = 1), by at most three products deep (w^2, w^4 and the rest from them).
__device__ __forceinline__ void powers8(float2 w, float2 (&p)[8]) {
    p[0] = make_float2(1.f, 0.f);
    p[1] = w;
    p[2] = cmul(w, w);
    p[3] = cmul(p[2], w);
    p[4] = cmul(p[2], p[2]);
    p[5] = cmul(p[4], w);
    p[6] = cmul(p[4], p[2]);
    p[7] = cmul(p[4], p[3]);
}

struct FftTcArgs {
    long long rows;
    int n_sc, pitch;
};

__global__ void __launch_bounds__(kThreads, kCtasPerSm)
fft_tc_kernel(const __grid_constant__ CUtensorMap tin, __half *__restrict__ out, const float2 *__restrict__ tw,
              FftTcArgs g, uint32_t *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[kStages];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ __align__(8) uint64_t bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3;     // TMEM lane quarter of this warp
    const int wh = warp >> 2;   // which of the two warps of that quarter
    volatile int *abort = &s_abort;
    uint32_t *errw = err;

    // ---------------------------------------------------------------- B operands (resident)
    for (int e = tid; e < 32 * 16; e += kThreads) {          // B1[n = 2 k0 + o][a]
        const int n = e >> 4, a = e & 15, k0 = n >> 1;
        float s, c;
        sincospif((float)((a * k0) & 15) / 8.f, &s, &c);       // angle 2 pi a k0 / 16
        *reinterpret_cast<__half *>(gbase + kOffB1 + kmajor_off(n, a, 128, 256)) = __float2half_rn((n & 1) ? -s : c);
    }
    for (int e = tid; e < 32 * 32; e += kThreads) {          // B2[n = 2 k1 + o][k = 2 b + i]
        const int n = e >> 5, k = e & 31, k1 = n >> 1, b = k >> 1;
        float s, c;
        sincospif((float)((b * k1) & 15) / 8.f, &s, &c);
        const int o = n & 1, i = k & 1;
        const float v = (o == i) ? c : (o == 0 ? s : -s);
        *reinterpret_cast<__half *>(gbase + kOffB2 + kmajor_off(n, k, 128, 512)) = __float2half_rn(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bar_full[s]), 1);
        mbar_init(smem_u32(&bar_mma), 1);
        mbar_init(smem_u32(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;

    const long long n_my = g.rows > blockIdx.x ? (g.rows - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto issue = [&](long long it) {       // thread 0: the 8 boxes of row `it` into ring stage it % 2
        const int s = (int)(it & 1);
        const long long row = blockIdx.x + it * gridDim.x;
        const uint32_t bar = smem_u32(&bar_full[s]);
        mbar_expect_tx(bar, kRowBytes);
        for (int bx = 0; bx < 8; ++bx)
            tma_load_2d(base + kOffIn + (uint32_t)s * kRowBytes + (uint32_t)bx * 2048u, &tin, 64 * bx, (int)(row * 16),
                        bar);
    };
    long long issued = 0;
    if (tid == 0)
        for (; issued < kStages && issued < n_my; ++issued) issue(issued);

    const int h = g.n_sc >> 1;
    const uint32_t id_mn = idesc_f16(128, 32, true, false), id_k = idesc_f16(128, 32, false, false);
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    uint32_t mma_phase = 0;
    long long it = 0;
    for (; it < n_my; ++it) {
        const int s = (int)(it & 1);
        const long long row = blockIdx.x + it * gridDim.x;

        // ------------------------------------------------------------ stage 1: 4 MMAs (M tiles of mu)
        if (tid == 0 && mbar_wait(smem_u32(&bar_full[s]), (uint32_t)((it >> 1) & 1), abort, errw)) {
            fence_after_sync();
            const uint64_t bd = smem_desc(base + kOffB1, 128, 256, 0);
            for (int t = 0; t < 4; ++t)
                mma_f16(tmem + 32u * t, smem_desc(base + kOffIn + (uint32_t)s * kRowBytes + (uint32_t)t * 4096u, 2048, 1024, 2),
                        bd, id_mn, 0u);
            mma_commit(smem_u32(&bar_mma));
        }
        // one thread polls the MMA barrier (bounded); the others wait at the CTA barrier without issuing
        bool ok = tid != 0 || mbar_wait(smem_u32(&bar_mma), mma_phase, abort, errw);
        if (__syncthreads_or(!ok)) break;
        mma_phase ^= 1u;
        fence_after_sync();
        if (tid == 0 && issued < n_my && issued == it + kStages) issue(issued++);   // stage s is free again

        // ------------------------------------------------------------ epilogue 1 -> A2
        {
            const int ri = lane & 1, c = lane >> 1;
#pragma unroll 1
            for (int u = 0; u < 2; ++u) {
                const int t = wh + 2 * u;
                uint32_t r[32];
                tmem_ld32(tq + 32u * t, r);
                const int m = 64 * t + 16 * q + c, b = 4 * t + q;
                // twiddles W^(m k0), k0 = 8 ri + i: W^(8 ri m) times the powers W^(m i), from two table entries
                float2 pw[8];
                powers8(__ldg(&tw[m]), pw);
                const float2 base8 = ri ? __ldg(&tw[(8 * m) & (kN - 1)]) : make_float2(1.f, 0.f);
                float2 Y[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 lo = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
                    const float2 hi = make_float2(__uint_as_float(r[2 * i + 16]), __uint_as_float(r[2 * i + 17]));
                    const float2 own = ri ? hi : lo, snd = ri ? lo : hi;
                    const float2 rcv = make_float2(__shfl_xor_sync(0xffffffffu, snd.x, 1),
                                                   __shfl_xor_sync(0xffffffffu, snd.y, 1));
                    // Y1 = P_re + i P_im: lane ri = 0 holds P_re (k0 = i), lane ri = 1 holds P_im (k0 = 8 + i)
                    Y[i] = ri ? make_float2(rcv.x - own.y, rcv.y + own.x) : make_float2(own.x - rcv.y, own.y + rcv.x);
                    Y[i] = cmul(Y[i], ri ? cmul(base8, pw[i]) : pw[i]);
                }
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    // store order: lanes ri = 1 take element j ^ 2, so that the two lane halves hit distinct banks
                    const float2 y = ri ? Y[j ^ 2] : Y[j];
                    const int M = c + 16 * (ri ? 8 + (j ^ 2) : j);
                    const __half2 v = __floats2half2_rn(y.x, y.y);
                    *reinterpret_cast<__half *>(gbase + kOffA2 + a2_off(M, 2 * b)) = __low2half(v);
                    *reinterpret_cast<__half *>(gbase + kOffA2 + a2_off(M, 2 * b + 1)) = __high2half(v);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before_sync();
        __syncthreads();

        // ------------------------------------------------------------ stage 2: 2 M tiles x 2 K steps
        if (tid == 0) {
            fence_after_sync();
            for (int t = 0; t < 2; ++t)
                for (int ks = 0; ks < 2; ++ks)
                    mma_f16(tmem + 32u * t, smem_desc(base + kOffA2 + (uint32_t)t * 8192u + (uint32_t)ks * 2048u, 4096, 1024, 2),
                            smem_desc(base + kOffB2 + (uint32_t)ks * 256u, 128, 512, 0), id_mn, ks > 0 ? 1u : 0u);
            mma_commit(smem_u32(&bar_mma));
        }
        ok = tid != 0 || mbar_wait(smem_u32(&bar_mma), mma_phase, abort, errw);
        if (__syncthreads_or(!ok)) break;
        mma_phase ^= 1u;
        fence_after_sync();

        // ------------------------------------------------------------ epilogue 2 -> A3
        {
            const int M2 = 128 * wh + 32 * q + lane, c = M2 & 15, k0 = M2 >> 4;
            // twiddles W^(16 c k1) = v^k1, v = W^(16 c): the powers below 8, then v^8 times them
            float2 pv[8];
            powers8(__ldg(&tw[16 * c]), pv);
            const float2 v8 = cmul(pv[4], pv[4]);
            uint32_t r[32];
            tmem_ld32(tq + 32u * wh, r);
#pragma unroll
            for (int k1 = 0; k1 < 16; ++k1) {
                float2 z = make_float2(__uint_as_float(r[2 * k1]), __uint_as_float(r[2 * k1 + 1]));
                z = cmul(z, k1 < 8 ? pv[k1] : cmul(v8, pv[k1 - 8]));
                const __half2 v = __floats2half2_rn(z.x, z.y);
                *reinterpret_cast<__half2 *>(gbase + kOffA3 + kmajor_off(k0 + 16 * k1, 2 * c, kA3Lbo, kA3Sbo)) = v;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before_sync();
        __syncthreads();

        // ------------------------------------------------------------ stage 3: 2 M tiles x 2 K steps
        if (tid == 0) {
            fence_after_sync();
            for (int t = 0; t < 2; ++t)
                for (int ks = 0; ks < 2; ++ks)
                    mma_f16(tmem + 32u * t,
                            smem_desc(base + kOffA3 + (uint32_t)t * 16u * kA3Sbo + (uint32_t)ks * 2u * kA3Lbo, kA3Lbo, kA3Sbo, 0),
                            smem_desc(base + kOffB2 + (uint32_t)ks * 256u, 128, 512, 0), id_k, ks > 0 ? 1u : 0u);
            mma_commit(smem_u32(&bar_mma));
        }
        ok = tid != 0 || mbar_wait(smem_u32(&bar_mma), mma_phase, abort, errw);
        if (__syncthreads_or(!ok)) break;
        mma_phase ^= 1u;
        fence_after_sync();

        // ------------------------------------------------------------ epilogue 3 -> FP16 planes
        {
            const int M3 = 128 * wh + 32 * q + lane;
            uint32_t r[32];
            tmem_ld32(tq + 32u * wh, r);
            __half *o = out + row * 2 * (long long)g.pitch;
#pragma unroll
            for (int k2 = 0; k2 < 16; ++k2) {
                const int a = (M3 + 256 * k2 + h) & (kN - 1);
                if (a < g.n_sc) {
                    const __half2 v = __floats2half2_rn(__uint_as_float(r[2 * k2]), __uint_as_float(r[2 * k2 + 1]));
                    o[a] = __low2half(v);
                    o[g.pitch + a] = __high2half(v);
                }
            }
            for (int a = g.n_sc + tid; a < g.pitch; a += kThreads) {
                o[a] = __float2half_rn(0.f);
                o[g.pitch + a] = __float2half_rn(0.f);
            }
        }
        fence_before_sync();
        __syncthreads();     // the TMEM columns and A2 / A3 are free for the next row
    }

    if (*abort && tid == 0) {
        // drain: the row copies still in flight and every MMA issued (bounded waits)
        for (long long j = it; j < issued; ++j)
            mbar_drain(smem_u32(&bar_full[(int)(j & 1)]), (uint32_t)((j >> 1) & 1));
        mma_commit(smem_u32(&bar_drain));
        mbar_drain(smem_u32(&bar_drain), 0);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

}  // namespace

bool fft_tc_supported(const Geometry &g) {
    return g.form == PUSCH_FORM_MIXED && g.n_fft == kN && g.in_fp16 && !g.cp && !g.shift;
}

cudaError_t launch_fft_tc(const Geometry &g, long long rows, const void *in, void *out, const float2 *tw,
                          uint32_t *err, cudaStream_t st) {
    if (!fft_tc_supported(g)) return cudaErrorNotSupported;
    if (rows == 0) return cudaSuccess;
    if (rows * 16 > 0x7fffffffLL) return cudaErrorInvalidValue;     // TMA row coordinate is 32-bit
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    cuuint64_t dims[2] = {512, (cuuint64_t)(rows * 16)};
    cuuint64_t strides[1] = {1024};
    cuuint32_t box[2] = {64, 16};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void *>(in), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(fft_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // kCtasPerSm resident CTAs per SM (shared memory and registers allow three; 3 x 128 TMEM columns fit in
    // 512). The CTAs are independent, so a CTA that cannot be resident at once simply runs later.
    long long grid = (long long)sms * kCtasPerSm;
    if (grid > rows) grid = rows;
    FftTcArgs a;
    a.rows = rows;
    a.n_sc = g.n_sc;
    a.pitch = g.sc_pitch;
    fft_tc_kernel<<<(unsigned)grid, kThreads, kSmemBytes, st>>>(map, static_cast<__half *>(out), tw, a, err);
    return cudaGetLastError();
}

}  // namespace pusch
