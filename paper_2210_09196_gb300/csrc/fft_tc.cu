// OFDM demodulation on the 5th-generation tensor cores (Section II: one FFT per antenna and OFDM symbol;
// Table I "OFDM dem."): the mixed form's 4096-point FFTs of FP16 time samples as two 64-point stages, each a
// tcgen05 product with the 64-point DFT matrix (FP16 operands, FP32 accumulation in TMEM), the twiddles between
// the stages applied in FP32 by the threads that read the first accumulator.
//
// The transform. With n = 64 a + m and k = k0 + 64 k1 (a, m, k0, k1 in [0, 64)), W = exp(-2 pi i / 4096) and
// w = W^64:
//   stage 1  Y[m][k0]   = W^(m k0) sum_a x[64 a + m] w^(a k0)
//   stage 2  X[k0 + 64 k1] = sum_m Y[m][k0] w^(m k1)
// Both stages multiply real rows by the same real matrix B[n = 2 k + o][j] = (cos, -sin)(2 pi j k / 64)
// (N = 128: 64 outputs x (re, im); K = 64): a real row v gives sum_j v_j w^(j k) for every k.
//   stage 1  A = the row as TMA loads it, read as a [64 a][128 mu] FP16 matrix, mu = 2 m + (re, im): M = mu
//            (128 real rows), K = a, MN-major with 128-byte swizzling. Row (m, re) gives P_re[k0] =
//            sum_a Re(x) w^(a k0), row (m, im) gives P_im[k0]; the two lanes of m combine
//            Y = P_re + i P_im with one exchange per eight values and apply W^(m k0).
//   stage 2  A2 = Y written by those lanes as real rows: row 2 k0 = Re Y[.][k0], row 2 k0 + 1 = Im Y[.][k0],
//            K = m, MN-major with 128-byte swizzling (the layout of stage 1's operand): a lane holds one m and
//            eight consecutive k0, i.e. 16 consecutive rows n = 2 k0 + (re, im), and writes them as two
//            16-byte pieces. The lanes of row pair (2 k0, 2 k0 + 1) combine X = D_re + i D_im the same way and
//            write bins k0 + 64 k1, consecutive across lanes, into the FP16 output planes.
// A 4096-point transform thus costs two MMA passes (8 MMAs of 128 x 128 x 16) and one pass of twiddles and
// transposition through shared memory.
//
// Roles (persistent CTAs, four per SM, 128 TMEM columns each): warps 0-3 read the accumulators (warp q owns TMEM
// lane quarter q) and write the next operand or the output; warp 4 issues the row copies (TMA, a one-stage ring)
// and the MMAs. They hand over through mbarriers: the MMA commits signal the accumulator, the four reading
// warps' arrivals signal the second operand and the free accumulator. Every wait is bounded (2 s); on expiry
// the CTA sets the tensor-core bit (kErrTensorWait) of the error word, every role leaves its loop, the copies
// and MMAs in flight are drained (bounded) and TMEM is freed.
//
// Error: the input enters the first product exactly; the intermediate Y and the DFT matrix are rounded to FP16
// (round to nearest) and the output is stored as FP16, so the transform carries about 2^-11 relative error
// (measured against the FP64 oracle in the tests), far under the chain's -40 dB gate.
#include "tc_common.cuh"

namespace pusch {
namespace {

using namespace tc;

constexpr int kN = 4096;
constexpr int kEpiWarps = 4;
constexpr int kThreads = 32 * (kEpiWarps + 1);
constexpr int kCtasPerSm = 4;
constexpr int kTmemCols = 128;
constexpr int kStages = 1;

constexpr uint32_t kRowBytes = kN * 4;                      // one row of FP16 complex samples: 16 KB
constexpr uint32_t kOffIn = 0;                              // input ring (stage-1 A operands, 1024-aligned)
constexpr uint32_t kOffB = kOffIn + kStages * kRowBytes;    // B: [128][64] FP16, K-major, 16 KB
constexpr uint32_t kOffA2 = kOffB + 16384;                  // A2: [2 halves of 64 n][64 m][128 B], 16 KB
constexpr uint32_t kSmemUsed = kOffA2 + 16384;
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

// Bounded wait by one lane of the warp, the result broadcast to the warp.
__device__ __forceinline__ bool warp_wait(uint32_t bar, uint32_t parity, volatile int *abort, uint32_t *err, int lane) {
    bool ok = true;
    if (lane == 0) ok = mbar_wait_sleep(bar, parity, abort, err, 32);
    return __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
}

// The 16 complex values of one 32-column accumulator chunk of a real row, combined with the partner row's
// (lane ^ 1): lane 2 j (the row of real parts) returns V[i] = D_re[i] + i D_im[i] for the chunk's outputs
// 0..7, lane 2 j + 1 (imaginary parts) returns them for outputs 8..15.
__device__ __forceinline__ void combine_pair(const uint32_t (&r)[32], int odd, float2 (&V)[8]) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float2 lo = make_float2(__uint_as_float(r[2 * i]), __uint_as_float(r[2 * i + 1]));
        const float2 hi = make_float2(__uint_as_float(r[2 * i + 16]), __uint_as_float(r[2 * i + 17]));
        const float2 own = odd ? hi : lo, snd = odd ? lo : hi;
        const float2 rcv = make_float2(__shfl_xor_sync(0xffffffffu, snd.x, 1), __shfl_xor_sync(0xffffffffu, snd.y, 1));
        V[i] = odd ? make_float2(rcv.x - own.y, rcv.y + own.x) : make_float2(own.x - rcv.y, own.y + rcv.x);
    }
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
    __shared__ __align__(8) uint64_t bar_acc;     // MMA commits: the accumulator holds a finished product
    __shared__ __align__(8) uint64_t bar_op;      // 4 warp arrivals: A2 written / the accumulator read out
    __shared__ __align__(8) uint64_t bar_drain;
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *abort = &s_abort;

    // ---------------------------------------------------------------- B (resident): (cos, -sin)(2 pi j k / 64)
    // from the twiddle table (w^(j k) = W^(64 (j k mod 64))), eight K values (one 16-byte core-matrix row) per
    // thread and store
    for (int e = tid; e < 128 * 8; e += kThreads) {
        const int n = e >> 3, j0 = (e & 7) * 8, k = n >> 1;
        __align__(16) __half v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const float2 w = __ldg(&tw[64 * (((j0 + u) * k) & 63)]);
            v[u] = __float2half_rn((n & 1) ? w.y : w.x);     // Im W^q = -sin
        }
        *reinterpret_cast<uint4 *>(gbase + kOffB + kmajor_off(n, j0, 128, 1024)) = *reinterpret_cast<const uint4 *>(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(smem_u32(&bar_full[s]), 1);
        mbar_init(smem_u32(&bar_acc), 1);
        mbar_init(smem_u32(&bar_op), kEpiWarps);
        mbar_init(smem_u32(&bar_drain), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == kEpiWarps) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = s_tmem;
    const long long n_my = g.rows > blockIdx.x ? (g.rows - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

    if (warp == kEpiWarps) {
        // ------------------------------------------------------------ control: row copies and MMAs
        if (lane == 0) {
            const uint32_t idesc = idesc_f16(128, 128, true, false);   // A MN-major in both stages
            // the time samples are read once: evict-first, so that they do not push the FFT output (the next
            // kernel's input) out of L2 (an evict-last hint on the 2-byte output stores measured slower)
            const uint64_t pol_in = l2_policy_evict_first();
            auto issue = [&](long long i) {
                const int s = (int)(i % kStages);
                const long long row = blockIdx.x + i * gridDim.x;
                const uint32_t bar = smem_u32(&bar_full[s]);
                mbar_expect_tx(bar, kRowBytes);
                for (int h = 0; h < 2; ++h)
                    tma_load_2d_hint(base + kOffIn + (uint32_t)s * kRowBytes + (uint32_t)h * 8192u, &tin, 64 * h,
                                     (int)(row * 64), bar, pol_in);
            };
            long long issued = 0;
            for (; issued < kStages && issued < n_my; ++issued) issue(issued);
            uint32_t op_phase = 0;
            long long it = 0;
            bool ok = true;
            for (; it < n_my && ok; ++it) {
                const int s = (int)(it % kStages);
                ok = mbar_wait_sleep(smem_u32(&bar_full[s]), (uint32_t)((it / kStages) & 1), abort, err, 64);
                if (ok && it > 0) {   // the reading warps have emptied the accumulator of row it - 1
                    ok = mbar_wait_sleep(smem_u32(&bar_op), op_phase, abort, err, 128);
                    op_phase ^= 1u;
                }
                if (!ok) break;
                fence_after_sync();
                const uint32_t a0 = base + kOffIn + (uint32_t)s * kRowBytes;
                for (int ks = 0; ks < 4; ++ks)
                    mma_f16(tmem, smem_desc(a0 + (uint32_t)ks * 2048u, 8192, 1024, 2),
                            smem_desc(base + kOffB + (uint32_t)ks * 256u, 128, 1024, 0), idesc, ks > 0 ? 1u : 0u);
                mma_commit(smem_u32(&bar_acc));
                // the stage-1 products have read the row: its ring slot takes a later row
                ok = mbar_wait_sleep(smem_u32(&bar_acc), 0u, abort, err, 32);
                if (!ok) break;
                if (issued < n_my) issue(issued++);
                ok = mbar_wait_sleep(smem_u32(&bar_op), op_phase, abort, err, 128);   // A2 written
                op_phase ^= 1u;
                if (!ok) break;
                fence_after_sync();
                for (int ks = 0; ks < 4; ++ks)
                    mma_f16(tmem, smem_desc(base + kOffA2 + (uint32_t)ks * 2048u, 8192, 1024, 2),
                            smem_desc(base + kOffB + (uint32_t)ks * 256u, 128, 1024, 0), idesc, ks > 0 ? 1u : 0u);
                mma_commit(smem_u32(&bar_acc));
            }
            if (ok && n_my > 0) mbar_wait_sleep(smem_u32(&bar_op), op_phase, abort, err, 128);   // the last row read out
            if (*abort) {
                // drain: the row copies still in flight and every MMA issued (bounded waits)
                for (long long j = it; j < issued; ++j)
                    mbar_drain(smem_u32(&bar_full[(int)(j % kStages)]), (uint32_t)((j / kStages) & 1));
                mma_commit(smem_u32(&bar_drain));
                mbar_drain(smem_u32(&bar_drain), 0);
            }
        }
    } else {
        // ------------------------------------------------------------ accumulator readers (warp q = lane quarter)
        const int q = warp, odd = lane & 1, j = 16 * q + (lane >> 1);   // stage 1: m = j; stage 2: k0 = j
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        // twiddles W^(m k0), k0 = 16 c + 8 odd + i: W^(m (16 c + 8 odd)) * W^(m i), from exact table entries
        float2 pw[8], bs[4];
#pragma unroll
        for (int i = 0; i < 8; ++i) pw[i] = __ldg(&tw[j * i]);
#pragma unroll
        for (int c = 0; c < 4; ++c) bs[c] = __ldg(&tw[j * (16 * c + 8 * odd)]);
        const int h = g.n_sc >> 1;
        uint32_t acc_phase = 0;
        for (long long it = 0; it < n_my; ++it) {
            const long long row = blockIdx.x + it * gridDim.x;
            // ---- stage-1 accumulator -> A2 (twiddled, transposed, FP16)
            if (!warp_wait(smem_u32(&bar_acc), acc_phase, abort, err, lane)) break;
            acc_phase ^= 1u;
            fence_after_sync();
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t r[32];
                tmem_ld32(tq + 32u * c, r);
                float2 Y[8];
                combine_pair(r, odd, Y);
                // k0 = 16 c + 8 odd + i: rows n = 2 k0 + (re, im) = 32 c + 16 odd .. + 15, i.e. 16-byte pieces
                // q0 and q0 + 1 (q0 = (c % 2) 4 + 2 odd) of row half c / 2, K row m = j, swizzled by j % 8
                uint32_t v[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float2 y = cmul(cmul(Y[i], pw[i]), bs[c]);
                    const __half2 hv = __floats2half2_rn(y.x, y.y);
                    v[i] = *reinterpret_cast<const uint32_t *>(&hv);
                }
                uint8_t *rowp = gbase + kOffA2 + (uint32_t)(c >> 1) * 8192u + (uint32_t)j * 128u;
                const int q0 = (c & 1) * 4 + 2 * odd;
                *reinterpret_cast<uint4 *>(rowp + ((q0 ^ (j & 7)) << 4)) = make_uint4(v[0], v[1], v[2], v[3]);
                *reinterpret_cast<uint4 *>(rowp + (((q0 + 1) ^ (j & 7)) << 4)) = make_uint4(v[4], v[5], v[6], v[7]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_op));
            // ---- stage-2 accumulator -> output planes
            if (!warp_wait(smem_u32(&bar_acc), acc_phase, abort, err, lane)) break;
            acc_phase ^= 1u;
            fence_after_sync();
            __half *o = out + row * 2 * (long long)g.pitch;
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                uint32_t r[32];
                tmem_ld32(tq + 32u * c, r);
                float2 X[8];
                combine_pair(r, odd, X);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int a = (j + 64 * (16 * c + 8 * odd + i) + h) & (kN - 1);
                    if (a < g.n_sc) {
                        const __half2 v = __floats2half2_rn(X[i].x, X[i].y);
                        o[a] = __low2half(v);
                        o[g.pitch + a] = __high2half(v);
                    }
                }
            }
            for (int a = g.n_sc + tid; a < g.pitch; a += 32 * kEpiWarps) {
                o[a] = __float2half_rn(0.f);
                o[g.pitch + a] = __float2half_rn(0.f);
            }
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&bar_op));
        }
    }

    fence_before_sync();
    __syncthreads();
    if (warp == kEpiWarps) {
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
    if (rows * 64 > 0x7fffffffLL) return cudaErrorInvalidValue;     // TMA row coordinate is 32-bit
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    cuuint64_t dims[2] = {128, (cuuint64_t)(rows * 64)};          // [rows * 64 a][128 mu] FP16
    cuuint64_t strides[1] = {256};
    cuuint32_t box[2] = {64, 64};
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
    // kCtasPerSm resident CTAs per SM (4 x 52 KB of shared memory; 4 x 128 TMEM columns = 512). The CTAs are
    // independent, so a CTA that cannot be resident at once simply runs later.
    long long grid = (long long)sms * (g.fft_cap > 0 && g.fft_cap < kCtasPerSm ? g.fft_cap : kCtasPerSm);
    if (grid > rows) grid = rows;
    FftTcArgs a;
    a.rows = rows;
    a.n_sc = g.n_sc;
    a.pitch = g.sc_pitch;
    fft_tc_kernel<<<(unsigned)grid, kThreads, kSmemBytes, st>>>(map, static_cast<__half *>(out), tw, a, err);
    return cudaGetLastError();
}

}  // namespace pusch
