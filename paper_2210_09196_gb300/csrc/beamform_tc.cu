// Beamforming, mixed form, on the 5th-generation tensor cores (tcgen05 + TMEM, operands staged by TMA).
//
// The per-symbol product Y = W^H X of Section II (Table I "BF") is computed as a real GEMM with the
// complex values embedded:  D[a][2b + c] = sum_k A[a][k] B[2b + c][k],  k = 2r + ri, where
//   A[a][2r + 0] = Re X[r][a],  A[a][2r + 1] = Im X[r][a]                        (the FFT output, FP16)
//   B[2b][2r] = Re W[r][b],  B[2b][2r+1] = Im W[r][b],  B[2b+1][2r] = -Im W[r][b],  B[2b+1][2r+1] = Re W[r][b]
// so that D[a][2b] = Re y_b and D[a][2b + 1] = Im y_b, i.e. each accumulator row is the c64 output row of
// subcarrier a. The MMA's M dimension is the subcarrier axis (tiles of 128), N = 2 N_B, K = 2 N_R.
//
// A is the mixed-form FFT output [rows][2 N_R][pitch] binary16 (subcarriers contiguous): an MN-major
// operand. TMA copies two 64-subcarrier x K boxes per tile with 128-byte swizzling into shared memory;
// B is built once per CTA from W (complex64) in the no-swizzle K-major core-matrix layout. One thread
// issues K/16 tcgen05.mma (kind::f16, FP32 accumulate) into TMEM; the four warps read their 32 TMEM lanes
// back with tcgen05.ld and store the rows. CTAs are persistent over tiles with a 2-stage TMA ring.
// Every wait is bounded (%globaltimer); on expiry the CTA records a timeout, drains and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"

namespace pusch {
namespace {

constexpr int kTcThreads = 128;
constexpr int kTileM = 128;
constexpr int kStages = 2;
constexpr uint64_t kWaitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase; false when the deadline passed first.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint64_t deadline) {
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() > deadline) return false;
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

// tcgen05 shared-memory matrix descriptor: start >> 4 [0,14), LBO >> 4 [16,30), SBO >> 4 [32,46),
// version 1 at [46,48), base offset 0, layout type at [61,64) (0 = no swizzle, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7u) << 61;
    return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = F16, A MN-major, B K-major, N >> 3 at [17,23),
// M >> 4 at [24,29).
__host__ __device__ constexpr uint32_t instr_desc_f16(int M, int N) {
    return (1u << 4) | (1u << 15) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

struct TcArgs {
    int n_rx, n_beams, n_sc, n_mtiles, tmem_cols;
    long long total_tiles;
};

__global__ void __launch_bounds__(kTcThreads, 2)
beamform_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs g, const float2 *__restrict__ W,
                   float2 *__restrict__ beam, uint32_t *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    const int K = 2 * g.n_rx;
    const int N = 2 * g.n_beams;
    const uint32_t a_bytes = (uint32_t)kTileM * K * 2;
    const uint32_t b_sbo = (uint32_t)K * 16;  // bytes between 8-row groups of B

    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    const uint32_t sA = base;
    const uint32_t sB = base + kStages * a_bytes;
    uint8_t *gB = gbase + kStages * a_bytes;
    const uint32_t sBar = sB + (uint32_t)N * K * 2;
    uint64_t *gBar = reinterpret_cast<uint64_t *>(gB + (size_t)N * K * 2);
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(gBar + kStages + 1);
    __shared__ int s_abort;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // ---- B operand from W: element (n, k) at (n/8)*SBO + (k/8)*128 + (n%8)*16 + (k%8)*2
    for (int idx = tid; idx < g.n_rx * g.n_beams; idx += kTcThreads) {
        const int r = idx / g.n_beams, b = idx - r * g.n_beams;
        const float2 w = __ldg(&W[idx]);
        const __half wr = __float2half_rn(w.x), wi = __float2half_rn(w.y), nwi = __float2half_rn(-w.y);
        auto put = [&](int n, int k, __half v) {
            *reinterpret_cast<__half *>(gB + (n >> 3) * b_sbo + (k >> 3) * 128 + (n & 7) * 16 + (k & 7) * 2) = v;
        };
        put(2 * b, 2 * r, wr);
        put(2 * b, 2 * r + 1, wi);
        put(2 * b + 1, 2 * r, nwi);
        put(2 * b + 1, 2 * r + 1, wr);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    if (tid == 0) {
        for (int s = 0; s <= kStages; ++s) mbar_init(sBar + 8 * s, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    const uint32_t mma_bar = sBar + 8 * kStages;
    const uint32_t idesc = instr_desc_f16(kTileM, N);

    const long long n_my =
        g.total_tiles > blockIdx.x ? (g.total_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    auto issue = [&](int s, long long i) {
        const long long t = blockIdx.x + i * gridDim.x;
        const long long row = t / g.n_mtiles;
        const int mt = (int)(t - row * g.n_mtiles);
        const uint32_t dst = sA + s * a_bytes;
        mbar_expect_tx(sBar + 8 * s, a_bytes);
        tma_load_2d(dst, &tmap, mt * kTileM, (int)(row * K), sBar + 8 * s);
        tma_load_2d(dst + (uint32_t)K * 128, &tmap, mt * kTileM + 64, (int)(row * K), sBar + 8 * s);
    };
    if (tid == 0)
        for (int s = 0; s < kStages && s < n_my; ++s) issue(s, s);

    long long issued = n_my < kStages ? n_my : kStages;
    long long i = 0;
    for (; i < n_my; ++i) {
        const int s = (int)(i % kStages);
        const uint32_t ph = (uint32_t)((i / kStages) & 1);
        const uint64_t deadline = globaltimer() + kWaitNs;
        int bad = 0;
        if (tid == 0) {
            if (mbar_wait(sBar + 8 * s, ph, deadline)) {
                fence_after_sync();
                const uint32_t a0 = sA + s * a_bytes;
                for (int ks = 0; ks < K / 16; ++ks) {
                    const uint64_t ad = smem_desc(a0 + ks * 2048, (uint32_t)K * 128, 1024, 2);
                    const uint64_t bd = smem_desc(sB + ks * 256, 128, b_sbo, 0);
                    mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
                mma_commit(mma_bar);
            } else {
                bad = 1;
            }
        }
        if (!bad && !mbar_wait(mma_bar, (uint32_t)(i & 1), deadline)) bad = 1;
        if (__syncthreads_or(bad)) {
            if (tid == 0) {
                s_abort = 1;
                atomicOr(err, 1u);
            }
            break;
        }
        fence_after_sync();
        if (tid == 0 && i + kStages < n_my) {
            issue(s, i + kStages);
            ++issued;
        }
        const long long t = blockIdx.x + i * gridDim.x;
        const long long row = t / g.n_mtiles;
        const int mt = (int)(t - row * g.n_mtiles);
        const int a = mt * kTileM + warp * 32 + lane;
        float *dst = reinterpret_cast<float *>(beam + (row * g.n_sc + a) * (long long)g.n_beams);
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t r[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
            const int ncol = N - c0 < 32 ? N - c0 : 32;  // N is a multiple of 16: 16 or 32 columns here
            if (a < g.n_sc) {
#pragma unroll
                for (int j = 0; j < 32; j += 4)
                    if (j < ncol)
                        *reinterpret_cast<float4 *>(dst + c0 + j) =
                            make_float4(__uint_as_float(r[j]), __uint_as_float(r[j + 1]), __uint_as_float(r[j + 2]),
                                        __uint_as_float(r[j + 3]));
            }
        }
        fence_before_sync();
        __syncthreads();
    }

    if (s_abort && tid == 0) {
        // drain the TMA loads still in flight for this CTA (bounded), so no copy lands after exit
        const uint64_t d2 = globaltimer() + kWaitNs;
        for (long long j = i; j < issued; ++j)
            mbar_wait(sBar + 8 * (int)(j % kStages), (uint32_t)((j / kStages) & 1), d2);
        mbar_wait(mma_bar, (uint32_t)(i & 1), d2);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols));
    }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

size_t tc_smem_bytes(const Geometry &g) {
    const size_t K = 2 * (size_t)g.n_rx, N = 2 * (size_t)g.n_beams;
    return 1024 + kStages * (size_t)kTileM * K * 2 + N * K * 2 + 8 * (kStages + 1) + 16;
}

}  // namespace

bool bf_tc_supported(const Geometry &g) {
    return g.n_rx % 8 == 0 && g.n_rx >= 8 && g.n_rx <= 128 && g.n_beams % 8 == 0 && g.n_beams >= 8 &&
           g.n_beams <= 64 && tc_smem_bytes(g) <= 227 * 1024;
}

cudaError_t launch_beamform_tc(const Geometry &g, int n_slots, const __half *freq16, const float2 *W, float2 *beam,
                               uint32_t *err_word, cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    if (!bf_tc_supported(g)) return cudaErrorNotSupported;
    if (reinterpret_cast<uintptr_t>(freq16) % 16 != 0 || reinterpret_cast<uintptr_t>(beam) % 16 != 0)
        return cudaErrorMisalignedAddress;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const int K = 2 * g.n_rx;
    const long long rows = (long long)n_slots * g.n_sym;
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)g.sc_pitch, (cuuint64_t)(rows * K)};
    cuuint64_t strides[1] = {(cuuint64_t)g.sc_pitch * 2};
    cuuint32_t box[2] = {64, (cuuint32_t)K};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half *>(freq16), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    TcArgs a;
    a.n_rx = g.n_rx;
    a.n_beams = g.n_beams;
    a.n_sc = g.n_sc;
    a.n_mtiles = (g.n_sc + kTileM - 1) / kTileM;
    a.total_tiles = rows * a.n_mtiles;
    int cols = 32;
    while (cols < 2 * g.n_beams) cols *= 2;
    a.tmem_cols = cols;
    const size_t smem = tc_smem_bytes(g);
    cudaError_t e = cudaFuncSetAttribute(beamform_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = 2LL * sms;
    if (grid > a.total_tiles) grid = a.total_tiles;
    beamform_tc_kernel<<<(unsigned)grid, kTcThreads, smem, st>>>(map, a, W, beam, err_word);
    return cudaGetLastError();
}

}  // namespace pusch
