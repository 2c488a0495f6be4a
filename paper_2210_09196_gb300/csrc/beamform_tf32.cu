// Beamforming of the plain FP32 form on the 5th-generation tensor cores with three TF32 products per FP32
// product (Section II, Table I "BF": Y = W^H X per symbol).
//
// The complex product is the real GEMM of the mixed form, D[a][2b + c] = sum_k A[a][k] B[2b + c][k] with
// k = 2r + ri, A[a][2r] = Re X[r][a], A[a][2r + 1] = Im X[r][a], B[2b][2r] = Re W[r][b], B[2b][2r + 1] =
// Im W[r][b], B[2b + 1][2r] = -Im W[r][b], B[2b + 1][2r + 1] = Re W[r][b]. Every FP32 operand v is split
// into two TF32 values, hi = TF32(v) and lo = TF32(v - hi) (round to nearest), so that hi + lo holds v to
// about 2^-22, and D = A_hi B_hi + A_hi B_lo + A_lo B_hi (the dropped A_lo B_lo is below 2^-22 of |A||B|)
// with FP32 accumulation in TMEM: three tcgen05.mma kind::tf32 per K step of 8.
//
// Warp roles (persistent CTAs, one per SM):
//   warp 0      TMA producer: the (tile, K chunk) sequence of c64 FFT rows (16 antennas x 128 subcarriers
//               per chunk, no swizzle) into a landing ring;
//   warp 1      owns the TMEM allocation; one lane issues the MMAs of each chunk into one of two TMEM
//               accumulators and commits the chunk's operand stage back to the convert warps;
//   warps 2-5   epilogue: tcgen05.ld of the finished accumulator (one 32-lane quarter per warp), stores of
//               the c64 beam rows;
//   warps 6-13  split each landed chunk into the hi and lo operands (K-major core matrices, no swizzle).
// B (hi and lo, K-major) is built once per CTA from W staged through the still idle operand ring.
// Every wait is bounded (%globaltimer, 2 s); on expiry the CTA records a timeout in err_word bit 0, all roles
// leave their loops, in-flight copies and MMAs are drained (bounded) and TMEM is freed.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "tc_common.cuh"

namespace pusch {
namespace {

using namespace tc;

constexpr int kTileM = 128;
constexpr int kCR = 16;                 // antennas per K chunk
constexpr int kKC = 2 * kCR;            // K values per chunk
constexpr int kMaxStages = 8;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kConvWarps = 8;        // warps that split the landed chunks (12 measured within 2 %)
constexpr int kThreads = 192 + 32 * kConvWarps;
constexpr uint32_t kABytes = (uint32_t)kTileM * kKC * 4;   // one operand (hi or lo) of a chunk: 16 KB
constexpr uint32_t kASbo = (uint32_t)(kKC / 4) * 128;      // bytes between 8-row groups of an A stage
constexpr uint32_t kLandBytes = (uint32_t)kCR * kTileM * 8; // landed c64 chunk: 16 KB

struct Tf32Args {
    int n_rx, n_beams, n_sc, n_mtiles, K, N, n_chunks, n_stages, n_land, tmem_cols;
    uint32_t b_bytes;      // one of B's two operands (hi or lo)
    uint32_t land_off;     // offset of the landing ring from the aligned base
    long long total_tiles;
};

struct Tf32Shared {
    uint64_t full[kMaxStages], lempty[kMaxStages], ready[kMaxStages], empty[kMaxStages];
    uint64_t tfull[2], tempty[2], drain;
    uint32_t tmem_base;
    int abort;
};

// TF32 rounding of an FP32 value (round to nearest, ties away): the FP32 bit pattern with the low 13 mantissa
// bits cleared.
__device__ __forceinline__ uint32_t tf32_of(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ void split_tf32(float x, uint32_t &hi, uint32_t &lo) {
    hi = tf32_of(x);
    lo = tf32_of(x - __uint_as_float(hi));
}

// Instruction descriptor of kind::tf32: D F32 (bits 4-5 = 1), A and B TF32 (format code 2 at bits 7-9 and
// 10-12), both K-major, N >> 3 at [17,23), M >> 4 at [24,29).
constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__global__ void __launch_bounds__(kThreads, 1)
beamform_tf32_kernel(const __grid_constant__ CUtensorMap tmap, Tf32Args g, const float2 *__restrict__ W,
                     float2 *__restrict__ beam, uint32_t *__restrict__ err) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ Tf32Shared sh;

    const int K = g.K, N = g.N;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t *gbase = smem_raw + (base - raw);
    // [A ring: n_stages x (hi, lo)][B hi][B lo][landing ring]
    const uint32_t sA = base;
    const uint32_t sB = base + (uint32_t)g.n_stages * 2u * kABytes;
    uint8_t *gB = gbase + (size_t)g.n_stages * 2u * kABytes;
    const uint32_t b_sbo = (uint32_t)(K / 4) * 128u;     // bytes between 8-row groups of B

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    volatile int *abort = &sh.abort;

    // ---------------------------------------------------------------- B (hi, lo) from W
    // W [n_rx][n_beams] (smaller than the operand ring whenever B fits) is staged with 8-byte cp.async; unit
    // (n, kq) writes the 16-byte core-matrix row of beam row n for antennas 2 kq, 2 kq + 1: element (n, k) at
    // (n/8)*SBO + (k/4)*128 + (n%8)*16 + (k%4)*4.
    {
        float2 *Ws = reinterpret_cast<float2 *>(gbase);
        const int cnt = g.n_rx * g.n_beams;
        for (int i = tid; i < cnt; i += kThreads)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(Ws + i)), "l"(W + i) : "memory");
        asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        const int units = N * (K / 4);
        for (int u = tid; u < units; u += kThreads) {
            const int kq = u / N, n = u - kq * N;
            const int b = n >> 1;
            const float2 w0 = Ws[(2 * kq) * g.n_beams + b], w1 = Ws[(2 * kq + 1) * g.n_beams + b];
            // row 2b: (Re, Im); row 2b + 1: (-Im, Re)
            const float v[4] = {(n & 1) ? -w0.y : w0.x, (n & 1) ? w0.x : w0.y, (n & 1) ? -w1.y : w1.x,
                                (n & 1) ? w1.x : w1.y};
            uint32_t hi[4], lo[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) split_tf32(v[e], hi[e], lo[e]);
            const size_t off = (size_t)(n >> 3) * b_sbo + (size_t)kq * 128 + (n & 7) * 16;
            *reinterpret_cast<uint4 *>(gB + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
            *reinterpret_cast<uint4 *>(gB + g.b_bytes + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
        }
        __syncthreads();                                 // B complete; the ring is free again
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");

    if (tid == 0) {
        for (int s = 0; s < kMaxStages; ++s) {
            mbar_init(smem_u32(&sh.full[s]), 1);
            mbar_init(smem_u32(&sh.lempty[s]), kConvWarps);
            mbar_init(smem_u32(&sh.ready[s]), kConvWarps);
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
                     "r"(g.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = sh.tmem_base;

    const long long n_my =
        g.total_tiles > blockIdx.x ? (g.total_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const int NS = g.n_stages, NR = g.n_land;

    if (warp == 0) {
        // ------------------------------------------------------------------ TMA producer
        if (lane == 0) {
            long long gch = 0;
            bool ok = true;
            for (long long i = 0; i < n_my && ok; ++i) {
                const long long t = blockIdx.x + i * gridDim.x;
                const long long row = t / g.n_mtiles;    // (slot, symbol)
                const int mt = (int)(t - row * g.n_mtiles);
                for (int c = 0; c < g.n_chunks; ++c, ++gch) {
                    const int s = (int)(gch % NR);
                    const uint32_t ph = (uint32_t)((gch / NR) & 1);
                    if (!mbar_wait(smem_u32(&sh.lempty[s]), ph ^ 1u, abort, err)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bar = smem_u32(&sh.full[s]);
                    mbar_expect_tx(bar, kLandBytes);
                    tma_load_2d(base + g.land_off + (uint32_t)s * kLandBytes, &tmap, mt * 2 * kTileM,
                                (int)(row * g.n_rx) + c * kCR, bar);
                }
            }
            if (*abort) {
                for (long long j = gch - 1; j >= 0 && j >= gch - NR; --j)
                    mbar_drain(smem_u32(&sh.full[(int)(j % NR)]), (uint32_t)((j / NR) & 1));
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t idesc = idesc_tf32(kTileM, N);
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
                    if (!mbar_wait(smem_u32(&sh.ready[s]), ph, abort, err)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint32_t a_hi = sA + (uint32_t)s * 2u * kABytes, a_lo = a_hi + kABytes;
#pragma unroll
                    for (int ks = 0; ks < kKC / 8; ++ks) {
                        const uint32_t kb = (uint32_t)(c * (kKC / 8) + ks) * 256u;
                        const uint64_t ah = smem_desc(a_hi + (uint32_t)ks * 256u, 128, kASbo, 0);
                        const uint64_t al = smem_desc(a_lo + (uint32_t)ks * 256u, 128, kASbo, 0);
                        const uint64_t bh = smem_desc(sB + kb, 128, b_sbo, 0);
                        const uint64_t bl = smem_desc(sB + g.b_bytes + kb, 128, b_sbo, 0);
                        mma_tf32(d, ah, bh, idesc, (c > 0 || ks > 0) ? 1u : 0u);
                        mma_tf32(d, ah, bl, idesc, 1u);
                        mma_tf32(d, al, bh, idesc, 1u);
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
        const int q = warp & 3;                          // TMEM lane quarter this warp may access
        for (long long i = 0; i < n_my; ++i) {
            const int buf = (int)(i & 1);
            const long long t = blockIdx.x + i * gridDim.x;
            const long long row = t / g.n_mtiles;
            const int mt = (int)(t - row * g.n_mtiles);
            const bool okw = mbar_wait(smem_u32(&sh.tfull[buf]), (uint32_t)((i >> 1) & 1), abort, err);
            if (!__all_sync(0xFFFFFFFFu, okw)) break;     // warp-uniform: tcgen05.ld is warp-collective
            fence_after_sync();
            const int a = mt * kTileM + q * 32 + lane;
            float *dst = reinterpret_cast<float *>(beam + (row * g.n_sc + a) * (long long)g.n_beams);
            const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * N);
            for (int c0 = 0; c0 < N; c0 += 32) {
                uint32_t r[32];
                const int ncol = N - c0 < 32 ? N - c0 : 32;   // N is a multiple of 16
                if (ncol == 32) tmem_ld32(tbase + (uint32_t)c0, r);
                else tmem_ld16(tbase + (uint32_t)c0, r);
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
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sh.tempty[buf]));
        }
    } else {
        // ------------------------------------------------------------------ split into TF32 hi and lo
        // Unit u = (antenna pair p, subcarrier m), u = 128 p + m: the landed values X[2p][m], X[2p + 1][m]
        // (row r of the landing stage at r * 1024, subcarrier m at m * 8) become the core-matrix row of k = 4p
        // .. 4p + 3 at (m/8)*1024 + p*128 + (m%8)*16 of the hi and the lo operand. Antennas past n_rx (the last
        // chunk of a symbol whose antenna count is not a multiple of 16 reads the next symbol's rows) are zero.
        const int w4 = warp - 6;
        long long gch = 0;
        bool ok = true;
        for (long long i = 0; i < n_my && ok; ++i) {
            for (int c = 0; c < g.n_chunks; ++c, ++gch) {
                const int s = (int)(gch % NS), sl = (int)(gch % NR);
                const uint32_t ph = (uint32_t)((gch / NS) & 1), phl = (uint32_t)((gch / NR) & 1);
                // the chunk has landed, and the MMAs of the operand stage's previous chunk have completed
                bool okw = mbar_wait(smem_u32(&sh.full[sl]), phl, abort, err);
                okw = okw && mbar_wait(smem_u32(&sh.empty[s]), ph ^ 1u, abort, err);
                if (!__all_sync(0xFFFFFFFFu, okw)) {
                    ok = false;
                    break;
                }
                const uint8_t *land = gbase + g.land_off + (size_t)sl * kLandBytes;
                uint8_t *ahi = gbase + (size_t)s * 2u * kABytes, *alo = ahi + kABytes;
                const int r_left = g.n_rx - c * kCR;     // antennas of this chunk that exist
#pragma unroll 2
                for (int u = w4 * 32 + lane; u < kTileM * (kCR / 2); u += 32 * kConvWarps) {
                    const int p = u >> 7, m = u & 127;
                    float2 x0 = *reinterpret_cast<const float2 *>(land + (size_t)(2 * p) * 1024 + m * 8);
                    float2 x1 = *reinterpret_cast<const float2 *>(land + (size_t)(2 * p + 1) * 1024 + m * 8);
                    if (2 * p >= r_left) x0 = make_float2(0.f, 0.f);
                    if (2 * p + 1 >= r_left) x1 = make_float2(0.f, 0.f);
                    uint32_t hi[4], lo[4];
                    split_tf32(x0.x, hi[0], lo[0]);
                    split_tf32(x0.y, hi[1], lo[1]);
                    split_tf32(x1.x, hi[2], lo[2]);
                    split_tf32(x1.y, hi[3], lo[3]);
                    const size_t off = (size_t)(m >> 3) * kASbo + (size_t)p * 128 + (m & 7) * 16;
                    *reinterpret_cast<uint4 *>(ahi + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                    *reinterpret_cast<uint4 *>(alo + off) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
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

struct Tf32Plan {
    bool ok;
    int n_stages, n_land, tmem_cols;
    uint32_t b_bytes, land_off;
    size_t smem;
};

// Two operand stages (hi + lo, 32 KB each), B (hi + lo), and as many landing stages as the rest of shared memory
// holds (at most 8): the landing ring's bytes in flight set the load bandwidth.
Tf32Plan tf32_plan(const Geometry &g) {
    Tf32Plan p{};
    const int K = 2 * g.n_rx, N = 2 * g.n_beams;
    p.b_bytes = (uint32_t)((size_t)N * K * 4);
    int cols = 32;
    while (cols < 2 * N) cols *= 2;
    p.tmem_cols = cols;
    p.n_stages = 2;
    const size_t fixed = 1024 + sizeof(Tf32Shared) + 256 + (size_t)p.n_stages * 2 * kABytes + 2 * (size_t)p.b_bytes;
    const long long rest = (long long)kSmemLimit - (long long)fixed;
    int nl = rest > 0 ? (int)(rest / kLandBytes) : 0;
    if (nl > kMaxStages) nl = kMaxStages;
    p.n_land = nl;
    p.land_off = (uint32_t)((size_t)p.n_stages * 2 * kABytes + 2 * (size_t)p.b_bytes);
    p.smem = 1024 + (size_t)p.land_off + (size_t)nl * kLandBytes;
    // W is staged through the operand ring before B is built
    const bool w_fits = (size_t)g.n_rx * g.n_beams * 8 <= (size_t)p.n_stages * 2 * kABytes;
    p.ok = cols <= 256 && nl >= 2 && w_fits;
    return p;
}

}  // namespace

bool bf_tf32_supported(const Geometry &g) {
    if (g.form != PUSCH_FORM_FP32) return false;
    if (g.n_sc % 2 != 0 || g.n_rx % kCR != 0 || g.n_beams % 8 != 0 || g.n_beams < 8 || g.n_beams > 64) return false;
    return tf32_plan(g).ok;
}

cudaError_t launch_beamform_tf32(const Geometry &g, int n_slots, const float2 *freq, const float2 *W, float2 *beam,
                                 uint32_t *err_word, cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    if (!bf_tf32_supported(g)) return cudaErrorNotSupported;
    if (reinterpret_cast<uintptr_t>(freq) % 16 != 0 || reinterpret_cast<uintptr_t>(beam) % 16 != 0 ||
        reinterpret_cast<uintptr_t>(W) % 8 != 0)
        return cudaErrorMisalignedAddress;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    const Tf32Plan p = tf32_plan(g);
    const long long rows = (long long)n_slots * g.n_sym;          // (slot, symbol) rows of the output
    // the FFT output [rows][n_rx][n_sc] c64 as float rows of 2 n_sc; a box is 16 antennas x 128 subcarriers
    CUtensorMap map;
    cuuint64_t dims[2] = {(cuuint64_t)(2 * g.n_sc), (cuuint64_t)(rows * g.n_rx)};
    cuuint64_t strides[1] = {(cuuint64_t)g.n_sc * 8};
    cuuint32_t box[2] = {(cuuint32_t)(2 * kTileM), (cuuint32_t)kCR};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float2 *>(freq), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
    Tf32Args a;
    a.n_rx = g.n_rx;
    a.n_beams = g.n_beams;
    a.n_sc = g.n_sc;
    a.n_mtiles = (g.n_sc + kTileM - 1) / kTileM;
    a.K = 2 * g.n_rx;
    a.N = 2 * g.n_beams;
    a.n_chunks = g.n_rx / kCR;
    a.n_stages = p.n_stages;
    a.n_land = p.n_land;
    a.tmem_cols = p.tmem_cols;
    a.b_bytes = p.b_bytes;
    a.land_off = p.land_off;
    a.total_tiles = rows * a.n_mtiles;
    cudaError_t e = cudaFuncSetAttribute(beamform_tf32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long grid = sms;
    if (grid > a.total_tiles) grid = a.total_tiles;
    beamform_tf32_kernel<<<(unsigned)grid, kThreads, p.smem, st>>>(map, a, W, beam, err_word);
    return cudaGetLastError();
}

}  // namespace pusch
