// Ragged multi-cell batches (pusch_batch_*): cells of different sizes, users on their own contiguous
// subcarrier ranges with their own layer counts, the whole receive chain in one CUDA graph launch.
//
// Host side: the users of each cell are cut into constant-user-set segments (a segment is a subcarrier
// range covered by the same users); at every subcarrier all layers of all covering users are detected
// jointly (Eq. 2 with N_L = those layers). Device descriptor tables list, per segment, its layers (user,
// port, allocation range, LS table and output offsets), and per layer class (2, 4, 8, 16, 32 lanes per
// subcarrier) the work items (segment, first subcarrier of a group).
// Device side, captured into one graph: per cell the FFT and beamforming kernels of the single-cell path;
// one LS-at-pilots kernel over every (user, layer); one persistent detector per layer class whose warps pull
// work items from an atomic counter (no waits), with the detection core of the single-cell path. The cells'
// FFT/beamforming chains and the layer classes' detectors run on parallel graph branches.
//
// Autotuning (pusch_batch_autotune): the launch shapes are timed on the batch's own buffers and the fastest
// kept: per distinct cell shape (form, N_R, N_B, N_SC) the tensor-core GEMM's K rows per stage and output
// path, per layer class the detector's warps per CTA and CTAs per SM, and the number of graph branches.
// Choices are written to / read from a text cache, one line per key.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "chest_common.cuh"
#include "detect_core.cuh"
#include "detect_tc.cuh"
#include "tune_cache.cuh"

namespace {

using pusch::Geometry;

constexpr int kClasses = 5;        // NL = 2, 4, 8, 16, 32
constexpr int kDetMaxWarps = 4;    // detector CTAs have 1, 2 or 4 warps (a tuned launch shape)
constexpr int kMaxBranches = 8;
constexpr int kMaxData = 14;

struct SegLayer {                  // one layer of a segment
    long long ls_off;              // LS table row of the layer's first pilot
    long long out_off;             // x_hat / bits offset of (user, layer, symbol 0, sc_start)
    int first, last;               // first / last pilot subcarrier of the layer inside its user's range
    int a0, n;                     // the user's range
    int qam;
    int pad;
};

struct Segment {
    long long beam_off;            // float2 offset of the cell's beamformed grid
    int cell, a0, n, nl, layer0, nb, n_sc, comb;
    float load;
    int pad;
};

struct LsJob {                     // LS values at the pilots of one (user, layer)
    long long beam_off, pil_off, ls_off;
    int n_sc, nb, first, npil, comb, a0, n, pad;
};

struct DetArgs {
    int n_sym, n_data, dmrs0, dmrs1;
    int dmrs_lo, dmrs_hi;  // the two DMRS symbols in increasing order
};

// Symbol index of data symbol d (all non-DMRS symbols in increasing order), computed: a run-time index into
// a kernel parameter array would copy the parameter block to local memory.
__device__ __forceinline__ int data_symbol(const DetArgs &g, int d) {
    int s = d;
    if (s >= g.dmrs_lo) ++s;
    if (s >= g.dmrs_hi) ++s;
    return s;
}

// ------------------------------------------------------------------------------------------------ kernels

__global__ void batch_reset_kernel(int *counters, uint32_t *status) {
    if (threadIdx.x < kClasses) counters[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        status[0] = 0u;
        status[1] = 0u;
        status[2] = 0xffffffffu;
        status[3] = 0u;
    }
}

// One CTA per (user, layer): ls[k][b] = 1/2 (y0[q][b] / p0[q] + y1[q][b] / p1[q]), q = first + k * comb.
__global__ void __launch_bounds__(256)
batch_ls_kernel(const LsJob *__restrict__ jobs, DetArgs g, const float2 *__restrict__ beam,
                const float2 *__restrict__ pilots, float2 *__restrict__ ls) {
    const LsJob j = jobs[blockIdx.x];
    const float2 *y0 = beam + j.beam_off + (long long)g.dmrs0 * j.n_sc * j.nb;
    const float2 *y1 = beam + j.beam_off + (long long)g.dmrs1 * j.n_sc * j.nb;
    const float2 *p0 = pilots + j.pil_off;
    const float2 *p1 = p0 + j.n;
    for (int idx = threadIdx.x; idx < j.npil * j.nb; idx += blockDim.x) {
        const int k = idx / j.nb, b = idx - k * j.nb;
        const int q = j.first + k * j.comb;
        ls[j.ls_off + idx] = pusch::ls_value(__ldg(&y0[(long long)q * j.nb + b]), __ldg(&y1[(long long)q * j.nb + b]),
                                             pusch::pilot_inverse(__ldg(&p0[q - j.a0])),
                                             pusch::pilot_inverse(__ldg(&p1[q - j.a0])));
    }
}

struct BRow {                      // interpolation parameters of one (subcarrier, layer) row
    long long lo, hi;
    float w;
    int valid;
};

template <int NL>
__host__ __device__ __forceinline__ size_t batch_warp_smem(int nbmax, int nd) {
    return (size_t)(32 / NL) * ((pusch::htile<NL>(nbmax) + (size_t)nd * pusch::y_stride<NL>(nbmax)) * sizeof(float2) +
                                NL * sizeof(BRow));
}

// Persistent detector for one layer class. Each warp takes work items (segment, first subcarrier of a group
// of 32/NL subcarriers) from *counter until the list is exhausted.
template <int NL, int ND>
__global__ void __launch_bounds__(kDetMaxWarps * 32)
batch_detect_kernel(DetArgs g, int nbmax, const Segment *__restrict__ segs, const SegLayer *__restrict__ layers,
                    const int2 *__restrict__ items, int n_items, int *__restrict__ counter,
                    const float2 *__restrict__ beam, const float2 *__restrict__ ls, float2 *__restrict__ xhat,
                    uint8_t *__restrict__ bits, uint32_t *__restrict__ status) {
    constexpr int SPW = 32 / NL;
    constexpr int NR = ND > 0 ? ND : kMaxData;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int grp = lane / NL, i = lane - grp * NL;
    const int src0 = grp * NL;
    const int nd = ND > 0 ? ND : g.n_data;
    const int ht = pusch::htile<NL>(nbmax);
    unsigned char *wbase = smem_raw + (size_t)warp * batch_warp_smem<NL>(nbmax, nd);
    float2 *Ht = reinterpret_cast<float2 *>(wbase);
    float2 *Yt = Ht + SPW * ht;
    BRow *rp = reinterpret_cast<BRow *>(Yt + (size_t)SPW * nd * pusch::y_stride<NL>(nbmax));

    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(counter, 1);
        item = __shfl_sync(pusch::kDetFull, item, 0);
        if (item >= n_items) break;
        const int2 it = items[item];
        const Segment sg = segs[it.x];
        const int nb = sg.nb, nl = sg.nl, hs = pusch::row_stride(nb), ys = pusch::y_stride<NL>(nb);
        const int a = it.y + grp;
        const bool valid = a < sg.a0 + sg.n;

        // 0. y rows of the group's subcarrier -> shared memory (cp.async: 16-byte pieces of two beams when the
        //    segment's beam count and its rows' start are even, else 8-byte pieces)
        {
            const bool wide = (nb & 1) == 0 && (sg.beam_off & 1) == 0;
            const int pw = wide ? 2 : 1;                 // beams per piece
            const int ppr = nb / pw;                     // pieces per row
            for (int idx = lane; idx < SPW * nd * ppr; idx += 32) {
                const int gg = idx / (nd * ppr);
                const int rem = idx - gg * nd * ppr;
                const int d = rem / ppr, b = (rem - d * ppr) * pw;
                const int aa = it.y + gg;
                float2 *dst = Yt + (gg * nd + d) * ys + b;
                const float2 *src = beam + sg.beam_off + ((long long)data_symbol(g, d) * sg.n_sc + aa) * nb + b;
                if (aa < sg.a0 + sg.n) {
                    if (wide)
                        pusch::cp_async16(dst, src);
                    else
                        pusch::cp_async8(dst, src);
                } else {
                    dst[0] = make_float2(0.f, 0.f);
                    if (wide) dst[1] = make_float2(0.f, 0.f);
                }
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // 1. interpolated estimate rows (LS table of each layer's own user)
        {
            BRow q;
            q.valid = (valid && i < nl) ? 1 : 0;
            q.lo = q.hi = 0;
            q.w = 0.f;
            if (q.valid) {
                const SegLayer L = layers[sg.layer0 + i];
                int lo, hi;
                if (a <= L.first) {
                    lo = hi = L.first;
                } else if (a >= L.last) {
                    lo = hi = L.last;
                } else {
                    lo = L.first + ((a - L.first) / sg.comb) * sg.comb;
                    hi = (lo == a) ? lo : lo + sg.comb;
                }
                q.lo = L.ls_off + (long long)((lo - L.first) / sg.comb) * nb;
                q.hi = L.ls_off + (long long)((hi - L.first) / sg.comb) * nb;
                q.w = pusch::interp_weight(a, lo, hi);
            }
            rp[lane] = q;
        }
        __syncwarp();
        // kB elements per lane at a time: their LS-table loads are all issued before any is used
        constexpr int kB = 8;
        for (int idx0 = lane; idx0 < SPW * NL * nb; idx0 += 32 * kB) {
            float2 lo[kB], hi[kB];
            float w[kB];
            int off[kB];
#pragma unroll
            for (int u = 0; u < kB; ++u) {
                const int idx = idx0 + 32 * u;
                off[u] = -1;
                lo[u] = hi[u] = make_float2(0.f, 0.f);
                w[u] = 0.f;
                if (idx < SPW * NL * nb) {
                    const int r = idx / nb, b = idx - r * nb;
                    const int gg = r / NL, l = r - gg * NL;
                    off[u] = gg * ht + l * hs + b;
                    const BRow &q = rp[r];
                    if (q.valid) {
                        lo[u] = __ldg(&ls[q.lo + b]);
                        hi[u] = q.hi != q.lo ? __ldg(&ls[q.hi + b]) : lo[u];
                        w[u] = q.w;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kB; ++u)
                if (off[u] >= 0) Ht[off[u]] = pusch::interp(lo[u], hi[u], w[u]);
        }
        __syncwarp();

        // 2-4. Gram, right-hand sides, Cholesky, solves
        float2 acc[NR];
        bool bad;
        bool tc = false;   // 16 and 32 lanes, 12 data symbols, a beam count that is a multiple of 4: G and r_d
        if constexpr (ND == 12 && NL >= 16) {   // on the tensor cores
            tc = (nb & 3) == 0 && ht >= NL * (NL + 2);
            if (tc) bad = pusch::detect_group_tc<NL, 0>(Ht, ht, hs, Yt, ys, nl, sg.load, grp, i, src0, lane, acc, nullptr, 0, nb);
        }
        if (!tc)
            bad = pusch::detect_group<NL, ND, NR>(Ht + grp * ht + i * hs, Ht + grp * ht, Yt + grp * nd * ys,
                                                  Ht + grp * ht, hs, nb, nd, nl, sg.load, i, src0, acc, nullptr, 0, ys);
        if (valid && bad && i == 0) {
            atomicAdd(&status[1], 1u);
            atomicMin(&status[2], (unsigned)(sg.cell * 65536 + a));
            atomicOr(&status[0], (unsigned)PUSCH_STATUS_PIVOT);
        }
        bool nonfinite = false;
        if (valid && i < nl) {
            const SegLayer L = layers[sg.layer0 + i];
            const long long o0 = L.out_off + (a - L.a0);
#pragma unroll
            for (int d = 0; d < NR; ++d) {
                if (ND > 0 || d < nd) {
                    const float2 x = acc[d];
                    xhat[o0 + (long long)d * L.n] = x;
                    bits[o0 + (long long)d * L.n] = pusch::det_demap(x, L.qam);
                    if (!isfinite(x.x) || !isfinite(x.y)) nonfinite = true;
                }
            }
        }
        if (__any_sync(pusch::kDetFull, nonfinite) && lane == 0) atomicOr(&status[0], (unsigned)PUSCH_STATUS_NONFINITE);
        __syncwarp();  // shared tiles are rewritten by the next item
    }
}

template <int NL, int ND>
cudaError_t launch_detect_nl(const DetArgs &g, int nbmax, const Segment *segs, const SegLayer *layers,
                             const int2 *items, int n_items, int *counter, const float2 *beam, const float2 *ls,
                             float2 *xhat, uint8_t *bits, uint32_t *status, int warps, int ctas_per_sm,
                             cudaStream_t st) {
    const int nd = ND > 0 ? ND : g.n_data;
    const size_t per_warp = batch_warp_smem<NL>(nbmax, nd);
    const size_t limit = 227 * 1024;                  // dynamic shared memory a CTA may opt in to
    const int fit = (int)std::min<size_t>(kDetMaxWarps, limit / per_warp);
    if (fit < 1) return cudaErrorInvalidValue;
    if (warps > fit) warps = fit;                     // a shape that does not fit runs with fewer warps
    const size_t smem = (size_t)warps * per_warp;
    auto k = batch_detect_kernel<NL, ND>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)((size_t)fit * per_warp));
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 152, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, warps * 32, smem);
    if (per_sm < 1) per_sm = 1;
    if (ctas_per_sm > 0 && ctas_per_sm < per_sm) per_sm = ctas_per_sm;
    long long grid = (long long)sms * per_sm;
    const long long need = ((long long)n_items + warps - 1) / warps;
    if (grid > need) grid = need;
    k<<<(unsigned)grid, warps * 32, smem, st>>>(g, nbmax, segs, layers, items, n_items, counter, beam, ls, xhat, bits,
                                                status);
    return cudaGetLastError();
}

template <int NL>
cudaError_t launch_detect(const DetArgs &g, int nbmax, const Segment *segs, const SegLayer *layers,
                          const int2 *items, int n_items, int *counter, const float2 *beam, const float2 *ls,
                          float2 *xhat, uint8_t *bits, uint32_t *status, int warps, int ctas_per_sm,
                          cudaStream_t st) {
    if (g.n_data == 12)
        return launch_detect_nl<NL, 12>(g, nbmax, segs, layers, items, n_items, counter, beam, ls, xhat, bits, status,
                                        warps, ctas_per_sm, st);
    return launch_detect_nl<NL, 0>(g, nbmax, segs, layers, items, n_items, counter, beam, ls, xhat, bits, status,
                                   warps, ctas_per_sm, st);
}

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct pusch_batch {
    std::vector<pusch_cell_cfg> cells;
    std::vector<Geometry> geo;
    std::vector<pusch_user_desc> users;
    std::vector<long long> t_off, w_off, beam_off;  // elements (complex)
    std::vector<size_t> f_off;                      // bytes
    size_t sizes[5] = {0, 0, 0, 0, 0};
    DetArgs det;
    int nbmax = 0;
    int n_jobs = 0;
    int n_items[kClasses] = {0, 0, 0, 0, 0};
    std::map<int, float2 *> twiddle;  // per FFT size
    unsigned char *freq = nullptr;
    float2 *beam = nullptr, *ls = nullptr;
    Segment *d_segs = nullptr;
    SegLayer *d_layers = nullptr;
    LsJob *d_jobs = nullptr;
    int2 *d_items[kClasses] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    int *d_counters = nullptr;
    uint32_t *kernel_err = nullptr, *status_sink = nullptr;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void *key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    // launch shapes (defaults until pusch_batch_autotune chooses)
    std::vector<pusch::TcTune> bf_tune;                      // per cell
    int det_warps[kClasses] = {2, 2, 2, 2, 2};
    int det_ctas[kClasses] = {0, 0, 0, 0, 0};                // CTAs per SM cap, 0 = occupancy limit
    int branches = 4;                                         // parallel graph branches
    cudaStream_t fork[kMaxBranches] = {};
    cudaEvent_t ev[2 + kMaxBranches + kClasses] = {};        // fork, LS done, branch joins, detector joins
};

namespace {

using namespace pusch::tune;

pusch_status bfail(pusch_status st, const char *fmt, int a = 0, int b = 0, int c = 0) {
    char buf[512];
    snprintf(buf, sizeof buf, fmt, a, b, c);
    pusch::set_last_error(buf);
    return st;
}

pusch_status bcuda(cudaError_t e, const char *what) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    pusch::set_last_error(buf);
    return PUSCH_ERR_CUDA;
}

template <typename T>
cudaError_t upload(T **dst, const std::vector<T> &v) {
    if (v.empty()) return cudaSuccess;
    cudaError_t e = cudaMalloc((void **)dst, v.size() * sizeof(T));
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

int class_of(int nl) {
    int c = 0, w = 2;
    while (w < nl) {
        w *= 2;
        ++c;
    }
    return c;
}

// Records the chain on stream s (used under stream capture; also run directly by the autotuner). With
// branches > 1 the cells' FFT/beamforming chains are spread over that many forked streams and the layer
// classes' detectors over the forked streams, joined back into s by events.
pusch_status enqueue(pusch_batch *b, const void *time_in, const void *W, const void *pilots, void *x_hat,
                     uint8_t *bits, uint32_t *status, cudaStream_t s, int only_class = -1) {
    cudaError_t e;
    const int nbr = std::max(1, std::min(b->branches, kMaxBranches));
    auto fail_e = [&](const char *what) { return bcuda(e, what); };
    batch_reset_kernel<<<1, 32, 0, s>>>(b->d_counters, status);
    if ((e = cudaGetLastError()) != cudaSuccess) return fail_e("batch reset launch");
    if (only_class < 0) {
        const size_t tsz = b->cells[0].in_fp16 ? 4 : 8;
        if (nbr > 1) {
            if ((e = cudaEventRecord(b->ev[0], s)) != cudaSuccess) return fail_e("fork record");
            for (int k = 0; k < nbr; ++k)
                if ((e = cudaStreamWaitEvent(b->fork[k], b->ev[0], 0)) != cudaSuccess) return fail_e("fork wait");
        }
        for (size_t c = 0; c < b->cells.size(); ++c) {
            const Geometry &g = b->geo[c];
            cudaStream_t sc = nbr > 1 ? b->fork[c % nbr] : s;
            const void *tin = static_cast<const unsigned char *>(time_in) + (size_t)b->t_off[c] * tsz;
            if ((e = pusch::launch_fft(g, 1, tin, b->freq + b->f_off[c], b->twiddle[g.n_fft], b->kernel_err, sc)) !=
                cudaSuccess)
                return fail_e("batch FFT launch");
            const float2 *w = static_cast<const float2 *>(W) + b->w_off[c];
            e = pusch::launch_beamform(g, 1, b->freq + b->f_off[c], w, b->beam + b->beam_off[c], b->kernel_err, sc,
                                       &b->bf_tune[c]);
            if (e != cudaSuccess) return fail_e("batch beamforming launch");
        }
        if (nbr > 1)
            for (int k = 0; k < nbr; ++k) {
                if ((e = cudaEventRecord(b->ev[2 + k], b->fork[k])) != cudaSuccess) return fail_e("join record");
                if ((e = cudaStreamWaitEvent(s, b->ev[2 + k], 0)) != cudaSuccess) return fail_e("join wait");
            }
        if (b->n_jobs > 0) {
            batch_ls_kernel<<<b->n_jobs, 256, 0, s>>>(b->d_jobs, b->det, b->beam, static_cast<const float2 *>(pilots),
                                                      b->ls);
            if ((e = cudaGetLastError()) != cudaSuccess) return fail_e("batch LS launch");
        }
    }
    float2 *xh = static_cast<float2 *>(x_hat);
    int used = 0;
    const bool fan = nbr > 1 && only_class < 0;
    if (fan && (e = cudaEventRecord(b->ev[1], s)) != cudaSuccess) return fail_e("detector fork record");
    for (int c = 0; c < kClasses; ++c) {
        if (b->n_items[c] == 0 || (only_class >= 0 && c != only_class)) continue;
        cudaStream_t sd = s;
        if (fan) {
            sd = b->fork[used % nbr];
            if ((e = cudaStreamWaitEvent(sd, b->ev[1], 0)) != cudaSuccess) return fail_e("detector fork wait");
        }
        int *ctr = b->d_counters + c;
        const int wps = b->det_warps[c], cps = b->det_ctas[c];
        switch (c) {
            case 0: e = launch_detect<2>(b->det, b->nbmax, b->d_segs, b->d_layers, b->d_items[c], b->n_items[c], ctr, b->beam, b->ls, xh, bits, status, wps, cps, sd); break;
            case 1: e = launch_detect<4>(b->det, b->nbmax, b->d_segs, b->d_layers, b->d_items[c], b->n_items[c], ctr, b->beam, b->ls, xh, bits, status, wps, cps, sd); break;
            case 2: e = launch_detect<8>(b->det, b->nbmax, b->d_segs, b->d_layers, b->d_items[c], b->n_items[c], ctr, b->beam, b->ls, xh, bits, status, wps, cps, sd); break;
            case 3: e = launch_detect<16>(b->det, b->nbmax, b->d_segs, b->d_layers, b->d_items[c], b->n_items[c], ctr, b->beam, b->ls, xh, bits, status, wps, cps, sd); break;
            default: e = launch_detect<32>(b->det, b->nbmax, b->d_segs, b->d_layers, b->d_items[c], b->n_items[c], ctr, b->beam, b->ls, xh, bits, status, wps, cps, sd); break;
        }
        if (e != cudaSuccess) return fail_e("batch detection launch");
        if (fan) {
            if ((e = cudaEventRecord(b->ev[2 + kMaxBranches + c], sd)) != cudaSuccess) return fail_e("detector join record");
            if ((e = cudaStreamWaitEvent(s, b->ev[2 + kMaxBranches + c], 0)) != cudaSuccess) return fail_e("detector join wait");
        }
        ++used;
    }
    // expired waits of the batch's FFT and tensor-core kernels -> PUSCH_STATUS_TIMEOUT
    if ((e = pusch::launch_status_fold(status, b->kernel_err, s)) != cudaSuccess) return fail_e("status fold launch");
    return PUSCH_OK;
}

void drop_graph(pusch_batch *b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    memset(b->key, 0, sizeof b->key);
}

// ---------------------------------------------------------------------------------------- autotuning

std::string bf_key(const Geometry &g) {
    char buf[128];
    snprintf(buf, sizeof buf, "bf form=%d n_rx=%d n_beams=%d n_sc=%d", g.form, g.n_rx, g.n_beams, g.n_sc);
    return buf;
}
std::string det_key(const pusch_batch *b, int c) {
    char buf[128];
    snprintf(buf, sizeof buf, "det form=%d class=%d nbmax=%d n_data=%d", b->geo[0].form, 2 << c, b->nbmax,
             b->det.n_data);
    return buf;
}
std::string graph_key(const pusch_batch *b) {
    char buf[128];
    snprintf(buf, sizeof buf, "graph form=%d n_cells=%d", b->geo[0].form, (int)b->cells.size());
    return buf;
}

}  // namespace

extern "C" {

pusch_status pusch_batch_destroy(pusch_batch *b) {
    if (!b) return PUSCH_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (int k = 0; k < kMaxBranches; ++k)
        if (b->fork[k]) cudaStreamDestroy(b->fork[k]);
    for (auto &ev : b->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto &kv : b->twiddle) cudaFree(kv.second);
    cudaFree(b->freq);
    cudaFree(b->beam);
    cudaFree(b->ls);
    cudaFree(b->d_segs);
    cudaFree(b->d_layers);
    cudaFree(b->d_jobs);
    for (int c = 0; c < kClasses; ++c) cudaFree(b->d_items[c]);
    cudaFree(b->d_counters);
    cudaFree(b->kernel_err);
    cudaFree(b->status_sink);
    delete b;
    return PUSCH_OK;
}

pusch_status pusch_batch_create(pusch_batch **out, const pusch_cell_cfg *cells, int n_cells,
                                const pusch_user_desc *users, int n_users) {
    if (!out) return bfail(PUSCH_ERR_ARG, "batch output pointer is NULL");
    *out = nullptr;
    if (!cells || n_cells < 1 || n_cells > 1024) return bfail(PUSCH_ERR_ARG, "n_cells must be in [1, 1024]");
    if (!users || n_users < 1 || n_users > 65536) return bfail(PUSCH_ERR_ARG, "n_users must be in [1, 65536]");
    for (int c = 0; c < n_cells; ++c) {
        pusch_cell_cfg cc = cells[c];
        cc.n_layers = 1;  // users carry the layers; validate the rest of the cell
        cc.port[0] = 0;
        cc.qam_bits = 2;
        size_t ws;
        pusch_status st = pusch_workspace_size(&cc, 1, &ws);
        if (st != PUSCH_OK) return st;
        if (cells[c].cp != 0 || cells[c].shift_7p5khz != 0)
            return bfail(PUSCH_ERR_UNSUPPORTED, "cell %d: the batch takes time samples without prefixes or shift", c);
        if (cells[c].dmrs_type != 0)
            return bfail(PUSCH_ERR_UNSUPPORTED, "cell %d: the batch uses the comb pilot model (dmrs_type 0)", c);
        if (cells[c].chol_every != 0)
            return bfail(PUSCH_ERR_UNSUPPORTED, "cell %d: the batch detects with one estimate per slot (chol_every 0)", c);
        if (cells[c].noise_var == PUSCH_NOISE_ESTIMATE)
            return bfail(PUSCH_ERR_UNSUPPORTED, "cell %d: the batch takes a given noise variance per cell", c);
        if (cells[c].in_fp16 != cells[0].in_fp16 || cells[c].form != cells[0].form ||
            cells[c].n_sym != cells[0].n_sym || cells[c].dmrs_sym[0] != cells[0].dmrs_sym[0] ||
            cells[c].dmrs_sym[1] != cells[0].dmrs_sym[1])
            return bfail(PUSCH_ERR_ARG, "cell %d: in_fp16, form, n_sym and dmrs_sym must match cell 0", c);
    }
    pusch_batch *b = new (std::nothrow) pusch_batch();
    if (!b) return bfail(PUSCH_ERR_ARG, "out of host memory");
    b->cells.assign(cells, cells + n_cells);
    b->users.assign(users, users + n_users);
    const pusch_cell_cfg &c0 = cells[0];
    for (int c = 0; c < n_cells; ++c) {
        pusch_cell_cfg cc = cells[c];
        cc.n_layers = 1;
        cc.port[0] = 0;
        cc.qam_bits = 2;
        b->geo.push_back(pusch::make_geometry(cc));
        b->nbmax = std::max(b->nbmax, cc.n_beams);
    }
    const Geometry &g0 = b->geo[0];
    b->det.n_sym = g0.n_sym;
    b->det.n_data = g0.n_data;
    b->det.dmrs0 = g0.dmrs0;
    b->det.dmrs1 = g0.dmrs1;
    b->det.dmrs_lo = g0.dmrs0 < g0.dmrs1 ? g0.dmrs0 : g0.dmrs1;
    b->det.dmrs_hi = g0.dmrs0 < g0.dmrs1 ? g0.dmrs1 : g0.dmrs0;
    const int nd = g0.n_data;

    // ---- per-cell offsets
    long long t = 0, w = 0, bm = 0;
    size_t f = 0;
    for (int c = 0; c < n_cells; ++c) {
        const Geometry &g = b->geo[c];
        b->t_off.push_back(t);
        b->w_off.push_back(w);
        b->beam_off.push_back(bm);
        b->f_off.push_back(f);
        t += pusch::time_elems_per_slot(g);
        w += (long long)g.n_rx * g.n_beams;
        bm += (long long)g.n_sym * g.n_sc * g.n_beams;
        f += up256(pusch::freq_bytes_of(g, 1));
    }
    b->sizes[0] = (size_t)t;
    b->sizes[1] = (size_t)w;

    // ---- users: validation, pilots, LS jobs, output offsets
    std::vector<LsJob> jobs;
    std::vector<long long> pil_off(n_users), out_off(n_users);
    std::vector<std::vector<long long>> ls_off(n_users);
    std::vector<std::vector<int>> first(n_users), last(n_users);
    long long p = 0, o = 0, lsz = 0;
    for (int u = 0; u < n_users; ++u) {
        const pusch_user_desc &U = users[u];
        if (U.cell < 0 || U.cell >= n_cells) {
            pusch_batch_destroy(b);
            return bfail(PUSCH_ERR_ARG, "user %d: cell %d out of range", u, U.cell);
        }
        const Geometry &g = b->geo[U.cell];
        if (U.sc_count < 1 || U.sc_start < 0 || U.sc_start + U.sc_count > g.n_sc || U.n_layers < 1 ||
            U.n_layers > 32 || U.port0 < 0 || U.port0 + U.n_layers > g.comb || (U.qam_bits != 2 && U.qam_bits != 4)) {
            pusch_batch_destroy(b);
            return bfail(PUSCH_ERR_ARG, "user %d: range, layers, ports or qam_bits invalid for cell %d", u, U.cell);
        }
        pil_off[u] = p;
        out_off[u] = o;
        p += (long long)U.n_layers * 2 * U.sc_count;
        o += (long long)U.n_layers * nd * U.sc_count;
        for (int l = 0; l < U.n_layers; ++l) {
            const int port = U.port0 + l;
            const int fst = U.sc_start + ((port - U.sc_start) % g.comb + g.comb) % g.comb;
            if (fst >= U.sc_start + U.sc_count) {
                pusch_batch_destroy(b);
                return bfail(PUSCH_ERR_ARG, "user %d layer %d: no pilot of its port inside its range", u, l);
            }
            const int lst = fst + ((U.sc_start + U.sc_count - 1 - fst) / g.comb) * g.comb;
            first[u].push_back(fst);
            last[u].push_back(lst);
            ls_off[u].push_back(lsz);
            LsJob j;
            memset(&j, 0, sizeof j);
            j.beam_off = b->beam_off[U.cell];
            j.pil_off = pil_off[u] + (long long)l * 2 * U.sc_count;
            j.ls_off = lsz;
            j.n_sc = g.n_sc;
            j.nb = g.n_beams;
            j.first = fst;
            j.npil = (lst - fst) / g.comb + 1;
            j.comb = g.comb;
            j.a0 = U.sc_start;
            j.n = U.sc_count;
            jobs.push_back(j);
            lsz += (long long)j.npil * g.n_beams;
        }
    }
    b->sizes[2] = (size_t)p;
    b->sizes[3] = b->sizes[4] = (size_t)o;
    b->n_jobs = (int)jobs.size();

    // ---- segments and work items
    std::vector<Segment> segs;
    std::vector<SegLayer> layers;
    std::vector<int2> items[kClasses];
    for (int c = 0; c < n_cells; ++c) {
        const Geometry &g = b->geo[c];
        std::vector<int> pts;
        for (int u = 0; u < n_users; ++u)
            if (users[u].cell == c) {
                pts.push_back(users[u].sc_start);
                pts.push_back(users[u].sc_start + users[u].sc_count);
            }
        std::sort(pts.begin(), pts.end());
        pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
        for (size_t k = 0; k + 1 < pts.size(); ++k) {
            const int a0 = pts[k], a1 = pts[k + 1];
            Segment sg;
            memset(&sg, 0, sizeof sg);
            sg.beam_off = b->beam_off[c];
            sg.cell = c;
            sg.a0 = a0;
            sg.n = a1 - a0;
            sg.layer0 = (int)layers.size();
            sg.nb = g.n_beams;
            sg.n_sc = g.n_sc;
            sg.comb = g.comb;
            sg.load = g.noise_var + g.loading;
            for (int u = 0; u < n_users; ++u) {
                const pusch_user_desc &U = users[u];
                if (U.cell != c || U.sc_start > a0 || U.sc_start + U.sc_count <= a0) continue;
                for (int l = 0; l < U.n_layers; ++l) {
                    SegLayer L;
                    memset(&L, 0, sizeof L);
                    L.ls_off = ls_off[u][l];
                    L.out_off = out_off[u] + (long long)l * nd * U.sc_count;
                    L.first = first[u][l];
                    L.last = last[u][l];
                    L.a0 = U.sc_start;
                    L.n = U.sc_count;
                    L.qam = U.qam_bits;
                    layers.push_back(L);
                }
            }
            sg.nl = (int)layers.size() - sg.layer0;
            if (sg.nl == 0) continue;
            if (sg.nl > 32 || sg.nl > g.n_beams) {
                pusch_batch_destroy(b);
                return bfail(PUSCH_ERR_ARG, "cell %d: %d layers overlap at subcarrier %d (more than min(32, n_beams))",
                             c, sg.nl, a0);
            }
            const int cls = class_of(sg.nl);
            const int spw = 32 / (2 << cls);
            const int si = (int)segs.size();
            for (int a = a0; a < a1; a += spw) items[cls].push_back(make_int2(si, a));
            segs.push_back(sg);
        }
    }

    // ---- device memory
    cudaError_t e = cudaSuccess;
    size_t beam_total = (size_t)bm * sizeof(float2);
    if ((e = cudaMalloc((void **)&b->freq, f)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&b->beam, beam_total)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&b->ls, (size_t)std::max<long long>(lsz, 1) * sizeof(float2))) != cudaSuccess)
        goto cuda_error;
    if ((e = upload(&b->d_segs, segs)) != cudaSuccess) goto cuda_error;
    if ((e = upload(&b->d_layers, layers)) != cudaSuccess) goto cuda_error;
    if ((e = upload(&b->d_jobs, jobs)) != cudaSuccess) goto cuda_error;
    for (int c = 0; c < kClasses; ++c) {
        b->n_items[c] = (int)items[c].size();
        if ((e = upload(&b->d_items[c], items[c])) != cudaSuccess) goto cuda_error;
    }
    if ((e = cudaMalloc((void **)&b->d_counters, kClasses * sizeof(int))) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&b->kernel_err, 16)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMemset(b->kernel_err, 0, 16)) != cudaSuccess) goto cuda_error;
    if ((e = cudaMalloc((void **)&b->status_sink, 16)) != cudaSuccess) goto cuda_error;
    for (int c = 0; c < n_cells; ++c) {
        const int N = b->geo[c].n_fft;
        if (b->twiddle.count(N)) continue;
        const std::vector<float2> tw = pusch::fft_twiddle_table(N);
        float2 *d = nullptr;
        if ((e = upload(&d, tw)) != cudaSuccess) goto cuda_error;
        b->twiddle[N] = d;
    }
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) goto cuda_error;
    for (int k = 0; k < kMaxBranches; ++k)
        if ((e = cudaStreamCreateWithFlags(&b->fork[k], cudaStreamNonBlocking)) != cudaSuccess) goto cuda_error;
    for (auto &ev : b->ev)
        if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) goto cuda_error;
    b->bf_tune.assign(n_cells, pusch::TcTune{});
    b->branches = std::min(4, n_cells);
    (void)c0;
    *out = b;
    pusch::set_last_error("");
    return PUSCH_OK;
cuda_error:
    pusch_batch_destroy(b);
    return bcuda(e, "pusch_batch_create allocation");
}

pusch_status pusch_batch_sizes(const pusch_batch *b, size_t sizes[5]) {
    if (!b || !sizes) return bfail(PUSCH_ERR_ARG, "NULL argument");
    for (int k = 0; k < 5; ++k) sizes[k] = b->sizes[k];
    return PUSCH_OK;
}

pusch_status pusch_batch_run(pusch_batch *b, const void *time_in, const void *W, const void *pilots, void *x_hat,
                             uint8_t *bits, uint32_t *status, void *stream) {
    if (!b) return bfail(PUSCH_ERR_ARG, "batch is NULL");
    if (!time_in || !W || !pilots || !x_hat || !bits) return bfail(PUSCH_ERR_ARG, "pusch_batch_run: NULL buffer");
    uint32_t *stat = status ? status : b->status_sink;
    const void *key[6] = {time_in, W, pilots, x_hat, bits, stat};
    cudaError_t e;
    if (!b->exec || memcmp(key, b->key, sizeof key) != 0) {
        drop_graph(b);
        if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess)
            return bcuda(e, "graph capture begin");
        pusch_status st = enqueue(b, time_in, W, pilots, x_hat, bits, stat, b->cap);
        cudaGraph_t gph = nullptr;
        e = cudaStreamEndCapture(b->cap, &gph);
        if (st != PUSCH_OK) {
            if (gph) cudaGraphDestroy(gph);
            return st;
        }
        if (e != cudaSuccess) return bcuda(e, "graph capture end");
        b->graph = gph;
        if ((e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) return bcuda(e, "graph instantiate");
        memcpy(b->key, key, sizeof key);
    }
    if ((e = cudaGraphLaunch(b->exec, (cudaStream_t)stream)) != cudaSuccess) return bcuda(e, "graph launch");
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_batch_autotune(pusch_batch *b, const void *time_in, const void *W, const void *pilots,
                                  void *x_hat, uint8_t *bits, uint32_t *status, const char *cache_path, void *stream,
                                  int *n_timed) {
    if (!b) return bfail(PUSCH_ERR_ARG, "batch is NULL");
    if (!time_in || !W || !pilots || !x_hat || !bits) return bfail(PUSCH_ERR_ARG, "pusch_batch_autotune: NULL buffer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t *stat = status ? status : b->status_sink;
    std::map<std::string, std::string> cache = read_cache(cache_path);
    std::vector<std::string> lines;
    int timed = 0;
    cudaError_t e = cudaSuccess;
    const int reps = 10;
    char buf[256];
    drop_graph(b);
    // one uncaptured pass: FFT output, beams and the LS table the candidates below read
    pusch_status st = enqueue(b, time_in, W, pilots, x_hat, bits, stat, s);
    if (st != PUSCH_OK) return st;
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return bcuda(e, "autotune first pass");

    // 1. tensor-core GEMM shape per distinct cell shape
    std::map<std::string, pusch::TcTune> bf_choice;
    for (size_t c = 0; c < b->cells.size(); ++c) {
        const Geometry &g = b->geo[c];
        if (g.form == PUSCH_FORM_FP32) continue;
        const std::string k = bf_key(g);
        if (!bf_choice.count(k)) {
            pusch::TcTune best;
            auto it = cache.find(k);
            if (it != cache.end()) {
                best.chunk_rows = value_of(it->second, "chunk", 0);
                best.staged = value_of(it->second, "staged", 0);
            } else {
                pusch::TcTune cand[8];
                const int n = pusch::bf_tc_candidates(g, cand, 8);
                float best_ms = 1e30f;
                const float2 *w = static_cast<const float2 *>(W) + b->w_off[c];
                for (int i = 0; i < n; ++i) {
                    const float ms = time_ms(s, reps, [&] {
                        pusch::launch_beamform(g, 1, b->freq + b->f_off[c], w, b->beam + b->beam_off[c],
                                               b->kernel_err, s, &cand[i]);
                    }, &e);
                    if (e != cudaSuccess) return bcuda(e, "autotune beamforming");
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = cand[i];
                    }
                }
                ++timed;
                snprintf(buf, sizeof buf, "%s | chunk=%d staged=%d ms=%.5f", k.c_str(), best.chunk_rows, best.staged,
                         best_ms);
                lines.push_back(buf);
            }
            bf_choice[k] = best;
        }
        b->bf_tune[c] = bf_choice[k];
    }

    // 2. detector shape per layer class (the LS table from the first pass stays valid)
    const int warps_c[3] = {1, 2, 4}, ctas_c[3] = {0, 1, 2};
    for (int c = 0; c < kClasses; ++c) {
        if (b->n_items[c] == 0) continue;
        const std::string k = det_key(b, c);
        auto it = cache.find(k);
        if (it != cache.end()) {
            b->det_warps[c] = value_of(it->second, "warps", 2);
            b->det_ctas[c] = value_of(it->second, "ctas", 0);
            continue;
        }
        float best_ms = 1e30f;
        int bw = 2, bc = 0;
        for (int wi = 0; wi < 3; ++wi)
            for (int ci = 0; ci < 3; ++ci) {
                b->det_warps[c] = warps_c[wi];
                b->det_ctas[c] = ctas_c[ci];
                const float ms = time_ms(s, reps, [&] { enqueue(b, time_in, W, pilots, x_hat, bits, stat, s, c); }, &e);
                if (e != cudaSuccess) return bcuda(e, "autotune detection");
                if (ms < best_ms) {
                    best_ms = ms;
                    bw = warps_c[wi];
                    bc = ctas_c[ci];
                }
            }
        b->det_warps[c] = bw;
        b->det_ctas[c] = bc;
        ++timed;
        snprintf(buf, sizeof buf, "%s | warps=%d ctas=%d ms=%.5f", k.c_str(), bw, bc, best_ms);
        lines.push_back(buf);
    }

    // 3. graph branches, timed as whole captured graphs
    {
        const std::string k = graph_key(b);
        auto it = cache.find(k);
        if (it != cache.end()) {
            b->branches = std::max(1, std::min(kMaxBranches, value_of(it->second, "branches", 4)));
        } else {
            float best_ms = 1e30f;
            int best_k = 1;
            for (int nbr = 1; nbr <= kMaxBranches && nbr <= (int)b->cells.size(); nbr *= 2) {
                b->branches = nbr;
                drop_graph(b);
                st = pusch_batch_run(b, time_in, W, pilots, x_hat, bits, status, stream);
                if (st != PUSCH_OK) return st;
                const float ms = time_ms(s, reps, [&] { cudaGraphLaunch(b->exec, s); }, &e);
                if (e != cudaSuccess) return bcuda(e, "autotune graph");
                if (ms < best_ms) {
                    best_ms = ms;
                    best_k = nbr;
                }
            }
            b->branches = best_k;
            ++timed;
            snprintf(buf, sizeof buf, "%s | branches=%d ms=%.5f", k.c_str(), best_k, best_ms);
            lines.push_back(buf);
        }
    }
    drop_graph(b);
    if (cache_path && !lines.empty()) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return bfail(PUSCH_ERR_ARG, "cannot append to the autotune cache file");
        for (const auto &l : lines) fprintf(f, "%s\n", l.c_str());
        fclose(f);
    }
    if (n_timed) *n_timed = timed;
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_batch_tuning(const pusch_batch *b, int *out, int n_out) {
    if (!b || !out || n_out < 1 + 2 * kClasses) return bfail(PUSCH_ERR_ARG, "pusch_batch_tuning: bad arguments");
    out[0] = b->branches;
    for (int c = 0; c < kClasses; ++c) {
        out[1 + 2 * c] = b->det_warps[c];
        out[2 + 2 * c] = b->det_ctas[c];
    }
    int k = 1 + 2 * kClasses;
    for (size_t c = 0; c < b->cells.size() && k + 1 < n_out; ++c, k += 2) {
        out[k] = b->bf_tune[c].chunk_rows;
        out[k + 1] = b->bf_tune[c].staged;
    }
    return PUSCH_OK;
}

}  // extern "C"
