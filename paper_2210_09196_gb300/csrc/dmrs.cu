// 3GPP type-1 DMRS values (TS 38.211 5.2.1 pseudo-random sequence, 6.4.1.1 mapping): the pilots input of the
// chain for cells with dmrs_type = 1. An extension beyond the paper, whose pilots are a block-type model.
//
// One CTA per (slot, DMRS symbol): one thread steps the two length-31 LFSRs of the Gold sequence (1600 steps of
// offset, then n_sc + 2 output bits into shared memory; a few thousand dependent steps, far below the chain's
// cost), then the CTA maps r(m) with the layers' CDM groups and OCC signs onto the subcarriers.
#include <stdio.h>
#include <string.h>

#include "internal.cuh"

namespace {

constexpr int kSlotsPerLaunch = 64;

struct DmrsArgs {
    int n_sc, n_layers;
    int port[4];
    uint32_t c_init[kSlotsPerLaunch][2];  // per (slot of this launch, DMRS symbol)
};

// LFSR state s holds x(n) .. x(n + 30) in bits 0 .. 30; one step appends x(n + 31) from the taps.
__device__ __forceinline__ uint32_t step_x1(uint32_t s) { return (s >> 1) | ((((s >> 3) ^ s) & 1u) << 30); }
__device__ __forceinline__ uint32_t step_x2(uint32_t s) {
    return (s >> 1) | ((((s >> 3) ^ (s >> 2) ^ (s >> 1) ^ s) & 1u) << 30);
}

__global__ void __launch_bounds__(256) dmrs_type1_kernel(DmrsArgs a, float2 *__restrict__ pilots) {
    __shared__ uint8_t c[4096 + 8];
    const int si = blockIdx.x, j = blockIdx.y;  // slot of this launch, DMRS symbol
    const int len = a.n_sc + 2;
    if (threadIdx.x == 0) {
        uint32_t x1 = 1u, x2 = a.c_init[si][j] & 0x7FFFFFFFu;
        for (int n = 0; n < 1600; ++n) {
            x1 = step_x1(x1);
            x2 = step_x2(x2);
        }
        for (int n = 0; n < len; ++n) {
            c[n] = (uint8_t)((x1 ^ x2) & 1u);
            x1 = step_x1(x1);
            x2 = step_x2(x2);
        }
    }
    __syncthreads();
    const float r = 0.70710678118654752440f;  // 1 / sqrt(2)
    float2 *out = pilots + (long long)si * a.n_layers * 2 * a.n_sc;
    for (int idx = threadIdx.x; idx < a.n_layers * a.n_sc; idx += blockDim.x) {
        const int l = idx / a.n_sc, k = idx - l * a.n_sc;
        const int p = a.port[l], delta = p >> 1;
        float2 v = make_float2(0.f, 0.f);
        if ((k & 1) == delta) {
            const int m = (k - delta) >> 1;  // k = 4n + 2k' + delta, m = 2n + k'
            const float w = ((p & 1) && (m & 1)) ? -1.f : 1.f;
            v = make_float2(w * r * (1.f - 2.f * (float)c[2 * m]), w * r * (1.f - 2.f * (float)c[2 * m + 1]));
        }
        out[((long long)l * 2 + j) * a.n_sc + k] = v;
    }
}

}  // namespace

extern "C" pusch_status pusch_dmrs_type1_pilots(const pusch_cell_cfg *cfg, int n_slots, const int *slot_numbers,
                                                int n_id, int n_scid, void *pilots, void *stream) {
    size_t ws = 0;
    pusch_status st = pusch_workspace_size(cfg, 1, &ws);  // validates cfg (and sets the error text)
    if (st != PUSCH_OK) return st;
    char buf[160];
    if (cfg->dmrs_type != 1) {
        snprintf(buf, sizeof buf, "pusch_dmrs_type1_pilots: cfg.dmrs_type is %d, not 1", cfg->dmrs_type);
        pusch::set_last_error(buf);
        return PUSCH_ERR_ARG;
    }
    if (n_slots < 0 || (n_slots > 0 && (!slot_numbers || !pilots)) || n_id < 0 || n_id > 65535 ||
        (n_scid != 0 && n_scid != 1)) {
        pusch::set_last_error("pusch_dmrs_type1_pilots: arguments out of range");
        return PUSCH_ERR_ARG;
    }
    for (int i = 0; i < n_slots; ++i)
        if (slot_numbers[i] < 0 || slot_numbers[i] > 159) {
            pusch::set_last_error("pusch_dmrs_type1_pilots: slot numbers must be in [0, 159]");
            return PUSCH_ERR_ARG;
        }
    DmrsArgs a;
    memset(&a, 0, sizeof a);
    a.n_sc = cfg->n_sc;
    a.n_layers = cfg->n_layers;
    for (int l = 0; l < cfg->n_layers; ++l) a.port[l] = cfg->port[l];
    cudaStream_t s = (cudaStream_t)stream;
    for (int i0 = 0; i0 < n_slots; i0 += kSlotsPerLaunch) {
        const int n = n_slots - i0 < kSlotsPerLaunch ? n_slots - i0 : kSlotsPerLaunch;
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < 2; ++j) {
                const unsigned long long v = (1ull << 17) * (14ull * (unsigned)slot_numbers[i0 + i] +
                                                             (unsigned)cfg->dmrs_sym[j] + 1ull) *
                                                 (2ull * (unsigned)n_id + 1ull) +
                                             2ull * (unsigned)n_id + (unsigned)n_scid;
                a.c_init[i][j] = (uint32_t)(v % (1ull << 31));
            }
        float2 *out = static_cast<float2 *>(pilots) + (long long)i0 * cfg->n_layers * 2 * cfg->n_sc;
        dmrs_type1_kernel<<<dim3((unsigned)n, 2), 256, 0, s>>>(a, out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            snprintf(buf, sizeof buf, "pusch_dmrs_type1_pilots: %s", cudaGetErrorString(e));
            pusch::set_last_error(buf);
            return PUSCH_ERR_CUDA;
        }
    }
    pusch::set_last_error("");
    return PUSCH_OK;
}
