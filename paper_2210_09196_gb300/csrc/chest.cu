// LS channel estimation on the DMRS symbols (Section II: block-type pilots filling whole OFDM symbols;
// the estimate is an element-wise division of the received pilot REs by the known pilots, Table I "CHE"),
// followed by linear interpolation between each layer's comb of pilot subcarriers.
//
// One thread per output element (slot, subcarrier a, layer l, beam b), beam fastest, so that the
// [n_sc][n_layers][n_beams] estimate the detector reads is written with fully coalesced stores. The two
// pilot REs a thread needs are re-derived per thread (they are read from L1/L2; the DMRS rows are a
// small fraction of the slot).
#include "chest_common.cuh"

namespace pusch {
namespace {

struct ChestArgs {
    int n_sc, n_beams, n_layers, comb, n_sym, dmrs0, dmrs1;
    int port[32];
};

__global__ void __launch_bounds__(256)
chest_ls_kernel(ChestArgs g, long long total, const float2 *__restrict__ beam, const float2 *__restrict__ pilots,
                float2 *__restrict__ H) {
    const long long per_sc = (long long)g.n_layers * g.n_beams;
    const long long per_slot = per_sc * g.n_sc;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long slot = idx / per_slot;
        long long rem = idx - slot * per_slot;
        const int a = (int)(rem / per_sc);
        rem -= (long long)a * per_sc;
        const int l = (int)(rem / g.n_beams);
        const int b = (int)(rem - (long long)l * g.n_beams);

        int lo, hi;
        pilot_bracket(a, g.port[l], g.comb, g.n_sc, lo, hi);
        const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
        const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
        const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
        const float2 *p1 = p0 + g.n_sc;
        const float2 h_lo = ls_value(__ldg(&y0[(long long)lo * g.n_beams + b]), __ldg(&y1[(long long)lo * g.n_beams + b]),
                                     pilot_inverse(__ldg(&p0[lo])), pilot_inverse(__ldg(&p1[lo])));
        float2 h = h_lo;
        if (hi != lo) {
            const float2 h_hi =
                ls_value(__ldg(&y0[(long long)hi * g.n_beams + b]), __ldg(&y1[(long long)hi * g.n_beams + b]),
                         pilot_inverse(__ldg(&p0[hi])), pilot_inverse(__ldg(&p1[hi])));
            h = interp(h_lo, h_hi, interp_weight(a, lo, hi));
        }
        H[idx] = h;
    }
}

// LS estimate at every pilot subcarrier of every layer (the element-wise division alone):
// ls[slot][l][k][b] for the layer's k-th pilot q = port[l] + k * comb (k < kmax; zero past n_sc).
__global__ void __launch_bounds__(256)
ls_pilots_kernel(ChestArgs g, int kmax, long long total, const float2 *__restrict__ beam,
                 const float2 *__restrict__ pilots, float2 *__restrict__ ls) {
    const long long per_l = (long long)kmax * g.n_beams;
    const long long per_slot = per_l * g.n_layers;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        const long long slot = idx / per_slot;
        long long rem = idx - slot * per_slot;
        const int l = (int)(rem / per_l);
        rem -= (long long)l * per_l;
        const int k = (int)(rem / g.n_beams);
        const int b = (int)(rem - (long long)k * g.n_beams);
        const int q = g.port[l] + k * g.comb;
        float2 v = make_float2(0.f, 0.f);
        if (q < g.n_sc) {
            const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
            const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
            const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
            v = ls_value(__ldg(&y0[(long long)q * g.n_beams + b]), __ldg(&y1[(long long)q * g.n_beams + b]),
                         pilot_inverse(__ldg(&p0[q])), pilot_inverse(__ldg(&p0[g.n_sc + q])));
        }
        ls[idx] = v;
    }
}

// Noise-variance estimate (Section II "NE"), pass 1: CTA (part, slot) sums the squared pilot residuals
// |y_j[q][b] - LS[q][b] p_j[q]|^2 (both DMRS symbols; LS the two-symbol mean at the pilot, i.e. the estimate at
// its own pilot) over its share of the slot's (layer, pilot, beam) elements. partial[slot][part] = {sum, count}.
// Fixed grid and reduction order: the result does not depend on scheduling.
__global__ void __launch_bounds__(256)
ne_partial_kernel(ChestArgs g, int kmax, const float2 *__restrict__ beam, const float2 *__restrict__ pilots,
                  float2 *__restrict__ partial) {
    __shared__ float2 red[8];
    const long long slot = blockIdx.y;
    const long long per_slot = (long long)g.n_layers * kmax * g.n_beams;
    const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
    const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
    float sum = 0.f, cnt = 0.f;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < per_slot;
         idx += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(idx / ((long long)kmax * g.n_beams));
        const long long rem = idx - (long long)l * kmax * g.n_beams;
        const int k = (int)(rem / g.n_beams), b = (int)(rem - (long long)k * g.n_beams);
        const int q = g.port[l] + k * g.comb;
        if (q >= g.n_sc) continue;
        const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
        const float2 pv0 = __ldg(&p0[q]), pv1 = __ldg(&p0[g.n_sc + q]);
        const float2 v0 = __ldg(&y0[(long long)q * g.n_beams + b]), v1 = __ldg(&y1[(long long)q * g.n_beams + b]);
        const float2 ls = ls_value(v0, v1, pilot_inverse(pv0), pilot_inverse(pv1));
        const float2 e0 = csub(v0, cmul(ls, pv0)), e1 = csub(v1, cmul(ls, pv1));
        sum += e0.x * e0.x + e0.y * e0.y + e1.x * e1.x + e1.y * e1.y;
        cnt += 2.f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(sum, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = cadd(t, red[w]);
        partial[slot * gridDim.x + blockIdx.x] = t;
    }
}

// Pass 2: one warp per slot adds the parts in a fixed order; sigma2[slot] = 2 * sum / count (the factor 2
// undoes the two-symbol mean: E|y_j - LS p_j|^2 = sigma^2 / 2 for unit-modulus pilots).
__global__ void ne_final_kernel(int n_parts, const float2 *__restrict__ partial, float *__restrict__ sigma2) {
    const int slot = blockIdx.x, lane = threadIdx.x;
    float2 t = make_float2(0.f, 0.f);
    for (int p = lane; p < n_parts; p += 32) t = cadd(t, partial[(long long)slot * n_parts + p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(0xFFFFFFFFu, t.x, o);
        t.y += __shfl_xor_sync(0xFFFFFFFFu, t.y, o);
    }
    if (lane == 0) sigma2[slot] = t.y > 0.f ? 2.f * t.x / t.y : 0.f;
}

}  // namespace

int ls_pilots_per_layer(const Geometry &g) { return (g.n_sc + g.comb - 1) / g.comb; }

cudaError_t launch_noise_est(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots,
                             float2 *partial, float *sigma2, cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    if (n_slots > 65535) return cudaErrorInvalidValue;
    ChestArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.comb = g.comb;
    a.n_sym = g.n_sym;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    ne_partial_kernel<<<dim3(kNoiseParts, (unsigned)n_slots), 256, 0, st>>>(a, ls_pilots_per_layer(g), beam, pilots,
                                                                             partial);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ne_final_kernel<<<(unsigned)n_slots, 32, 0, st>>>(kNoiseParts, partial, sigma2);
    return cudaGetLastError();
}

cudaError_t launch_ls_pilots(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *ls,
                             cudaStream_t st) {
    ChestArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.comb = g.comb;
    a.n_sym = g.n_sym;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    const int kmax = ls_pilots_per_layer(g);
    const long long total = (long long)n_slots * g.n_layers * kmax * g.n_beams;
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 32) blocks = 152LL * 32;
    ls_pilots_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, kmax, total, beam, pilots, ls);
    return cudaGetLastError();
}

cudaError_t launch_chest_ls(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *H,
                            cudaStream_t st) {
    ChestArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.comb = g.comb;
    a.n_sym = g.n_sym;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    const long long total = (long long)n_slots * g.n_sc * g.n_layers * g.n_beams;
    if (total == 0) return cudaSuccess;
    long long blocks = (total + 255) / 256;
    if (blocks > 152LL * 64) blocks = 152LL * 64;
    chest_ls_kernel<<<(unsigned)blocks, 256, 0, st>>>(a, total, beam, pilots, H);
    return cudaGetLastError();
}

}  // namespace pusch
