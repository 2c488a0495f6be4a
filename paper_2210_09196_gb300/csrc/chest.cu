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

}  // namespace

int ls_pilots_per_layer(const Geometry &g) { return (g.n_sc + g.comb - 1) / g.comb; }

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
