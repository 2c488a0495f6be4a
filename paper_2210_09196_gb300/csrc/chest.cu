// LS channel estimation on the DMRS symbols (Section II: block-type pilots filling whole OFDM symbols;
// the estimate is an element-wise division of the received pilot REs by the known pilots, Table I "CHE"),
// followed by linear interpolation between each layer's comb of pilot subcarriers.
//
// One thread per output element (slot, subcarrier a, layer l, beam b), beam fastest, so that the
// [n_sc][n_layers][n_beams] estimate the detector reads is written with fully coalesced stores. The two
// pilot REs a thread needs are re-derived per thread (they are read from L1/L2; the DMRS rows are a
// small fraction of the slot).
#include "internal.cuh"

namespace pusch {
namespace {

struct ChestArgs {
    int n_sc, n_beams, n_layers, comb, n_sym, dmrs0, dmrs1;
    int port[32];
};

// 1/2 sum_j Y_j / P_j, the division done as y * conj(p) / |p|^2.
__device__ __forceinline__ float2 ls_at(const float2 *__restrict__ y0, const float2 *__restrict__ y1,
                                        const float2 *__restrict__ p0, const float2 *__restrict__ p1, int q, int nb,
                                        int b) {
    const float2 ya = __ldg(&y0[(long long)q * nb + b]);
    const float2 yb = __ldg(&y1[(long long)q * nb + b]);
    const float2 pa = __ldg(&p0[q]);
    const float2 pb = __ldg(&p1[q]);
    const float2 da = cscale(cmulc(pa, ya), 1.f / (pa.x * pa.x + pa.y * pa.y));
    const float2 db = cscale(cmulc(pb, yb), 1.f / (pb.x * pb.x + pb.y * pb.y));
    return cscale(cadd(da, db), 0.5f);
}

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

        const int port = g.port[l];
        const int first = port;
        const int last = port + ((g.n_sc - 1 - port) / g.comb) * g.comb;
        int lo, hi;
        if (a <= first) {
            lo = hi = first;
        } else if (a >= last) {
            lo = hi = last;
        } else {
            lo = port + ((a - port) / g.comb) * g.comb;
            hi = (lo == a) ? lo : lo + g.comb;
        }
        const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
        const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
        const float2 *p0 = pilots + (slot * g.n_layers + l) * 2LL * g.n_sc;
        const float2 *p1 = p0 + g.n_sc;
        float2 h = ls_at(y0, y1, p0, p1, lo, g.n_beams, b);
        if (hi != lo) {
            const float2 h1 = ls_at(y0, y1, p0, p1, hi, g.n_beams, b);
            const float w = (float)(a - lo) / (float)(hi - lo);
            h = make_float2(fmaf(w, h1.x - h.x, h.x), fmaf(w, h1.y - h.y, h.y));
        }
        H[idx] = h;
    }
}

}  // namespace

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
