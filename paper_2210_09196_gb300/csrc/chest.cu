// LS channel estimation on the DMRS symbols (Section II: block-type pilots filling whole OFDM symbols;
// the estimate is an element-wise division of the received pilot REs by the known pilots, Table I "CHE"),
// followed by linear interpolation between each layer's comb of pilot subcarriers; and the noise-variance
// estimate from the pilot residuals (Section II "NE").
//
// Two passes: the LS values at every layer's pilot subcarriers (a small table, L2-resident; with type-1 DMRS
// the OCC-despread CDM pairs at their centres), then the full estimate: a CTA per (16-subcarrier run, slot)
// derives each (subcarrier, layer)'s two neighbouring pilots and weight once into shared memory, and each
// thread writes 16-byte units (two beams) of every subcarrier of the run, so that the [n_sc][n_layers][n_beams]
// estimate the detector reads is written with fully coalesced stores. For an estimate that varies in time the
// table pass runs per DMRS symbol and the second pass writes one estimate per detection group (interpolated
// in time to the group's mean symbol time).
#include <algorithm>

#include "chest_common.cuh"

namespace pusch {
namespace {

struct ChestArgs {
    int n_sc, n_beams, n_layers, comb, n_sym, dmrs0, dmrs1;
    int dmrs_type;                 // 1: type-1 DMRS, the table entries are OCC-despread CDM pairs
    int n_groups;                  // estimates interpolated in time: one per detection group
    float group_t[16];
    int port[32];
};

ChestArgs chest_args(const Geometry &g) {
    ChestArgs a;
    a.n_sc = g.n_sc;
    a.n_beams = g.n_beams;
    a.n_layers = g.n_layers;
    a.comb = g.comb;
    a.n_sym = g.n_sym;
    a.dmrs0 = g.dmrs0;
    a.dmrs1 = g.dmrs1;
    a.dmrs_type = g.dmrs_type;
    a.n_groups = g.n_groups;
    for (int q = 0; q < 16; ++q) a.group_t[q] = g.group_t[q];
    for (int l = 0; l < 32; ++l) a.port[l] = g.port[l];
    return a;
}

// The estimate H[slot][a][l][b] from the LS pilot table: linear interpolation between the layer's neighbouring
// pilot subcarriers, held outside the first/last. CTA (subcarrier run, slot) covers kRun consecutive
// subcarriers; thread t owns (layer l, beam unit u) = (t / units, t % units) for the whole run, so the pilot
// bracket is found once (one division) and then advanced, and consecutive threads write consecutive 16-byte
// (or 8-byte) units of a subcarrier's [n_layers][n_beams] block. T = float4 (beam pairs) or float2.
constexpr int kRun = 16;

__device__ __forceinline__ float4 lerp_unit(float4 lo, float4 hi, float w) {
    const float2 h0 = interp(make_float2(lo.x, lo.y), make_float2(hi.x, hi.y), w);
    const float2 h1 = interp(make_float2(lo.z, lo.w), make_float2(hi.z, hi.w), w);
    return make_float4(h0.x, h0.y, h1.x, h1.y);
}
__device__ __forceinline__ float2 lerp_unit(float2 lo, float2 hi, float w) { return interp(lo, hi, w); }

// TV (time-varying mode): tab holds the two DMRS symbols' tables back to back (second at tab_stride units);
// each unit's two frequency-interpolated values f0, f1 give the estimate of group q at its mean time,
// f0 + t_q (f1 - f0), written to H + q * h_stride.
template <typename T, bool TV>
__global__ void __launch_bounds__(1024)
chest_interp_kernel(ChestArgs g, int kmax, int units, int layers_per_cta, const T *__restrict__ ls,
                    long long tab_stride, T *__restrict__ H, long long h_stride) {
    __shared__ int s_klo[kRun][32], s_khi[kRun][32];
    __shared__ float s_w[kRun][32];
    const int t = threadIdx.x;
    const int l_base = blockIdx.z * layers_per_cta;
    const int n_l = min(layers_per_cta, g.n_layers - l_base);
    const long long slot = blockIdx.y;
    const int a0 = blockIdx.x * kRun;
    // 1. the run's (subcarrier, layer) brackets: table indices of the neighbouring pilots and the weight
    for (int e = t; e < kRun * n_l; e += blockDim.x) {
        const int r = e / n_l, ll = e - r * n_l, l = l_base + ll;
        const int a = min(a0 + r, g.n_sc - 1);
        int lo, hi;
        pilot_bracket(a, g.port[l], g.comb, g.n_sc, lo, hi);
        s_klo[r][ll] = (lo - g.port[l]) / g.comb;
        s_khi[r][ll] = (hi - g.port[l]) / g.comb;
        s_w[r][ll] = interp_weight(a, lo, hi);
    }
    __syncthreads();
    // 2. thread (layer, unit) writes its unit of every subcarrier of the run
    const int ll = t / units, u = t - ll * units;
    if (ll >= n_l) return;
    const int l = l_base + ll;
    const T *tab = ls + ((slot * g.n_layers + l) * (long long)kmax) * units + u;
    T *out = H + ((slot * g.n_sc + a0) * g.n_layers + l) * (long long)units + u;
    const long long stride = (long long)g.n_layers * units;
    const int rn = min(kRun, g.n_sc - a0);
    for (int r = 0; r < rn; ++r, out += stride) {
        const T f0 = lerp_unit(__ldg(&tab[s_klo[r][ll] * units]), __ldg(&tab[s_khi[r][ll] * units]), s_w[r][ll]);
        if constexpr (!TV) {
            *out = f0;
        } else {
            const T *tab1 = tab + tab_stride;
            const T f1 = lerp_unit(__ldg(&tab1[s_klo[r][ll] * units]), __ldg(&tab1[s_khi[r][ll] * units]), s_w[r][ll]);
            for (int q = 0; q < g.n_groups; ++q) out[q * h_stride] = lerp_unit(f0, f1, g.group_t[q]);
        }
    }
}

// LS estimate at every pilot subcarrier of every layer (the element-wise division alone):
// ls[slot][l][k][b] for the layer's k-th pilot q = port[l] + k * comb (k < kmax; zero past n_sc).
__global__ void __launch_bounds__(256)
ls_pilots_kernel(ChestArgs g, int kmax, int sym, const float2 *__restrict__ beam, const float2 *__restrict__ pilots,
                 float2 *__restrict__ ls) {
    // grid.y = slot * n_layers + l, grid.x: chunks of the layer's kmax * n_beams (pilot, beam) elements
    const long long sl = blockIdx.y;
    const long long slot = sl / g.n_layers;
    const int l = (int)(sl - slot * g.n_layers);
    const int per_l = kmax * g.n_beams;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= per_l) return;
    const int k = idx / g.n_beams, b = idx - k * g.n_beams;
    const int q = g.port[l] + k * g.comb;
    float2 v = make_float2(0.f, 0.f);
    if (q < g.n_sc) {
        const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
        const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
        const float2 *p0 = pilots + sl * 2LL * g.n_sc;
        if (g.dmrs_type == 1) {
            // type-1 DMRS: q is the centre of the CDM pair q - 1, q + 1 (both inside the band: n_sc % 4 == 0);
            // 1/2 (y(q-1) / p(q-1) + y(q+1) / p(q+1)) despreads the OCC, per DMRS symbol
            auto pair = [&](const float2 *y, int j) {
                const float2 *p = p0 + (long long)j * g.n_sc;
                return ls_value(__ldg(&y[(long long)(q - 1) * g.n_beams + b]), __ldg(&y[(long long)(q + 1) * g.n_beams + b]),
                                pilot_inverse(__ldg(&p[q - 1])), pilot_inverse(__ldg(&p[q + 1])));
            };
            if (sym < 0)
                v = cscale(cadd(pair(y0, 0), pair(y1, 1)), 0.5f);
            else
                v = sym == 0 ? pair(y0, 0) : pair(y1, 1);
        } else if (sym < 0)   // the mean of the two DMRS symbols
            v = ls_value(__ldg(&y0[(long long)q * g.n_beams + b]), __ldg(&y1[(long long)q * g.n_beams + b]),
                         pilot_inverse(__ldg(&p0[q])), pilot_inverse(__ldg(&p0[g.n_sc + q])));
        else           // one DMRS symbol alone
            v = cmul(__ldg(&(sym == 0 ? y0 : y1)[(long long)q * g.n_beams + b]),
                     pilot_inverse(__ldg(&p0[(sym == 0 ? 0 : g.n_sc) + q])));
    }
    ls[sl * per_l + idx] = v;
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
    const int per_l = kmax * g.n_beams;                     // < 2^31: n_sc <= 4096, n_beams <= 64
    const int per_slot = g.n_layers * per_l;
    const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
    const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
    float sum = 0.f, cnt = 0.f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < per_slot; idx += gridDim.x * blockDim.x) {
        const int l = idx / per_l;
        const int rem = idx - l * per_l;
        const int k = rem / g.n_beams, b = rem - k * g.n_beams;
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

// The same with type-1 DMRS (the two ports of a CDM group share its REs): element (group, pair, beam) fits the
// group's m = 1 or 2 layers to the pair's 4 observations y_j(k) (k = k0, k0 + 2; j = the two DMRS symbols) by
// h_l = 1/4 sum y_j(k) / p_{l,j}(k) (least squares: the group's pilot vectors are orthogonal, unit modulus) and
// sums |y_j(k) - sum_l h_l p_{l,j}(k)|^2 with 4 - m degrees of freedom. partial = {sum, degrees of freedom}.
struct NeType1Args {
    int n_sc, n_beams, n_layers, n_sym, dmrs0, dmrs1, n_pairs;
    int m0, m1;                  // layers in CDM group 0 / 1
    int l00, l01, l10, l11;      // their indices (group, slot in group)
};

__global__ void __launch_bounds__(256)
ne_partial_type1_kernel(NeType1Args g, const float2 *__restrict__ beam, const float2 *__restrict__ pilots,
                        float2 *__restrict__ partial) {
    __shared__ float2 red[8];
    const long long slot = blockIdx.y;
    const int per_group = g.n_pairs * g.n_beams;
    const float2 *y0 = beam + (slot * g.n_sym + g.dmrs0) * (long long)g.n_sc * g.n_beams;
    const float2 *y1 = beam + (slot * g.n_sym + g.dmrs1) * (long long)g.n_sc * g.n_beams;
    const float2 *pl = pilots + slot * g.n_layers * 2LL * g.n_sc;
    float sum = 0.f, dof = 0.f;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 2 * per_group; idx += gridDim.x * blockDim.x) {
        const int delta = idx >= per_group ? 1 : 0;
        const int rem = idx - delta * per_group;
        const int n = rem / g.n_beams, b = rem - n * g.n_beams;
        const int m = delta ? g.m1 : g.m0;
        if (m == 0) continue;
        const int la = delta ? g.l10 : g.l00, lb = delta ? g.l11 : g.l01;
        const int k0 = 4 * n + delta, k1 = k0 + 2;
        const float2 v[4] = {__ldg(&y0[(long long)k0 * g.n_beams + b]), __ldg(&y0[(long long)k1 * g.n_beams + b]),
                             __ldg(&y1[(long long)k0 * g.n_beams + b]), __ldg(&y1[(long long)k1 * g.n_beams + b])};
        float2 p[2][4], h[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const float2 *pu = pl + (long long)(u == 0 ? la : lb) * 2 * g.n_sc;
            p[u][0] = __ldg(&pu[k0]);
            p[u][1] = __ldg(&pu[k1]);
            p[u][2] = __ldg(&pu[g.n_sc + k0]);
            p[u][3] = __ldg(&pu[g.n_sc + k1]);
            h[u] = make_float2(0.f, 0.f);
#pragma unroll
            for (int o = 0; o < 4; ++o) h[u] = cadd(h[u], cmul(v[o], pilot_inverse(p[u][o])));
            h[u] = cscale(h[u], 0.25f);
        }
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            float2 e = csub(v[o], cmul(h[0], p[0][o]));
            if (m == 2) e = csub(e, cmul(h[1], p[1][o]));
            sum += e.x * e.x + e.y * e.y;
        }
        dof += (float)(4 - m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
        dof += __shfl_xor_sync(0xFFFFFFFFu, dof, o);
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = make_float2(sum, dof);
    __syncthreads();
    if (threadIdx.x == 0) {
        float2 t = make_float2(0.f, 0.f);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = cadd(t, red[w]);
        partial[slot * gridDim.x + blockIdx.x] = t;
    }
}

// Pass 2: one warp per slot adds the parts in a fixed order; sigma2[slot] = factor * sum / count. Comb pilots:
// factor 2 (it undoes the two-symbol mean: E|y_j - LS p_j|^2 = sigma^2 / 2 for unit-modulus pilots); type-1:
// factor 1 (the count is already the degrees of freedom).
__global__ void ne_final_kernel(int n_parts, const float2 *__restrict__ partial, float *__restrict__ sigma2,
                                float factor) {
    const int slot = blockIdx.x, lane = threadIdx.x;
    float2 t = make_float2(0.f, 0.f);
    for (int p = lane; p < n_parts; p += 32) t = cadd(t, partial[(long long)slot * n_parts + p]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t.x += __shfl_xor_sync(0xFFFFFFFFu, t.x, o);
        t.y += __shfl_xor_sync(0xFFFFFFFFu, t.y, o);
    }
    if (lane == 0) sigma2[slot] = t.y > 0.f ? factor * t.x / t.y : 0.f;
}

}  // namespace

int ls_pilots_per_layer(const Geometry &g) { return (g.n_sc + g.comb - 1) / g.comb; }

cudaError_t launch_noise_est(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots,
                             float2 *partial, float *sigma2, cudaStream_t st) {
    if (n_slots == 0) return cudaSuccess;
    if (n_slots > 65535) return cudaErrorInvalidValue;
    if (g.dmrs_type == 1) {
        NeType1Args a{};
        a.n_sc = g.n_sc;
        a.n_beams = g.n_beams;
        a.n_layers = g.n_layers;
        a.n_sym = g.n_sym;
        a.dmrs0 = g.dmrs0;
        a.dmrs1 = g.dmrs1;
        a.n_pairs = g.n_sc / 4;                    // n_sc % 4 == 0 for type-1 cells: every pair complete
        int cnt[2] = {0, 0}, lay[2][2] = {{0, 0}, {0, 0}};
        for (int l = 0; l < g.n_layers; ++l) {
            const int grp = g.port[l] - 1;         // the geometry's pair-centre offset is 1 + CDM group
            if (grp >= 0 && grp < 2 && cnt[grp] < 2) lay[grp][cnt[grp]++] = l;
        }
        a.m0 = cnt[0];
        a.m1 = cnt[1];
        a.l00 = lay[0][0];
        a.l01 = lay[0][1];
        a.l10 = lay[1][0];
        a.l11 = lay[1][1];
        ne_partial_type1_kernel<<<dim3(kNoiseParts, (unsigned)n_slots), 256, 0, st>>>(a, beam, pilots, partial);
    } else {
        const ChestArgs a = chest_args(g);
        ne_partial_kernel<<<dim3(kNoiseParts, (unsigned)n_slots), 256, 0, st>>>(a, ls_pilots_per_layer(g), beam,
                                                                                 pilots, partial);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ne_final_kernel<<<(unsigned)n_slots, 32, 0, st>>>(kNoiseParts, partial, sigma2, g.dmrs_type == 1 ? 1.f : 2.f);
    return cudaGetLastError();
}

cudaError_t launch_ls_pilots(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *ls,
                             cudaStream_t st, int sym) {
    const ChestArgs a = chest_args(g);
    const int kmax = ls_pilots_per_layer(g);
    const long long rows = (long long)n_slots * g.n_layers;
    if (rows == 0) return cudaSuccess;
    if (rows > 65535) return cudaErrorInvalidValue;   // grid.y; n_slots * n_layers per call
    const int per_l = kmax * g.n_beams;
    ls_pilots_kernel<<<dim3((unsigned)((per_l + 255) / 256), (unsigned)rows), 256, 0, st>>>(a, kmax, sym, beam, pilots,
                                                                                           ls);
    return cudaGetLastError();
}

size_t ls_table_elems(const Geometry &g, int n_slots) {
    return (size_t)n_slots * g.n_layers * ls_pilots_per_layer(g) * g.n_beams;
}

cudaError_t launch_chest_interp(const Geometry &g, int n_slots, const float2 *ls, float2 *H, cudaStream_t st,
                                bool time_groups) {
    const ChestArgs a = chest_args(g);
    if ((long long)n_slots * g.n_sc == 0) return cudaSuccess;
    if (n_slots > 65535) return cudaErrorInvalidValue;                 // grid.y
    const int kmax = ls_pilots_per_layer(g);
    const bool pairs = (g.n_beams & 1) == 0;
    const int units = pairs ? g.n_beams / 2 : g.n_beams;
    const int lpc = std::min(g.n_layers, 1024 / units);                  // layers per CTA (units <= 64)
    const dim3 grid((unsigned)((g.n_sc + kRun - 1) / kRun), (unsigned)n_slots, (unsigned)((g.n_layers + lpc - 1) / lpc));
    const int threads = lpc * units;
    // table and estimate strides in units (the second DMRS symbol's table; the next group's estimate)
    const long long tab_u = (long long)ls_table_elems(g, n_slots) / (pairs ? 2 : 1);
    const long long h_u = (long long)n_slots * g.n_sc * g.n_layers * units;
    if (pairs) {
        const float4 *l4 = reinterpret_cast<const float4 *>(ls);
        float4 *h4 = reinterpret_cast<float4 *>(H);
        if (time_groups) chest_interp_kernel<float4, true><<<grid, threads, 0, st>>>(a, kmax, units, lpc, l4, tab_u, h4, h_u);
        else chest_interp_kernel<float4, false><<<grid, threads, 0, st>>>(a, kmax, units, lpc, l4, tab_u, h4, h_u);
    } else {
        if (time_groups) chest_interp_kernel<float2, true><<<grid, threads, 0, st>>>(a, kmax, units, lpc, ls, tab_u, H, h_u);
        else chest_interp_kernel<float2, false><<<grid, threads, 0, st>>>(a, kmax, units, lpc, ls, tab_u, H, h_u);
    }
    return cudaGetLastError();
}

cudaError_t launch_chest_ls(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *H,
                            float2 *ls_scratch, cudaStream_t st) {
    cudaError_t e = launch_ls_pilots(g, n_slots, beam, pilots, ls_scratch, st);
    if (e != cudaSuccess) return e;
    return launch_chest_interp(g, n_slots, ls_scratch, H, st);
}

cudaError_t launch_chest_time(const Geometry &g, int n_slots, const float2 *beam, const float2 *pilots, float2 *H,
                              float2 *ls_scratch, cudaStream_t st) {
    cudaError_t e = launch_ls_pilots(g, n_slots, beam, pilots, ls_scratch, st, 0);
    if (e != cudaSuccess) return e;
    if ((e = launch_ls_pilots(g, n_slots, beam, pilots, ls_scratch + ls_table_elems(g, n_slots), st, 1)) != cudaSuccess)
        return e;
    return launch_chest_interp(g, n_slots, ls_scratch, H, st, true);
}

}  // namespace pusch
