// LS estimate at a pilot subcarrier and its linear interpolation (Section II: block-type pilots, LS is
// an element-wise division), shared by the channel-estimation kernels, the ragged batch's detector (which
// interpolates its estimate itself) and the learned estimator's fallback, so that all produce identical values.
#pragma once

#include "internal.cuh"

namespace pusch {

// 1 / p as conj(p) / |p|^2: the per-pilot factor of the element-wise division.
__device__ __forceinline__ float2 pilot_inverse(float2 p) {
    const float s = 1.f / (p.x * p.x + p.y * p.y);
    return make_float2(p.x * s, -p.y * s);
}

// LS estimate at a pilot subcarrier: 1/2 (y0 / p0 + y1 / p1) = 1/2 (y0 q0 + y1 q1) with q = 1 / p.
__device__ __forceinline__ float2 ls_value(float2 y0, float2 y1, float2 q0, float2 q1) {
    return cscale(cadd(cmul(y0, q0), cmul(y1, q1)), 0.5f);
}

// Neighbouring pilot subcarriers of subcarrier a for a layer with comb offset `port` (pilots on
// q % comb == port, q < n_sc): lo <= a <= hi, lo == hi at or outside the first/last pilot.
__device__ __forceinline__ void pilot_bracket(int a, int port, int comb, int n_sc, int &lo, int &hi) {
    const int first = port;
    const int last = port + ((n_sc - 1 - port) / comb) * comb;
    if (a <= first) {
        lo = hi = first;
    } else if (a >= last) {
        lo = hi = last;
    } else {
        lo = port + ((a - port) / comb) * comb;
        hi = (lo == a) ? lo : lo + comb;
    }
}

// Interpolation weight (a - lo) / (hi - lo) (0 when lo == hi).
__device__ __forceinline__ float interp_weight(int a, int lo, int hi) {
    return hi == lo ? 0.f : (float)(a - lo) / (float)(hi - lo);
}

// h_lo + w (h_hi - h_lo)
__device__ __forceinline__ float2 interp(float2 h_lo, float2 h_hi, float w) {
    return make_float2(fmaf(w, h_hi.x - h_lo.x, h_lo.x), fmaf(w, h_hi.y - h_lo.y, h_lo.y));
}

}  // namespace pusch
