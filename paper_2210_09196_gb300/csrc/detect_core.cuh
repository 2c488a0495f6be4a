// Per-subcarrier MMSE detection core (Eq. 2; Section II Cholesky + two triangular solves; Section V-C),
// shared by the single-cell detector and the ragged multi-cell detector.
//
// A group of NL lanes owns one subcarrier; lane i owns layer i. Inputs in shared memory: the group's
// estimate rows H[l][b] (stride hs, rows >= nl zero) and its data-symbol vectors y_d[b] (stride ys >= NL).
// Output: x_i for every data symbol in registers. The packed L (NL(NL-1)/2 broadcast-ready float4 entries +
// NL floats 1/L[k][k]) aliases the H rows: it is written only after the last read of H.
#pragma once

#include "internal.cuh"

namespace pusch {

constexpr unsigned kDetFull = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Shared memory per subcarrier, in float2 units: the H tile (NL rows of an even stride >= nb + 1), which
// later holds the packed L (at most NL(NL + 1) + NL/2 float2, the second term of the maximum below).
__host__ __device__ __forceinline__ int row_stride(int nb) { return (nb + 3) & ~1; }
template <int NL>
__host__ __device__ __forceinline__ int htile(int nb) {
    const int a = NL * row_stride(nb), b = NL * (NL + 1) + NL / 2;  // L tile + 1/L[k][k] (NL floats)
    const int m = a > b ? a : b;
    // the next subcarrier's tile starts 16 bytes further into the 128-byte bank cycle, so that the groups of a
    // warp reading the same element of their own tiles (broadcast 16-byte loads) hit different banks
    return m + ((2 - m) & 15);
}

// Row stride of the data-symbol rows: at least NL, because the solves transpose the right-hand sides through
// those rows (below NL only for the 16- and 32-lane classes with few beams; the smaller classes always have
// row_stride(nb) >= NL).
template <int NL>
__host__ __device__ __forceinline__ int y_stride(int nb) {
    const int hs = row_stride(nb);
    return NL >= 16 && hs < NL ? NL : hs;
}

// Shared memory of one warp of the single-cell detector: per subcarrier the H tile and the data-symbol rows.
template <int NL>
__host__ __device__ __forceinline__ size_t warp_smem_bytes(int nb, int nd) {
    return (size_t)(32 / NL) * ((htile<NL>(nb) + (size_t)nd * y_stride<NL>(nb)) * sizeof(float2));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}


// Gray hard decisions (3GPP TS 38.211 5.1.3 / 5.1.4), ties to bit 0.
__device__ __forceinline__ uint8_t det_demap(float2 x, int q) {
    const float thr = 0.63245553203367586640f;  // 2 / sqrt(10), rounded to float
    uint8_t v = (uint8_t)(x.x < 0.f) | (uint8_t)((x.y < 0.f) << 1);
    if (q == 4) v |= (uint8_t)((fabsf(x.x) > thr) << 2) | (uint8_t)((fabsf(x.y) > thr) << 3);
    return v;
}

// Returns true when a pivot was not a positive finite number (the factorisation continued with 1).
// load: sigma^2 + extra loading, or, when sigma2 is not NULL, sigma2[slot] + load (the per-slot noise estimate;
// read only where the diagonal is loaded, so nothing extra stays live across the Gram loop).
// Shared-memory load kept in program order (volatile): the fully unrolled factorisation and solves would
// otherwise hoist their L loads far ahead of use and run out of registers.
__device__ __forceinline__ float4 lds4_ordered(const float4 *p) {
    float4 v;
    asm volatile("ld.volatile.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(smem_addr(p)));
    return v;
}

// Steps 3-4 (lane i holds row i of G; r_d[i] in acc[d]):
//   * r_d[i] goes to the group's (dead) data-symbol rows T[d][i] (stride ys >= NL);
//   * Crout Cholesky, column j at step j: s_i = G[i][j] - sum_{k<j} L[i][k] conj(L[j][k]) in lane i, the pivot
//     s_j broadcast by one shuffle, L[i][j] = s_i / sqrt(s_j); lane i keeps its row of L in registers and
//     publishes each entry to shared memory as (-Re, -Re, Im, Im) (packed lower triangle, rows in order), so
//     that every complex multiply-add below is one broadcast 16-byte load and two packed FMAs;
//   * lane i solves data symbols i, i + NL, ...: forward z_k = (r_k - sum_{j<k} L[k][j] z_j) / L[k][k], back
//     x_k = (z_k - sum_{j>k} conj(L[j][k]) x_j) / L[k][k], in registers (a lane past the last symbol solves a
//     copy of symbol 0 and discards it); the results are written back only after every lane has read;
//   * x_d[i] returns to lane i through T.
// Uses the H tile (lt) for L: 120 float4 + NL floats.
// kRhsInT: the r_d are already in T (written there by the tensor-core Gram), acc is only the output.
template <int NL, int ND, int NR, bool kRhsInT = false>
__device__ __forceinline__ bool factor_solve_rhs_lanes(float2 (&G)[NL], float2 *yt, float2 *lt, int ys, int nd,
                                                       int i, int src0, float2 (&acc)[NR]) {
    constexpr unsigned kFull = kDetFull;
    if constexpr (!kRhsInT) {
#pragma unroll
        for (int d = 0; d < NR; ++d)
            if (ND > 0 || d < nd) yt[d * ys + i] = acc[d];
    }
    float4 *L4 = reinterpret_cast<float4 *>(lt);                 // L[k][j], j < k, at k (k - 1) / 2 + j
    float *dv = reinterpret_cast<float *>(L4 + NL * (NL - 1) / 2);  // 1 / L[k][k]
    bool bad = false;
    float dinv = 1.f;
    {
        float2 Lrot[NL];  // (-Im, Re) of lane i's L entries
#pragma unroll
        for (int j = 0; j < NL; ++j) {
            // two partial sums (even and odd k) halve the dependent FMA chain where the registers allow (the
            // 16-layer class is at its 128-register cap and spills with them)
            constexpr bool kSplit = NL >= 16;
            float2 sj = G[j], sj1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < j; ++k) {
                const float4 b = lds4_ordered(L4 + j * (j - 1) / 2 + k);  // L[j][k], broadcast
                float2 &acc2 = (kSplit && (k & 1)) ? sj1 : sj;
                acc2 = __ffma2_rn(make_float2(b.x, b.y), G[k], acc2);      // G[k] holds L[i][k] by now
                acc2 = __ffma2_rn(make_float2(b.z, b.w), Lrot[k], acc2);
            }
            sj = __fadd2_rn(sj, sj1);
            float dj = __shfl_sync(kFull, sj.x, src0 + j);
            if (!(dj > 0.f) || !isfinite(dj)) {
                bad = true;
                dj = 1.f;
            }
            const float inv = rsqrtf(dj);
            if (i > j) G[j] = cscale(sj, inv);
            else if (i == j) G[j] = make_float2(dj * inv, 0.f);
            else G[j] = make_float2(0.f, 0.f);
            if (i == j) dinv = inv;
            Lrot[j] = make_float2(-G[j].y, G[j].x);
            if (i > j) L4[i * (i - 1) / 2 + j] = make_float4(-G[j].x, -G[j].x, G[j].y, G[j].y);
            __syncwarp();
        }
    }
    dv[i] = dinv;
    __syncwarp();

    // right-hand sides per lane: lane i solves data symbols i, i + NL, ... (one for 16 and 32 lanes; the
    // small classes take several); a lane past the last symbol solves a copy of symbol 0 and discards it
    constexpr int RPL = (NR + NL - 1) / NL;
    constexpr bool kSplitSolve = NL >= 16;  // as in the factorisation
    float2 X[RPL][NL];
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int d = i + NL * r;
        const int dl = d < nd ? d : 0;
        float2 u[NL], w[NL];
#pragma unroll
        for (int k = 0; k < NL; k += 2) {
            const float4 v = *reinterpret_cast<const float4 *>(yt + dl * ys + k);
            u[k] = make_float2(v.x, v.y);
            u[k + 1] = make_float2(v.z, v.w);
        }
        // forward: u_k += (-Re L) u_j + (Im L) (Im u_j, -Re u_j) = u_k - L[k][j] u_j
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            float2 u1 = make_float2(0.f, 0.f);  // odd-j partial sum (shorter dependent chain)
#pragma unroll
            for (int j = 0; j < k; ++j) {
                const float4 b = lds4_ordered(L4 + k * (k - 1) / 2 + j);
                float2 &acc2 = (kSplitSolve && (j & 1)) ? u1 : u[k];
                acc2 = __ffma2_rn(make_float2(b.x, b.y), u[j], acc2);
                acc2 = __ffma2_rn(make_float2(b.z, b.w), w[j], acc2);
            }
            u[k] = cscale(__fadd2_rn(u[k], u1), dv[k]);
            w[k] = make_float2(u[k].y, -u[k].x);
        }
        // back: u_k += (-Re L) x_j + (Im L) (-Im x_j, Re x_j) = u_k - conj(L[j][k]) x_j
#pragma unroll
        for (int k = NL - 1; k >= 0; --k) {
            float2 u1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int j = k + 1; j < NL; ++j) {
                const float4 b = lds4_ordered(L4 + j * (j - 1) / 2 + k);
                float2 &acc2 = (kSplitSolve && (j & 1)) ? u1 : u[k];
                acc2 = __ffma2_rn(make_float2(b.x, b.y), u[j], acc2);
                acc2 = __ffma2_rn(make_float2(b.z, b.w), w[j], acc2);
            }
            u[k] = cscale(__fadd2_rn(u[k], u1), dv[k]);
            w[k] = make_float2(-u[k].y, u[k].x);
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) X[r][k] = u[k];
    }
    __syncwarp();  // every lane has read its rows of T
#pragma unroll
    for (int r = 0; r < RPL; ++r) {
        const int d = i + NL * r;
        if (d < nd) {
#pragma unroll
            for (int k = 0; k < NL; k += 2)
                *reinterpret_cast<float4 *>(yt + d * ys + k) = make_float4(X[r][k].x, X[r][k].y, X[r][k + 1].x, X[r][k + 1].y);
        }
    }
    __syncwarp();
#pragma unroll
    for (int d = 0; d < NR; ++d)
        if (ND > 0 || d < nd) acc[d] = yt[d * ys + i];
    return bad;
}

// Steps 2-4 for one subcarrier per lane group; the data-symbol rows yt (stride ys >= NL) are overwritten.
template <int NL, int ND, int NR>
__device__ __forceinline__ bool detect_group(const float2 *__restrict__ hr, const float2 *__restrict__ hg,
                                             float2 *yt, float2 *lt, int hs, int nb, int nd,
                                             int nl, float load, int i, int src0, float2 (&acc)[NR],
                                             const float *__restrict__ sigma2 = nullptr, long long slot = 0,
                                             int ys = 0) {
    if (ys == 0) ys = hs;
    // ---- 2a. Gram row i: G[j] = sum_b conj(H[i][b]) H[j][b], with packed FP32x2 FMAs: P[j] = sum_b Re(h_b) H[j][b]
    //         and Q[j] = sum_b Im(h_b) H[j][b] (h_b = H[i][b]), then G[j] = P[j] - i Q[j].
    float2 G[NL];
    {
        float2 P[NL], Q[NL];
#pragma unroll
        for (int j = 0; j < NL; ++j) P[j] = Q[j] = make_float2(0.f, 0.f);
        int b = 0;
        for (; b + 1 < nb; b += 2) {
            const float4 hv = *reinterpret_cast<const float4 *>(hr + b);
            const float2 hx0 = make_float2(hv.x, hv.x), hy0 = make_float2(hv.y, hv.y);
            const float2 hx1 = make_float2(hv.z, hv.z), hy1 = make_float2(hv.w, hv.w);
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const float4 gv = *reinterpret_cast<const float4 *>(hg + j * hs + b);
                const float2 g0 = make_float2(gv.x, gv.y), g1 = make_float2(gv.z, gv.w);
                P[j] = __ffma2_rn(hx0, g0, P[j]);
                Q[j] = __ffma2_rn(hy0, g0, Q[j]);
                P[j] = __ffma2_rn(hx1, g1, P[j]);
                Q[j] = __ffma2_rn(hy1, g1, Q[j]);
            }
        }
        if (b < nb) {
            const float2 h0 = hr[b];
            const float2 hx0 = make_float2(h0.x, h0.x), hy0 = make_float2(h0.y, h0.y);
#pragma unroll
            for (int j = 0; j < NL; ++j) {
                const float2 g0 = hg[j * hs + b];
                P[j] = __ffma2_rn(hx0, g0, P[j]);
                Q[j] = __ffma2_rn(hy0, g0, Q[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < NL; ++j) G[j] = make_float2(P[j].x + Q[j].y, P[j].y - Q[j].x);
    }
    if (sigma2) load += __ldg(&sigma2[slot]);
#pragma unroll
    for (int j = 0; j < NL; ++j)
        if (j == i) G[j] = (i < nl) ? make_float2(G[j].x + load, 0.f) : make_float2(1.f, 0.f);

    // ---- 2b. right-hand sides r_d = H^H y_d (y_d from the shared tile; a group reads one address), packed the
    //         same way: P[d] = sum_b Re(h_b) y_d[b], Q[d] = sum_b Im(h_b) y_d[b], r_d[i] = P[d] - i Q[d].
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncwarp();
    {
        float2 Q[NR];
#pragma unroll
        for (int d = 0; d < NR; ++d) acc[d] = Q[d] = make_float2(0.f, 0.f);
        int b = 0;
        for (; b + 1 < nb; b += 2) {
            const float4 hv = *reinterpret_cast<const float4 *>(hr + b);
            const float2 hx0 = make_float2(hv.x, hv.x), hy0 = make_float2(hv.y, hv.y);
            const float2 hx1 = make_float2(hv.z, hv.z), hy1 = make_float2(hv.w, hv.w);
#pragma unroll
            for (int d = 0; d < NR; ++d) {
                if (ND > 0 || d < nd) {
                    const float4 yv = *reinterpret_cast<const float4 *>(yt + d * ys + b);
                    const float2 y0 = make_float2(yv.x, yv.y), y1 = make_float2(yv.z, yv.w);
                    acc[d] = __ffma2_rn(hx0, y0, acc[d]);
                    Q[d] = __ffma2_rn(hy0, y0, Q[d]);
                    acc[d] = __ffma2_rn(hx1, y1, acc[d]);
                    Q[d] = __ffma2_rn(hy1, y1, Q[d]);
                }
            }
        }
        if (b < nb) {
            const float2 h0 = hr[b];
            const float2 hx0 = make_float2(h0.x, h0.x), hy0 = make_float2(h0.y, h0.y);
#pragma unroll
            for (int d = 0; d < NR; ++d)
                if (ND > 0 || d < nd) {
                    const float2 y0 = yt[d * ys + b];
                    acc[d] = __ffma2_rn(hx0, y0, acc[d]);
                    Q[d] = __ffma2_rn(hy0, y0, Q[d]);
                }
        }
#pragma unroll
        for (int d = 0; d < NR; ++d) acc[d] = make_float2(acc[d].x + Q[d].y, acc[d].y - Q[d].x);
    }
    __syncwarp();  // the H tile is reused for L below

    return factor_solve_rhs_lanes<NL, ND, NR>(G, yt, lt, ys, nd, i, src0, acc);
}

}  // namespace pusch
