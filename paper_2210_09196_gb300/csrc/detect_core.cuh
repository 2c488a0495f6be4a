// Per-subcarrier MMSE detection core (Eq. 2; Section II Cholesky + two triangular solves; Section V-C),
// shared by the single-cell detector and the ragged multi-cell detector.
//
// A group of NL lanes owns one subcarrier; lane i owns layer i. Inputs in shared memory: the group's
// estimate rows H[l][b] (stride hs, rows >= nl zero) and its data-symbol vectors y_d[b] (stride hs).
// Output: x_i for every data symbol in registers. The L tile ([NL][NL + 1] complex + NL floats) may alias
// the H rows: it is written only after the last read of H.
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
// later holds L ([NL][NL + 1]).
__host__ __device__ __forceinline__ int row_stride(int nb) { return (nb + 3) & ~1; }
template <int NL>
__host__ __device__ __forceinline__ int htile(int nb) {
    const int a = NL * row_stride(nb), b = NL * (NL + 1) + NL / 2;  // L tile + 1/L[k][k] (NL floats)
    const int m = a > b ? a : b;
    // the next subcarrier's tile starts 16 bytes further into the 128-byte bank cycle, so that the groups of a
    // warp reading the same element of their own tiles (broadcast 16-byte loads) hit different banks
    return m + ((2 - m) & 15);
}

// Row stride of the data-symbol rows in the single-cell detector: at least NL for the 16- and 32-layer classes,
// whose
// solve transposes the right-hand sides through those rows (detect_group, RHS_LANES).
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


__device__ __forceinline__ float2 det_shfl2(float2 v, int src) {
    return make_float2(__shfl_sync(kDetFull, v.x, src), __shfl_sync(kDetFull, v.y, src));
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

// Steps 3-4 for the 16- and 32-layer classes (lane i holds row i of G; r_d[i] in acc[d]):
//   * r_d[i] goes to the group's (dead) data-symbol rows T[d][i] (stride ys >= NL);
//   * Crout Cholesky, column j at step j: s_i = G[i][j] - sum_{k<j} L[i][k] conj(L[j][k]) in lane i, the pivot
//     s_j broadcast by one shuffle, L[i][j] = s_i / sqrt(s_j); lane i keeps its row of L in registers and
//     publishes each entry to shared memory as (-Re, -Re, Im, Im) (packed lower triangle, rows in order), so
//     that every complex multiply-add below is one broadcast 16-byte load and two packed FMAs;
//   * lane d solves data symbol d: forward z_k = (r_k - sum_{j<k} L[k][j] z_j) / L[k][k], back
//     x_k = (z_k - sum_{j>k} conj(L[j][k]) x_j) / L[k][k], in registers; lanes d >= nd solve a copy of symbol 0;
//   * x_d[i] returns to lane i through T.
// Uses the H tile (lt) for L: 120 float4 + NL floats.
template <int NL, int ND, int NR>
__device__ __forceinline__ bool factor_solve_rhs_lanes(float2 (&G)[NL], float2 *yt, float2 *lt, int ys, int nd,
                                                       int i, int src0, float2 (&acc)[NR]) {
    constexpr unsigned kFull = kDetFull;
#pragma unroll
    for (int d = 0; d < NR; ++d)
        if (ND > 0 || d < nd) yt[d * ys + i] = acc[d];
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
            constexpr bool kSplit = NL >= 32;
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

    const int dl = i < nd ? i : 0;
    constexpr bool kSplitSolve = NL >= 32;  // as in the factorisation
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
    __syncwarp();  // every lane has read its row of T
    if (i < nd) {
#pragma unroll
        for (int k = 0; k < NL; k += 2)
            *reinterpret_cast<float4 *>(yt + i * ys + k) = make_float4(u[k].x, u[k].y, u[k + 1].x, u[k + 1].y);
    }
    __syncwarp();
#pragma unroll
    for (int d = 0; d < NR; ++d)
        if (ND > 0 || d < nd) acc[d] = yt[d * ys + i];
    return bad;
}

// RHS_LANES (16- and 32-layer classes): the solves run with one data symbol per lane instead of one layer per lane
// (below); the data-symbol rows yt then have stride ys >= NL and are overwritten.
template <int NL, int ND, int NR, bool RHS_LANES = false>
__device__ __forceinline__ bool detect_group(const float2 *__restrict__ hr, const float2 *__restrict__ hg,
                                             float2 *yt, float2 *lt, int hs, int nb, int nd,
                                             int nl, float load, int i, int src0, float2 (&acc)[NR],
                                             const float *__restrict__ sigma2 = nullptr, long long slot = 0,
                                             int ys = 0) {
    if (ys == 0) ys = hs;
    constexpr unsigned kFull = kDetFull;
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

    if constexpr (RHS_LANES) return factor_solve_rhs_lanes<NL, ND, NR>(G, yt, lt, ys, nd, i, src0, acc);

    // ---- 3. Cholesky, right-looking, row i of L replaces row i of G; then L -> shared memory
    bool bad = false;
    float dinv = 1.f;
#pragma unroll
    for (int j = 0; j < NL; ++j) {
        float dj = __shfl_sync(kFull, G[j].x, src0 + j);
        if (!(dj > 0.f) || !isfinite(dj)) {
            bad = true;
            dj = 1.f;
        }
        const float ljj = sqrtf(dj);
        const float inv = 1.f / ljj;
        if (i > j) G[j] = cscale(G[j], inv);
        else if (i == j) G[j] = make_float2(ljj, 0.f);
        else G[j] = make_float2(0.f, 0.f);
        if (i == j) dinv = inv;
#pragma unroll
        for (int k = j + 1; k < NL; ++k) {
            const float2 lkj = det_shfl2(G[j], src0 + k);
            if (i >= k) {
                // G[i][k] -= L[i][j] conj(L[k][j])
                G[k].x -= G[j].x * lkj.x + G[j].y * lkj.y;
                G[k].y -= G[j].y * lkj.x - G[j].x * lkj.y;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < NL; ++k) lt[i * (NL + 1) + k] = G[k];
    __syncwarp();

    // ---- 4. forward L z = r, then back L^H x = z, for all data symbols, in unit-diagonal form:
    //         with D = diag(L), u = D z solves (L D^-1) u = r and x solves (D^-1 L^H) x = D^-1 z, so each step
    //         broadcasts an unknown that is already final (no scaling before the shuffle). Lane i's unknown is
    //         final at step i and not updated afterwards. dv[k] = 1 / L[k][k] sits after L in shared memory.
    float *dv = reinterpret_cast<float *>(lt + NL * (NL + 1));
    dv[i] = dinv;
    __syncwarp();
    const float2 *lrow = lt + i * (NL + 1);  // L[i][k]
    // the k loops stay rolled: their bodies (NR shuffled updates) are large, and unrolling them all made the
    // kernel miss in the instruction cache
#pragma unroll 1
    for (int k = 0; k < NL; ++k) {
        const float2 m = cscale(lrow[k], dv[k]);  // L[i][k] / L[k][k]
#pragma unroll
        for (int d = 0; d < NR; ++d) {
            if (ND > 0 || d < nd) {
                const float2 uk = det_shfl2(acc[d], src0 + k);
                if (i > k) cfms(acc[d], m, uk);
            }
        }
    }
#pragma unroll
    for (int d = 0; d < NR; ++d) acc[d] = cscale(acc[d], dinv * dinv);  // z_i / L[i][i]
#pragma unroll 1
    for (int k = NL - 1; k >= 0; --k) {
        const float2 lki = cscale(lt[k * (NL + 1) + i], dinv);  // L[k][i] / L[i][i]
#pragma unroll
        for (int d = 0; d < NR; ++d) {
            if (ND > 0 || d < nd) {
                const float2 xk = det_shfl2(acc[d], src0 + k);
                if (i < k) {
                    // acc -= conj(L[k][i] / L[i][i]) x_k
                    acc[d].x -= lki.x * xk.x + lki.y * xk.y;
                    acc[d].y -= lki.x * xk.y - lki.y * xk.x;
                }
            }
        }
    }
    return bad;
}

}  // namespace pusch
