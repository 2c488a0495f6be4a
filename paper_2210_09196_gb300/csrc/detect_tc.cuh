// Gram matrix and right-hand sides of the MMSE detector (Eq. 2: G = H^H H, r_d = H^H y_d) on the tensor
// cores, one subcarrier per warp at a time: warp-level mma.sync m16n8k8 with TF32 operands and FP32
// accumulation. A subcarrier's products are 16 (or 32) rows of layers against K = 2 N_B real values, which is
// the M = 16 of this instruction shape exactly (the 5th-generation tcgen05 products start at M = 64, where one
// subcarrier would fill an eighth of the tile).
//
// Real embedding, K along the interleaved (re, im) floats of a row, k = 2 b + c:
//   A[i][k]   = H[i][b].c                                 (the estimate tile as it sits in shared memory)
//   Re G = A A^T                                          (B = A^T: the A fragments serve as B fragments)
//   Im G = A R^T,  R[j][2 b] = Im H[j][b], R[j][2 b + 1] = -Re H[j][b]     (Im(conj(h_i) h_j))
//   Re r_d = A y_d,  Im r_d = A rot(y_d)                  (the 12 data symbols' re and im parts as 24 columns)
// FP32 accuracy from TF32 operands: every operand x is split into hi = x rounded to TF32 (10 explicit mantissa
// bits, ties away from zero, by an integer add and mask) and lo = x - hi (exact, |lo| <= 2^-11 |x|), which the
// tensor core reads truncated to TF32 (|x - hi - lo_tf32| <= 2^-21 |x|); each product is hi*hi + hi*lo + lo*hi
// (the lo*lo term, below 2^-22, dropped), accumulated small terms first. (The conversion instruction
// cvt.rna.tf32.f32 rounds the same way but measured 11 % slower here: it does not issue at the full rate.)
#pragma once

#include "detect_core.cuh"

namespace pusch {

__device__ __forceinline__ void tf32_split(float x, uint32_t &hi, uint32_t &lo) {
    hi = (__float_as_uint(x) + 0x1000u) & 0xffffe000u;   // round the magnitude at mantissa bit 13
    lo = __float_as_uint(x - __uint_as_float(hi));
}

__device__ __forceinline__ void mma_tf32_16x8x8(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// c += a b with a, b split in hi / lo parts (three products, the small ones first)
__device__ __forceinline__ void mma3_tf32(float (&c)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                          uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32_16x8x8(c, al, bh0, bh1);
    mma_tf32_16x8x8(c, ah, bl0, bl1);
    mma_tf32_16x8x8(c, ah, bh0, bh1);
}

// G and r_d (12 data symbols) of one subcarrier by the whole warp.
//   hf: the subcarrier's estimate rows as floats (row i at hf + i hsf, NL rows, 2 NB floats used)
//   yf: its data-symbol rows as floats (row d at yf + d ysf), overwritten by r_d: r_d[i] at float2 (d ys + i)
//   Gs: G[i][j] (float2) at Gs + i (NL + 2) + j, over the estimate rows (written after every lane has read them)
// Fragment layout of m16n8k8 (g = lane / 4, t = lane % 4): A rows g, g + 8 at columns t, t + 4; B column g at
// rows t, t + 4; the accumulator rows g, g + 8 at columns 2 t, 2 t + 1.
// NB = 0: the beam count nb at run time (a multiple of 4: K = 2 nb floats in steps of 8).
template <int NL, int NB>
__device__ __forceinline__ void gram_rhs_tc(const float *hf, int hsf, float *yf, int ysf, int ys, float2 *Gs, int lane,
                                            int nb = NB) {
    constexpr int MT = NL / 16;     // 16-row tiles of layers
    constexpr int NG = NL / 8;      // 8-column tiles of G's columns (each for Re and for Im)
    constexpr int GS = NL + 2;      // row stride of Gs (float2): the 16-byte row loads below spread over banks
    const int g = lane >> 2, t = lane & 3, to = t ^ 1;
    const float sg = (t & 1) ? -1.f : 1.f;  // the rotation's sign at column k0 + t (the parity of t)
    // right-hand-side columns of this lane's B fragments: tile 0 Re r_0..7; tile 1 Re r_8..11 (g < 4) or
    // Im r_0..3; tile 2 Im r_4..11
    const int d0 = g, d1 = g < 4 ? 8 + g : g - 4, d2 = 4 + g;
    const bool rot1 = g >= 4;
    float cg[MT][2 * NG][4], cr[MT][3][4];
#pragma unroll
    for (int m = 0; m < MT; ++m) {
#pragma unroll
        for (int n = 0; n < 2 * NG; ++n)
#pragma unroll
            for (int e = 0; e < 4; ++e) cg[m][n][e] = 0.f;
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) cr[m][q][e] = 0.f;
    }
    constexpr int kUnroll = NL == 16 ? 2 : 1;   // two K steps in flight for 16 layers (measured faster; not for 32)
#pragma unroll kUnroll
    for (int k0 = 0; k0 < 2 * (NB > 0 ? NB : nb); k0 += 8) {
        uint32_t ah[MT][4], al[MT][4];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const float *r0 = hf + (16 * m + g) * hsf + k0, *r1 = r0 + 8 * hsf;
            tf32_split(r0[t], ah[m][0], al[m][0]);
            tf32_split(r1[t], ah[m][1], al[m][1]);
            tf32_split(r0[t + 4], ah[m][2], al[m][2]);
            tf32_split(r1[t + 4], ah[m][3], al[m][3]);
        }
        // Re G: B column tile n = rows 8 n .. 8 n + 7 of A, i.e. registers (0, 2) or (1, 3) of A tile n / 2
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const int mb = n >> 1, j0 = n & 1, j1 = j0 + 2;
#pragma unroll
            for (int m = 0; m < MT; ++m)
                mma3_tf32(cg[m][n], ah[m], al[m], ah[mb][j0], ah[mb][j1], al[mb][j0], al[mb][j1]);
        }
        // Im G: B column tile n = the rotated rows 8 n .. 8 n + 7
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const float *rr = hf + (8 * n + g) * hsf + k0;
            uint32_t bh0, bl0, bh1, bl1;
            tf32_split(sg * rr[to], bh0, bl0);
            tf32_split(sg * rr[to + 4], bh1, bl1);
#pragma unroll
            for (int m = 0; m < MT; ++m) mma3_tf32(cg[m][NG + n], ah[m], al[m], bh0, bh1, bl0, bl1);
        }
        // right-hand sides: 24 columns in three tiles
        {
            uint32_t bh0, bl0, bh1, bl1;
            const float *y0 = yf + d0 * ysf + k0;
            tf32_split(y0[t], bh0, bl0);
            tf32_split(y0[t + 4], bh1, bl1);
#pragma unroll
            for (int m = 0; m < MT; ++m) mma3_tf32(cr[m][0], ah[m], al[m], bh0, bh1, bl0, bl1);
            const float *y1 = yf + d1 * ysf + k0;
            const int c1 = rot1 ? to : t;
            const float s1 = rot1 ? sg : 1.f;
            tf32_split(s1 * y1[c1], bh0, bl0);
            tf32_split(s1 * y1[c1 + 4], bh1, bl1);
#pragma unroll
            for (int m = 0; m < MT; ++m) mma3_tf32(cr[m][1], ah[m], al[m], bh0, bh1, bl0, bl1);
            const float *y2 = yf + d2 * ysf + k0;
            tf32_split(sg * y2[to], bh0, bl0);
            tf32_split(sg * y2[to + 4], bh1, bl1);
#pragma unroll
            for (int m = 0; m < MT; ++m) mma3_tf32(cr[m][2], ah[m], al[m], bh0, bh1, bl0, bl1);
        }
    }
    __syncwarp();  // every lane has read the estimate and data-symbol rows
#pragma unroll
    for (int m = 0; m < MT; ++m) {
#pragma unroll
        for (int n = 0; n < NG; ++n) {
            const int i = 16 * m + g, j = 8 * n + 2 * t;
            *reinterpret_cast<float4 *>(Gs + i * GS + j) =
                make_float4(cg[m][n][0], cg[m][NG + n][0], cg[m][n][1], cg[m][NG + n][1]);
            *reinterpret_cast<float4 *>(Gs + (i + 8) * GS + j) =
                make_float4(cg[m][n][2], cg[m][NG + n][2], cg[m][n][3], cg[m][NG + n][3]);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int c = 8 * q + 2 * t + (e & 1), i = 16 * m + g + 8 * (e >> 1);
                const int d = c < 12 ? c : c - 12;
                yf[2 * (d * ys + i) + (c < 12 ? 0 : 1)] = cr[m][q][e];
            }
    }
}

// Steps 2-4 of the 12-data-symbol detector for the warp's SPW = 32 / NL subcarriers: G and r_d of each on the
// tensor cores (gram_rhs_tc), then lane i of group grp takes row i of its subcarrier's G, adds the loading on
// the diagonal (identity rows past nl), and the Crout factorisation and the solves run as in detect_group.
//   Hw, Yw: the warp's estimate tiles (stride ht float2 per subcarrier, rows hs) and data-symbol rows (12 per
//   subcarrier, stride ys). Returns true when a pivot of lane i's subcarrier was not a positive finite number.
//   NB = 0: nb beams at run time (a multiple of 4; the ragged batch's segments). G overlays the estimate tile:
//   ht >= NL (NL + 2) float2.
template <int NL, int NB>
__device__ __forceinline__ bool detect_group_tc(float2 *Hw, int ht, int hs, float2 *Yw, int ys, int nl, float load,
                                                int grp, int i, int src0, int lane, float2 (&acc)[12],
                                                const float *__restrict__ sigma2 = nullptr, long long slot = 0,
                                                int nb = NB) {
    constexpr int SPW = 32 / NL, GS = NL + 2;
#pragma unroll 1
    for (int gg = 0; gg < SPW; ++gg)
        gram_rhs_tc<NL, NB>(reinterpret_cast<const float *>(Hw + gg * ht), 2 * hs,
                            reinterpret_cast<float *>(Yw + gg * 12 * ys), 2 * ys, ys, Hw + gg * ht, lane, nb);
    __syncwarp();
    float2 G[NL];
    {
        const float4 *row = reinterpret_cast<const float4 *>(Hw + grp * ht + i * GS);
#pragma unroll
        for (int j = 0; j < NL / 2; ++j) {
            const float4 v = row[j];
            G[2 * j] = make_float2(v.x, v.y);
            G[2 * j + 1] = make_float2(v.z, v.w);
        }
    }
    if (sigma2) load += __ldg(&sigma2[slot]);
#pragma unroll
    for (int j = 0; j < NL; ++j)
        if (j == i) G[j] = (i < nl) ? make_float2(G[j].x + load, 0.f) : make_float2(1.f, 0.f);
    __syncwarp();  // every lane holds its row of G: the tile takes L
    return factor_solve_rhs_lanes<NL, 12, 12, true>(G, Yw + grp * 12 * ys, Hw + grp * ht, ys, 12, i, src0, acc);
}

}  // namespace pusch
