"""Pins of the oracle's FP8 (E4M3) form of the beamforming product: the rounding against the format's own bit
definition and a library cast, the power-of-two block scale against its definition, the block quantiser's
error bound, and the block-scaled product against the pinned FP64 product (orc_beamform) of exactly
representable operands and of operands quantised by the pinned row quantiser."""
import numpy as np
import pytest

RNG = np.random.default_rng(8)


def e4m3_decode(code: int) -> float:
    """Value of an E4M3 bit pattern from the format definition (sign, 4-bit exponent bias 7, 3-bit mantissa;
    S.1111.111 is NaN)."""
    s = -1.0 if code & 0x80 else 1.0
    e = (code >> 3) & 0xF
    m = code & 0x7
    if e == 0xF and m == 0x7:
        return float("nan")
    if e == 0:
        return s * (m / 8.0) * 2.0 ** -6
    return s * (1.0 + m / 8.0) * 2.0 ** (e - 7)


FINITE = sorted({e4m3_decode(c) for c in range(256) if not np.isnan(e4m3_decode(c))})


def test_every_code_is_a_fixed_point_and_448_is_the_largest(orc):
    vals = np.array(FINITE)
    assert len(vals) == 253                 # 2 * 126 nonzero finite magnitudes + one zero (+0 == -0)
    assert np.array_equal(orc.e4m3_round(vals), vals)
    assert vals.max() == 448.0 and vals.min() == -448.0
    assert min(v for v in FINITE if v > 0) == 2.0 ** -9


def test_midpoints_round_to_even_mantissa(orc):
    pos = [v for v in FINITE if v >= 0]
    codes = {e4m3_decode(c): c for c in range(128) if not np.isnan(e4m3_decode(c))}
    for lo, hi in zip(pos[:-1], pos[1:]):
        mid = 0.5 * (lo + hi)
        want = lo if codes[lo] % 2 == 0 else hi
        assert orc.e4m3_round([mid])[0] == want, (lo, hi)
        assert orc.e4m3_round([-mid])[0] == -want
        # just off the midpoint the nearer value wins
        assert orc.e4m3_round([np.nextafter(mid, 0)])[0] == lo
        assert orc.e4m3_round([np.nextafter(mid, 1e9)])[0] == hi


def test_saturation_and_nan(orc):
    out = orc.e4m3_round([449.0, 464.0, 465.0, 1e30, -1e30, np.inf, np.nan])
    assert list(out[:6]) == [448.0, 448.0, 448.0, 448.0, -448.0, 448.0]
    assert np.isnan(out[6])


def test_rounding_matches_library_cast(orc):
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 dtype")
    v = RNG.uniform(-1, 1, 20000) * 2.0 ** RNG.integers(-12, 9, 20000)
    v = np.clip(v, -448, 448).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(orc.e4m3_round(v), ref)


def test_block_exponent_definition(orc):
    assert orc.e4m3_block_exp(448.0) == 0
    assert orc.e4m3_block_exp(448.0 * (1 + 2.0 ** -40)) == 1
    assert orc.e4m3_block_exp(224.0) == -1
    assert orc.e4m3_block_exp(448.0 * 2.0 ** -20) == -20
    assert orc.e4m3_block_exp(0.0) == -126 and orc.e4m3_block_exp(1e-300) == -126
    assert orc.e4m3_block_exp(np.inf) == 128 and orc.e4m3_block_exp(np.nan) == 128
    for a in RNG.uniform(0, 1, 200) * 10.0 ** RNG.integers(-20, 20, 200):
        e = orc.e4m3_block_exp(a)
        assert a <= 448.0 * 2.0 ** e and (e == -126 or a > 448.0 * 2.0 ** (e - 1))


def test_row_quantisation_error_bound_and_range(orc):
    x = (RNG.standard_normal((5, 300)) + 1j * RNG.standard_normal((5, 300))) * 10.0 ** RNG.integers(-3, 3, (5, 1))
    x[2, 128:256] = 0.0                                          # an all-zero block
    codes, exps = orc.e4m3_quant_rows(x)
    assert exps.shape == (5, 3)
    assert np.all(exps[2, 1] == -126) and np.all(codes[2, 128:256] == 0)
    for r in range(5):
        for j in range(3):
            blk = slice(128 * j, min(300, 128 * j + 128))
            v, c, e = x[r, blk], codes[r, blk], exps[r, j]
            comp_v = np.r_[v.real, v.imag]
            comp_c = np.r_[c.real, c.imag]
            if np.all(comp_v == 0):
                continue
            assert 224.0 < np.abs(comp_v).max() / 2.0 ** e <= 448.0
            assert np.abs(comp_c).max() <= 448.0
            err = np.abs(comp_c * 2.0 ** e - comp_v)
            # half a unit in the last place: 2^-4 relative for normal codes, 2^-10 * 2^e absolute below 2^-6
            bound = np.maximum(2.0 ** -4 * np.abs(comp_v), 2.0 ** -10 * 2.0 ** e)
            assert np.all(err <= bound * (1 + 1e-12))


def test_nonfinite_block_is_marked(orc):
    x = np.ones((1, 200), complex)
    x[0, 150] = np.nan
    codes, exps = orc.e4m3_quant_rows(x)
    assert exps[0, 0] == orc.e4m3_block_exp(1.0) == -8 and exps[0, 1] == 128
    assert np.all(np.isnan(codes[0, 128:]))


def test_fp8_product_of_coarse_grid_operands_by_brute_force(orc):
    """Codes on a coarse E4M3 grid and weights k/8 (exact at their block scale): the block-scaled product is
    W^H x of the dequantised operands, summed here by brute force."""
    n_sym, n_rx, n_sc, n_beams = 2, 20, 260, 3
    codes = (RNG.integers(-7, 8, (n_sym, n_rx, n_sc)) + 1j * RNG.integers(-7, 8, (n_sym, n_rx, n_sc))) * 16.0
    exps = RNG.integers(-3, 3, (n_sym, n_rx, 3)).astype(np.int32)
    # W with entries k/8 (k < 8) in one block: block max 7/8 -> exponent -9, codes k * 64 exactly
    W = (RNG.integers(-7, 8, (n_rx, n_beams)) + 1j * RNG.integers(-7, 8, (n_rx, n_beams))) / 8.0
    W[0, :] = 7.0 / 8.0                                          # every beam's block max is exactly 7/8
    beam = orc.beamform_fp8(codes, exps, W)
    X = codes * 2.0 ** np.repeat(exps, 128, axis=2)[:, :, :n_sc]
    want = np.einsum("rb,sra->sab", W.conj(), X)
    assert np.allclose(beam, want, rtol=0, atol=1e-12)


def test_fp8_product_keeps_small_blocks_exact(orc):
    """Hand case: two antennas, one subcarrier, W = [1, 1]^T. Antenna 1's block exponent is 8 below antenna 0's;
    the block-scaled product adds 1.125 * 2^-8 exactly (no operand is re-rounded onto another block's grid)."""
    codes = np.array([[[2.0], [1.125]]], complex)                # [sym][rx][sc]
    exps = np.array([[[0], [-8]]], np.int32)
    W = np.array([[1.0], [1.0]], complex)                        # block max 1 -> exponent -8, code 256
    beam = orc.beamform_fp8(codes, exps, W)
    assert beam[0, 0, 0] == 2.0 + 1.125 * 2.0 ** -8
    exps_nan = np.array([[[0], [128]]], np.int32)
    assert np.isnan(orc.beamform_fp8(codes, exps_nan, W)[0, 0, 0])


def _e4m3_values(shape):
    """Random finite E4M3 values (every code but NaN), from the format definition."""
    return np.array(FINITE)[RNG.integers(0, len(FINITE), shape)]


def test_fp8_product_equals_the_fp64_product_of_representable_operands(orc):
    """Samples that are E4M3 values times their block scales and weights that are E4M3 values on their own
    block's scale are reproduced exactly by the quantisation, so the FP8 product must equal the pinned FP64
    beamforming product orc_beamform of the same operands (130 antennas: two weight blocks)."""
    n_sym, n_rx, n_sc, n_beams = 2, 130, 200, 3
    codes = _e4m3_values((n_sym, n_rx, n_sc)) + 1j * _e4m3_values((n_sym, n_rx, n_sc))
    exps = RNG.integers(-20, 20, (n_sym, n_rx, 2)).astype(np.int32)
    x = codes * 2.0 ** np.repeat(exps, 128, axis=2)[:, :, :n_sc]
    # weights: E4M3 values whose block maximum is exactly 448 * 2^e_w, so the block exponent is e_w
    ew = np.array([[-12, -3], [-9, -9], [0, -20]])                 # [beam][block]
    W = _e4m3_values((n_rx, n_beams)) + 1j * _e4m3_values((n_rx, n_beams))
    for b in range(n_beams):
        W[0, b] = 448.0
        W[128, b] = 448.0
        W[:128, b] *= 2.0 ** ew[b, 0]
        W[128:, b] *= 2.0 ** ew[b, 1]
    beam = orc.beamform_fp8(codes, exps, W)
    want = orc.beamform(x, W)
    assert np.max(np.abs(beam - want)) <= 1e-13 * np.max(np.abs(want))


def test_fp8_product_quantises_w_like_the_row_quantiser(orc):
    """Arbitrary W: the product equals orc_beamform of the samples and of W quantised by the pinned row
    quantiser (orc_e4m3_quant_rows over W's beam rows: blocks of 128 antennas)."""
    n_sym, n_rx, n_sc, n_beams = 1, 300, 140, 5
    codes = _e4m3_values((n_sym, n_rx, n_sc)) + 1j * _e4m3_values((n_sym, n_rx, n_sc))
    exps = RNG.integers(-6, 6, (n_sym, n_rx, 2)).astype(np.int32)
    x = codes * 2.0 ** np.repeat(exps, 128, axis=2)[:, :, :n_sc]
    W = (RNG.standard_normal((n_rx, n_beams)) + 1j * RNG.standard_normal((n_rx, n_beams))) * 10.0 ** RNG.integers(-3, 3, (1, n_beams))
    cw, ew = orc.e4m3_quant_rows(W.T)
    Wq = (cw * 2.0 ** np.repeat(ew, 128, axis=1)[:, :n_rx]).T
    beam = orc.beamform_fp8(codes, exps, W)
    want = orc.beamform(x, Wq)
    assert np.max(np.abs(beam - want)) <= 1e-13 * np.max(np.abs(want))
