"""The operand split behind the detector's tensor-core Gram (Eq. 2: G = H^H H + sigma^2 I, r = H^H y), emulated
bit for bit in numpy: hi = x rounded to TF32 by adding half a TF32 unit to the magnitude bits and masking the
low 13 mantissa bits, lo = x - hi in FP32 (exact), and the tensor core reading lo truncated to TF32.

Pins: the split carries x to 2^-21 |x|; the three products hi*hi + hi*lo + lo*hi of two such operands are
within about 2^-21 of the exact product; a Gram matrix formed that way with FP32 accumulation is as close to
the FP64 Gram as one formed with plain FP32 multiply-adds (a factor of a few), and far closer than a single
TF32 product (about 2^-11)."""
import numpy as np
import pytest

MASK = np.uint32(0xFFFFE000)


def tf32_hi(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    return ((b + np.uint32(0x1000)) & MASK).view(np.float32)


def tf32_trunc(x):
    return (np.asarray(x, dtype=np.float32).view(np.uint32) & MASK).view(np.float32)


def split(x):
    x = np.asarray(x, dtype=np.float32)
    hi = tf32_hi(x)
    lo = (x - hi).astype(np.float32)
    return hi, tf32_trunc(lo)


def test_split_carries_the_operand_to_2_pow_minus_21():
    rng = np.random.default_rng(1)
    x = (rng.standard_normal(200000) * 10.0 ** rng.uniform(-6, 6, 200000)).astype(np.float32)
    hi, lo = split(x)
    # hi has at most 10 explicit mantissa bits, lo is exact before truncation
    assert np.all((hi.view(np.uint32) & ~MASK) == 0)
    rel = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64)) / np.abs(x.astype(np.float64))
    assert rel.max() <= 2.0 ** -21
    # the rounding of hi: |x - hi| <= half a TF32 unit (2^-11 relative), ties away from zero
    assert np.max(np.abs(x.astype(np.float64) - hi) / np.abs(x.astype(np.float64))) <= 2.0 ** -11
    assert tf32_hi(np.float32(1.0 + 2.0 ** -11)) == np.float32(1.0 + 2.0 ** -10)     # a tie rounds away
    assert tf32_hi(np.float32(-(1.0 + 2.0 ** -11))) == np.float32(-(1.0 + 2.0 ** -10))


def test_three_products_hold_the_product_to_about_2_pow_minus_21():
    rng = np.random.default_rng(2)
    a = rng.standard_normal(100000).astype(np.float32)
    b = rng.standard_normal(100000).astype(np.float32)
    ah, al = split(a)
    bh, bl = split(b)
    # each TF32 x TF32 product is exact in FP32 (11 x 11 significant bits)
    p3 = (ah.astype(np.float64) * bh + ah.astype(np.float64) * bl + al.astype(np.float64) * bh)
    exact = a.astype(np.float64) * b.astype(np.float64)
    rel = np.abs(p3 - exact) / np.abs(exact)
    assert rel.max() <= 3 * 2.0 ** -21


def _gram3(H):
    """Re and Im of H^H H with split operands, products summed in FP32 in K order (real embedding over the
    interleaved (re, im) floats, as the tensor-core kernel does)."""
    nl, nb = H.shape
    A = np.empty((nl, 2 * nb), dtype=np.float32)
    A[:, 0::2], A[:, 1::2] = H.real, H.imag
    R = np.empty_like(A)
    R[:, 0::2], R[:, 1::2] = H.imag, -H.real
    ah, al = split(A)
    rh, rl = split(R)
    f32 = np.float32
    re = np.zeros((nl, nl), dtype=f32)
    im = np.zeros((nl, nl), dtype=f32)
    for k in range(2 * nb):
        re = (re + (np.outer(al[:, k], ah[:, k]) + np.outer(ah[:, k], al[:, k])).astype(f32)).astype(f32)
        re = (re + np.outer(ah[:, k], ah[:, k]).astype(f32)).astype(f32)
        im = (im + (np.outer(al[:, k], rh[:, k]) + np.outer(ah[:, k], rl[:, k])).astype(f32)).astype(f32)
        im = (im + np.outer(ah[:, k], rh[:, k]).astype(f32)).astype(f32)
    return re.astype(np.float64) + 1j * im.astype(np.float64)


@pytest.mark.parametrize("nl,nb", [(16, 32), (32, 64)])
def test_split_gram_is_as_accurate_as_an_fp32_gram(nl, nb):
    rng = np.random.default_rng(nl + nb)
    H = ((rng.standard_normal((nl, nb)) + 1j * rng.standard_normal((nl, nb))) / np.sqrt(2)).astype(np.complex64)
    H64 = H.astype(np.complex128)
    exact = H64.conj() @ H64.T
    scale = np.linalg.norm(exact)
    e3 = np.linalg.norm(_gram3(H) - exact) / scale
    Hf = H.astype(np.complex64)
    f32 = (Hf.conj() @ Hf.T).astype(np.complex128)             # plain FP32 arithmetic
    ef = np.linalg.norm(f32 - exact) / scale
    A = np.concatenate([H.real, H.imag], axis=1).astype(np.float32)
    one = tf32_hi(A).astype(np.float64)
    e1 = np.linalg.norm(one @ one.T - exact.real) / np.linalg.norm(exact.real)   # one TF32 product per term
    assert e3 <= 4 * max(ef, 2.0 ** -24)
    assert e3 <= 2.0 ** -19
    assert e1 > 30 * e3
