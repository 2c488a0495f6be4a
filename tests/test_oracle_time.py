"""Pins of the oracle's time-varying estimate and per-group factorisation (Section VI's schedule: one Cholesky
per data symbol, or every K data symbols): the K = 12 case reduces to the two-symbol-average chain, a noiseless
channel that varies linearly in time is recovered exactly per data symbol, K = 1 equals an explicit-inverse
brute force, and the single-symbol estimates are exact on a flat channel and average to the plain estimate."""
import numpy as np
import pytest

RNG = np.random.default_rng(2024)
DMRS = (2, 11)
DATA = [s for s in range(14) if s not in DMRS]


def _qpsk(shape):
    return (RNG.choice([-1, 1], shape) + 1j * RNG.choice([-1, 1], shape)) / np.sqrt(2)


def _slot(n_sc=24, L=2, B=4, comb=2, Hfun=None, noise=0.0):
    """beam [14, n_sc, B], pilots [L, 2, n_sc], x [L, 12, n_sc] for per-symbol channels Hfun(s) -> [n_sc, L, B]."""
    a = np.arange(n_sc)
    pil = _qpsk((L, 2, n_sc)) * ((a[None, :] % comb) == np.arange(L)[:, None])[:, None, :]
    x = _qpsk((L, 12, n_sc))
    beam = np.zeros((14, n_sc, B), complex)
    for s in range(14):
        Hs = Hfun(s)
        v = pil[:, DMRS.index(s), :] if s in DMRS else x[:, DATA.index(s), :]
        beam[s] = np.einsum("alb,la->ab", Hs, v)
    if noise:
        beam += noise * (RNG.standard_normal(beam.shape) + 1j * RNG.standard_normal(beam.shape))
    return beam, pil, x, list(range(L)), comb


def test_single_symbol_estimates_exact_on_flat_channel_and_average_to_plain(orc):
    Hc = RNG.standard_normal((1, 2, 4)) + 1j * RNG.standard_normal((1, 2, 4))
    beam, pil, _, ports, comb = _slot(Hfun=lambda s: np.repeat(Hc, 24, axis=0), noise=0.0)
    H0 = orc.chest_ls_sym(beam, pil, ports, comb, 0)
    H1 = orc.chest_ls_sym(beam, pil, ports, comb, 1)
    assert np.allclose(H0, np.repeat(Hc, 24, axis=0), atol=1e-13) and np.allclose(H1, H0, atol=1e-13)
    beam_n, pil_n, _, _, _ = _slot(Hfun=lambda s: np.repeat(Hc, 24, axis=0), noise=0.1)
    avg = orc.chest_ls(beam_n, pil_n, ports, comb)
    h0 = orc.chest_ls_sym(beam_n, pil_n, ports, comb, 0)
    h1 = orc.chest_ls_sym(beam_n, pil_n, ports, comb, 1)
    assert np.allclose(0.5 * (h0 + h1), avg, atol=1e-13)


def test_k12_reduces_to_the_average_chain(orc):
    """The 12 data symbols' mean time is the DMRS midpoint, so one group uses (H0 + H1) / 2."""
    Hc = RNG.standard_normal((24, 2, 4)) + 1j * RNG.standard_normal((24, 2, 4))
    beam, pil, _, ports, comb = _slot(Hfun=lambda s: Hc, noise=0.05)
    H0 = orc.chest_ls_sym(beam, pil, ports, comb, 0)
    H1 = orc.chest_ls_sym(beam, pil, ports, comb, 1)
    xt, f1 = orc.mmse_tv(H0, H1, beam, 0.01, 12)
    xa, f2 = orc.mmse(orc.chest_ls(beam, pil, ports, comb), beam, 0.01)
    assert f1 == f2 == 0
    assert np.allclose(xt, xa, rtol=0, atol=1e-12)


def test_linear_time_variation_recovered_exactly_per_symbol(orc):
    """H(s) = A + s Bt, flat in frequency, no noise: each data symbol's interpolated estimate is exact, so
    K = 1 returns the transmitted symbols; one averaged estimate (K = 12) does not."""
    A = RNG.standard_normal((1, 2, 4)) + 1j * RNG.standard_normal((1, 2, 4))
    Bt = 0.05 * (RNG.standard_normal((1, 2, 4)) + 1j * RNG.standard_normal((1, 2, 4)))
    beam, pil, x, ports, comb = _slot(Hfun=lambda s: np.repeat(A + s * Bt, 24, axis=0))
    H0 = orc.chest_ls_sym(beam, pil, ports, comb, 0)
    H1 = orc.chest_ls_sym(beam, pil, ports, comb, 1)
    x1, f = orc.mmse_tv(H0, H1, beam, 0.0, 1)
    assert f == 0 and np.max(np.abs(x1 - x)) < 1e-10
    x12, _ = orc.mmse_tv(H0, H1, beam, 0.0, 12)
    assert np.max(np.abs(x12 - x)) > 1e-3
    # groups of 4: symbols inside a group share one estimate, so the error lies between the two
    x4, _ = orc.mmse_tv(H0, H1, beam, 0.0, 4)
    e1, e4, e12 = (np.linalg.norm(v - x) for v in (x1, x4, x12))
    assert e1 < e4 < e12


def test_k1_equals_explicit_inverse_brute_force(orc):
    Hs = {s: RNG.standard_normal((6, 2, 3)) + 1j * RNG.standard_normal((6, 2, 3)) for s in range(14)}
    beam, pil, _, ports, comb = _slot(n_sc=6, B=3, Hfun=lambda s: Hs[s], noise=0.1)
    H0 = orc.chest_ls_sym(beam, pil, ports, comb, 0)
    H1 = orc.chest_ls_sym(beam, pil, ports, comb, 1)
    sig = 0.02
    xk, _ = orc.mmse_tv(H0, H1, beam, sig, 1)
    for di, s in enumerate(DATA):
        t = (s - DMRS[0]) / (DMRS[1] - DMRS[0])
        Ht = H0 + t * (H1 - H0)
        for a in range(6):
            Hm = Ht[a].T                                   # [B, L]
            want = np.linalg.inv(Hm.conj().T @ Hm + sig * np.eye(2)) @ (Hm.conj().T @ beam[s, a])
            assert np.allclose(xk[:, di, a], want, atol=1e-11)
