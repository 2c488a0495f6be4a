"""Pins of the oracle's noise-variance estimate (Section II, the NE step): a hand-computed case, zero for a
noiseless static channel, unbiased on a large noisy draw (this fixes the factor 2 that undoes the two-symbol
average), and invariant to a common pilot phase."""
import numpy as np
import pytest

RNG = np.random.default_rng(123)


def test_hand_computed_case(orc):
    """1 beam, 1 layer, comb 1, 2 subcarriers, pilots 1 on both DMRS symbols (2 and 11).
    Subcarrier 0: y = 1+2i and 3 -> LS = 2+i, residuals -1+i and 1-i (|.|^2 = 2, 2).
    Subcarrier 1: y = 2i and 0 -> LS = i, residuals i and -i (|.|^2 = 1, 1).
    sigma2_hat = 2 * (2 + 2 + 1 + 1) / 4 = 3."""
    beam = np.zeros((14, 2, 1), complex)
    beam[2, 0, 0], beam[11, 0, 0] = 1 + 2j, 3
    beam[2, 1, 0], beam[11, 1, 0] = 2j, 0
    pil = np.ones((1, 2, 2), complex)
    assert orc.noise_est(beam, pil, [0], 1) == 3.0


def _static_slot(n_sc=240, B=8, L=4, comb=4):
    H = (RNG.standard_normal((n_sc, L, B)) + 1j * RNG.standard_normal((n_sc, L, B))) / np.sqrt(2)
    p = np.exp(2j * np.pi * RNG.integers(0, 4, (L, 2, n_sc)) / 4 + 1j * np.pi / 4)
    a = np.arange(n_sc)
    p = p * ((a[None, :] % comb) == np.arange(L)[:, None])[:, None, :]
    beam = np.zeros((14, n_sc, B), complex)
    for j, s in enumerate((2, 11)):
        beam[s] = np.einsum("alb,la->ab", H, p[:, j, :])
    return beam, p, list(range(L)), comb


def test_noiseless_static_channel_gives_zero(orc):
    beam, p, ports, comb = _static_slot()
    assert orc.noise_est(beam, p, ports, comb) < 1e-28


def test_unbiased_on_a_large_draw(orc):
    beam, p, ports, comb = _static_slot(n_sc=3000, B=16)
    sigma2 = 0.037
    for s in (2, 11):
        beam[s] += (RNG.standard_normal(beam[s].shape) + 1j * RNG.standard_normal(beam[s].shape)) * np.sqrt(sigma2 / 2)
    est = orc.noise_est(beam, p, ports, comb)
    # 96,000 residual samples: relative standard deviation about 0.5 %
    assert est == pytest.approx(sigma2, rel=0.03)


def test_common_pilot_phase_does_not_matter(orc):
    beam, p, ports, comb = _static_slot()
    beam[2] += 0.1 * RNG.standard_normal(beam[2].shape)
    e0 = orc.noise_est(beam, p, ports, comb)
    rot = np.exp(0.7j)
    beam2 = beam.copy()
    beam2[[2, 11]] *= rot
    assert orc.noise_est(beam2, p * rot, ports, comb) == pytest.approx(e0, rel=1e-12)
