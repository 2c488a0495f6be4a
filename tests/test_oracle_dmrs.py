"""Pins of the oracle's 3GPP type-1 DMRS (TS 38.211 5.2.1, 6.4.1.1; an extension beyond the paper's block
pilots): the Gold sequence against an independent jump-ahead computation (the two LFSRs as 31x31 matrices over
GF(2), raised to the 1600-step offset by repeated squaring), c_init against hand-worked values, the pilot
mapping's structure (CDM groups, OCC signs, QPSK from c(2m), c(2m+1)), and the OCC-despread LS estimate against
closed forms: exact per port on a flat channel with both ports of a group, exact interpolation on a channel
linear in frequency with one port per group, and the known leakage -slope of the other port otherwise."""
import numpy as np
import pytest

RNG = np.random.default_rng(1000)


def companion(taps):
    """State s = (x(n), ..., x(n+30)) -> (x(n+1), ..., x(n+31)) with x(n+31) = xor of x(n+t), t in taps."""
    A = np.zeros((31, 31), dtype=np.int64)
    for i in range(30):
        A[i, i + 1] = 1
    for t in taps:
        A[30, t] = 1
    return A


def matpow2(A, e):
    R = np.eye(31, dtype=np.int64)
    while e:
        if e & 1:
            R = (R @ A) % 2
        A = (A @ A) % 2
        e >>= 1
    return R


def gold_by_jump(c_init, n):
    A1, A2 = companion([0, 3]), companion([0, 1, 2, 3])
    s1 = np.zeros(31, dtype=np.int64)
    s1[0] = 1
    s2 = np.array([(c_init >> i) & 1 for i in range(31)], dtype=np.int64)
    s1 = matpow2(A1, 1600) @ s1 % 2
    s2 = matpow2(A2, 1600) @ s2 % 2
    out = []
    for _ in range(n):
        out.append(int(s1[0] ^ s2[0]))
        s1, s2 = A1 @ s1 % 2, A2 @ s2 % 2
    return np.array(out, dtype=np.uint8)


@pytest.mark.parametrize("c_init", [0, 1, 393216, 0x7FFFFFFF, int(RNG.integers(0, 2**31))])
def test_gold_sequence_equals_jump_ahead(orc, c_init):
    n = 200
    assert np.array_equal(orc.gold(c_init, n), gold_by_jump(c_init, n))


def test_gold_sequences_differ_and_are_balanced(orc):
    a, b = orc.gold(1, 4000), orc.gold(2, 4000)
    assert np.mean(a != b) > 0.4
    assert 0.45 < a.mean() < 0.55 and 0.45 < b.mean() < 0.55


def test_cinit_hand_values(orc):
    assert orc.dmrs_cinit(0, 0, 0, 2) == 2**17 * 3
    assert orc.dmrs_cinit(1, 1, 3, 11) == 2**17 * (42 + 11 + 1) * 3 + 2 + 1
    big = (2**17 * (14 * 19 + 13 + 1) * (2 * 65535 + 1) + 2 * 65535) % 2**31
    assert orc.dmrs_cinit(65535, 0, 19, 13) == big


def test_pilot_mapping_structure(orc):
    n_sc = 48
    P = orc.dmrs_type1_pilots(7, 0, 5, [0, 1, 2, 3], n_sc)
    k = np.arange(n_sc)
    for j, sym in enumerate((2, 11)):
        c = orc.gold(orc.dmrs_cinit(7, 0, 5, sym), n_sc + 2)
        for p in range(4):
            delta = p // 2
            on = (k % 2) == delta
            assert np.all(P[p, j, ~on] == 0)
            assert np.allclose(np.abs(P[p, j, on]), 1.0, atol=1e-15)
            m = (k[on] - delta) // 2                       # k = 4n + 2k' + Delta -> m = 2n + k'
            r = ((1 - 2.0 * c[2 * m]) + 1j * (1 - 2.0 * c[2 * m + 1])) / np.sqrt(2)
            w = np.where((p % 2 == 1) & (m % 2 == 1), -1.0, 1.0)
            assert np.allclose(P[p, j, on], w * r, atol=1e-15)
        # ports 0/1 share the even subcarriers: equal on k' = 0, opposite on k' = 1
        assert np.allclose(P[0, j, 0::4], P[1, j, 0::4]) and np.allclose(P[0, j, 2::4], -P[1, j, 2::4])


def _beams(H_of_k, P, n_sc, B):
    """Noiseless DMRS symbols: beam[s][k][b] = sum_l H_l(k)[b] P[l][j][k] on the DMRS symbols."""
    beam = np.zeros((14, n_sc, B), complex)
    for j, sym in enumerate((2, 11)):
        for k in range(n_sc):
            beam[sym, k] = sum(H_of_k(k)[l] * P[l, j, k] for l in range(P.shape[0]))
    return beam


def test_ls_exact_per_port_on_flat_channel(orc):
    n_sc, B = 48, 3
    P = orc.dmrs_type1_pilots(3, 1, 2, [0, 1, 2, 3], n_sc)
    Hc = RNG.standard_normal((4, B)) + 1j * RNG.standard_normal((4, B))
    H = orc.chest_ls_type1(_beams(lambda k: Hc, P, n_sc, B), P, [0, 1, 2, 3])
    assert np.allclose(H, np.broadcast_to(Hc, (n_sc, 4, B)), atol=1e-13)


def test_ls_interpolates_a_linear_channel_exactly_with_one_port_per_group(orc):
    n_sc, B = 60, 2
    P = orc.dmrs_type1_pilots(11, 0, 7, [0, 2], n_sc)
    A = RNG.standard_normal((2, B)) + 1j * RNG.standard_normal((2, B))
    S = 0.01 * (RNG.standard_normal((2, B)) + 1j * RNG.standard_normal((2, B)))
    H = orc.chest_ls_type1(_beams(lambda k: A + k * S, P, n_sc, B), P, [0, 2])
    for l, delta in ((0, 0), (1, 1)):
        first, last = delta + 1, 4 * ((n_sc - delta - 2) // 4) + delta + 1
        for a in range(n_sc):
            c = min(max(a, first), last)                  # held outside the first and last pair centre
            assert np.allclose(H[a, l], A[l] + c * S[l], atol=1e-12)


def test_ls_leakage_of_the_other_port_in_a_group(orc):
    """Ports 0 and 1 on a channel linear in frequency: at a pair centre the despread estimate of port 0 is
    h0(centre) + (h1(k0) - h1(k1)) / 2 = h0(centre) - slope1 (w_f = (+1, -1) for port 1)."""
    n_sc, B = 40, 2
    P = orc.dmrs_type1_pilots(0, 0, 0, [0, 1], n_sc)
    A = RNG.standard_normal((2, B)) + 1j * RNG.standard_normal((2, B))
    S = 0.02 * (RNG.standard_normal((2, B)) + 1j * RNG.standard_normal((2, B)))
    H = orc.chest_ls_type1(_beams(lambda k: A + k * S, P, n_sc, B), P, [0, 1])
    for n in range(1, 8):
        c = 4 * n + 1
        assert np.allclose(H[c, 0], A[0] + c * S[0] - S[1], atol=1e-12)
        assert np.allclose(H[c, 1], A[1] + c * S[1] - S[0], atol=1e-12)


def test_single_symbol_estimates_average_to_the_mean(orc):
    n_sc, B = 48, 2
    P = orc.dmrs_type1_pilots(1, 0, 4, [0, 1, 3], n_sc)
    beam = RNG.standard_normal((14, n_sc, B)) + 1j * RNG.standard_normal((14, n_sc, B))
    h0 = orc.chest_ls_type1_sym(beam, P, [0, 1, 3], 0)
    h1 = orc.chest_ls_type1_sym(beam, P, [0, 1, 3], 1)
    assert np.allclose(0.5 * (h0 + h1), orc.chest_ls_type1(beam, P, [0, 1, 3]), atol=1e-13)


def test_generator_transmits_the_same_pilots(orc):
    """The signal generator's own copy of the definition (the transmitter) agrees with the oracle exactly."""
    from paper_2210_09196_gb300 import synth
    for n_id, n_scid, slot in ((0, 0, 0), (517, 1, 13), (65535, 0, 19)):
        assert np.array_equal(synth.dmrs_type1(n_id, n_scid, slot, [0, 1, 2, 3], 132),
                              orc.dmrs_type1_pilots(n_id, n_scid, slot, [0, 1, 2, 3], 132))


@pytest.mark.parametrize("ports", [[0, 1, 2, 3], [0], [0, 2], [0, 1, 3]])
def test_noise_estimate_type1_zero_and_unbiased(orc, ports):
    """Zero on a noiseless channel that is flat over each CDM pair; for white noise of variance s2 the
    degrees-of-freedom normalisation (4 - m per pair, beam and group with m ports) makes the mean estimate s2
    whatever the number of ports per group."""
    n_sc, B = 48, 8
    P = orc.dmrs_type1_pilots(5, 0, 3, ports, n_sc)
    Hc = RNG.standard_normal((len(ports), B)) + 1j * RNG.standard_normal((len(ports), B))
    clean = _beams(lambda k: Hc, P, n_sc, B)
    assert orc.noise_est_type1(clean, P, ports) < 1e-25
    s2 = 0.037
    est = []
    for _ in range(150):
        n = np.sqrt(s2 / 2) * (RNG.standard_normal(clean.shape) + 1j * RNG.standard_normal(clean.shape))
        est.append(orc.noise_est_type1(clean + n, P, ports))
    assert np.mean(est) == pytest.approx(s2, rel=0.02)


def test_noise_estimate_type1_phase_invariant(orc):
    n_sc, B = 48, 4
    P = orc.dmrs_type1_pilots(2, 1, 9, [0, 1, 2], n_sc)
    beam = RNG.standard_normal((14, n_sc, B)) + 1j * RNG.standard_normal((14, n_sc, B))
    a = orc.noise_est_type1(beam, P, [0, 1, 2])
    assert orc.noise_est_type1(beam * np.exp(0.7j), P, [0, 1, 2]) == pytest.approx(a, rel=1e-12)
