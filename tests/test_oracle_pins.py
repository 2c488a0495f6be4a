"""Pins of the FP64 oracle against things other than itself: closed forms, invariants, hand-worked
examples (tests/golden), brute force on tiny inputs and special cases that reduce to library routines.

Each group is chosen so that a plausible slip in the oracle (a sign, a conjugate, a transposed operand, a
dropped term, an off-by-one in the bin map or the interpolation) fails at least one test here.
"""
from pathlib import Path

import numpy as np
import pytest

from paper_2210_09196_gb300 import synth

GOLDEN = Path(__file__).parent / "golden"
RNG = np.random.default_rng(1234)


def crandn(*shape, rng=RNG):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)


def rel(a, b):
    return np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300)


def _golden(name):
    vals = {}
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        vals[k] = np.array([float(t) for t in v])
    return vals


def _cplx(v, shape):
    return (v[0::2] + 1j * v[1::2]).reshape(shape)


# ------------------------------------------------------------------------------------------------ DFT / FFT


@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 12, 16])
def test_dft_closed_forms(orc, n):
    # delta at n0 -> exp(-2 pi i k n0 / N)
    for n0 in range(n):
        x = np.zeros(n, complex)
        x[n0] = 1
        k = np.arange(n)
        assert np.allclose(orc.dft(x), np.exp(-2j * np.pi * k * n0 / n), atol=1e-13)
    # exp(+2 pi i k0 n / N) -> N * delta[k - k0]
    for k0 in range(n):
        t = np.arange(n)
        X = orc.dft(np.exp(2j * np.pi * k0 * t / n))
        want = np.zeros(n, complex)
        want[k0] = n
        assert np.allclose(X, want, atol=1e-12)


@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
def test_fft_matches_dft(orc, n):
    x = crandn(n)
    assert rel(orc.fft(x), orc.dft(x)) < 1e-12


@pytest.mark.parametrize("n", [512, 2048, 4096])
def test_fft_matches_library_and_invariants(orc, n):
    x = crandn(n)
    X = orc.fft(x)
    assert rel(X, np.fft.fft(x)) < 1e-12                               # library special case
    assert abs(np.sum(abs(X) ** 2) - n * np.sum(abs(x) ** 2)) < 1e-9 * n * np.sum(abs(x) ** 2)  # Parseval
    assert rel(orc.fft(np.fft.ifft(X)), X) < 1e-12                     # IFFT round trip
    y = crandn(n)
    assert rel(orc.fft(2 * x - 3j * y), 2 * X - 3j * orc.fft(y)) < 1e-12  # linearity


def test_fft_rejects_non_power_of_two(orc):
    with pytest.raises(ValueError):
        orc.fft(np.ones(12))


@pytest.mark.parametrize("n_fft,n_sc", [(64, 36), (512, 300), (4096, 3276)])
def test_ofdm_demod_single_tone_lands_on_its_subcarrier(orc, n_fft, n_sc):
    # A tone at FFT bin (a - n_sc//2) mod N_F must appear, with amplitude N_F, at active index a only.
    for a in (0, 1, n_sc // 2 - 1, n_sc // 2, n_sc // 2 + 1, n_sc - 1):
        b = (a - n_sc // 2) % n_fft
        t = np.exp(2j * np.pi * b * np.arange(n_fft) / n_fft)
        freq = orc.ofdm_demod(t[None, None, :], n_sc)[0, 0]
        want = np.zeros(n_sc, complex)
        want[a] = n_fft
        assert np.allclose(freq, want, atol=1e-9 * n_fft)


def test_ofdm_demod_inverts_the_generator(orc):
    cfg = synth.SMALL_FP32
    s = synth.make_slot(cfg)
    freq = orc.ofdm_demod(s.time_as_complex128(), cfg.n_sc)
    # The generator places X on the active bins and applies ifft; numpy's fft recovers exactly that.
    spec = np.fft.fft(s.time_as_complex128(), axis=-1)[..., synth.active_bins(cfg.n_sc, cfg.n_fft)]
    assert rel(freq, spec) < 1e-12
    # and the pairs subset writes only the requested rows
    sub = orc.ofdm_demod(s.time_as_complex128(), cfg.n_sc, pairs=[(3, 5), (13, 0)])
    assert np.allclose(sub[3, 5], freq[3, 5]) and np.allclose(sub[13, 0], freq[13, 0])
    assert np.count_nonzero(np.abs(sub).sum(-1)) == 2


# --------------------------------------------------------------------------------------------- beamforming


def test_beamform_identity(orc):
    freq = crandn(3, 8, 20)
    beam = orc.beamform(freq, np.eye(8))
    assert np.array_equal(beam, np.transpose(freq, (0, 2, 1)))


def test_beamform_plane_wave_closed_form(orc):
    # DFT beams: a plane wave exp(-2 pi i r b0 / N_R) puts sqrt(N_R) into beam b0 and nothing elsewhere.
    R, B = 64, 32
    W = np.exp(-2j * np.pi * np.arange(R)[:, None] * np.arange(B)[None, :] / R) / np.sqrt(R)
    for b0 in (0, 5, 31):
        x = np.exp(-2j * np.pi * np.arange(R) * b0 / R)
        freq = np.tile(x[None, :, None], (1, 1, 4))
        beam = orc.beamform(freq, W)
        want = np.zeros(B, complex)
        want[b0] = np.sqrt(R)
        assert np.allclose(beam[0, 2], want, atol=1e-12)


def test_beamform_brute_force(orc):
    freq = crandn(2, 6, 7)
    W = crandn(6, 5)
    beam = orc.beamform(freq, W)
    want = np.zeros((2, 7, 5), complex)
    for s in range(2):
        for a in range(7):
            for b in range(5):
                want[s, a, b] = sum(np.conj(W[r, b]) * freq[s, r, a] for r in range(6))
    assert rel(beam, want) < 1e-14
    assert rel(beam, np.einsum("rb,sra->sab", W.conj(), freq)) < 1e-14


# ------------------------------------------------------------------------------------------------------ LS


def _pilots(L, n_sc, comb, rng):
    p = (rng.choice([-1, 1], (L, 2, n_sc)) + 1j * rng.choice([-1, 1], (L, 2, n_sc))) / np.sqrt(2)
    mask = (np.arange(n_sc)[None, :] % comb) == (np.arange(L) % comb)[:, None]
    return p * mask[:, None, :]


def _rx_dmrs(Hsym, pilots, n_sc, B):
    """beam [14, N_SC, B] with DMRS symbols y = sum_l H_s[a, l, :] p_l,s[a]; Hsym[j] is the channel at DMRS j."""
    beam = np.zeros((14, n_sc, B), complex)
    for j, s in enumerate((2, 11)):
        beam[s] = np.einsum("alb,la->ab", Hsym[j], pilots[:, j, :])
    return beam


def test_ls_flat_channel_is_exact(orc):
    L, B, n_sc = 4, 8, 40
    rng = np.random.default_rng(5)
    H = np.broadcast_to(crandn(1, L, B, rng=rng), (n_sc, L, B))
    pil = _pilots(L, n_sc, L, rng)
    Hh = orc.chest_ls(_rx_dmrs([H, H], pil, n_sc, B), pil, np.arange(L), L)
    assert rel(Hh, H) < 1e-14


def test_ls_linear_channel_interpolates_exactly_and_holds_at_edges(orc):
    L, B, n_sc, comb = 3, 4, 50, 3
    rng = np.random.default_rng(6)
    c0, c1 = crandn(L, B, rng=rng), crandn(L, B, rng=rng)
    a = np.arange(n_sc)[:, None, None]
    H = c0[None] + a * c1[None] * 0.01                                  # linear in a
    pil = _pilots(L, n_sc, comb, rng)
    Hh = orc.chest_ls(_rx_dmrs([H, H], pil, n_sc, B), pil, np.arange(L), comb)
    for l in range(L):
        pos = np.arange(l, n_sc, comb)
        first, last = pos[0], pos[-1]
        inner = np.arange(first, last + 1)
        assert rel(Hh[inner, l], H[inner, l]) < 1e-13
        for e in range(0, first):
            assert np.allclose(Hh[e, l], H[first, l], atol=1e-13)
        for e in range(last + 1, n_sc):
            assert np.allclose(Hh[e, l], H[last, l], atol=1e-13)


def test_ls_averages_the_two_dmrs_symbols(orc):
    L, B, n_sc = 1, 2, 10
    rng = np.random.default_rng(7)
    H0, H1 = crandn(n_sc, L, B, rng=rng), crandn(n_sc, L, B, rng=rng)
    pil = _pilots(L, n_sc, 1, rng)
    Hh = orc.chest_ls(_rx_dmrs([H0, H1], pil, n_sc, B), pil, [0], 1)
    assert rel(Hh, (H0 + H1) / 2) < 1e-14


def test_ls_respects_allocation_range(orc):
    L, B, n_sc, comb = 2, 2, 30, 2
    rng = np.random.default_rng(8)
    H = np.broadcast_to(crandn(1, L, B, rng=rng), (n_sc, L, B))
    pil = _pilots(L, n_sc, comb, rng)
    Hh = orc.chest_ls(_rx_dmrs([H, H], pil, n_sc, B), pil, [0, 1], comb, sc_start=[4, 10], sc_count=[7, 3])
    assert np.all(Hh[:4, 0] == 0) and np.all(Hh[11:, 0] == 0)
    assert rel(Hh[4:11, 0], H[4:11, 0]) < 1e-14
    assert rel(Hh[10:13, 1], H[10:13, 1]) < 1e-14
    with pytest.raises(ValueError):
        orc.chest_ls(_rx_dmrs([H, H], pil, n_sc, B), pil, [0, 1], comb, sc_start=[4, 10], sc_count=[7, 1])


# ------------------------------------------------------------------------------------- Gram and Cholesky


def test_golden_2x2(orc):
    g = _golden("mmse_2x2.txt")
    H = _cplx(g["H"], (2, 2))
    y = _cplx(g["y"], (2,))
    s2 = float(g["sigma2"][0])
    Hs = H.T.copy()                                                    # stored [N_L][N_B]
    G = orc.gram(Hs, s2)
    assert np.allclose(G, _cplx(g["G"], (2, 2)), atol=1e-15)
    Lf, st = orc.cholesky(G)
    assert st == 0 and np.allclose(Lf, _cplx(g["L"], (2, 2)), atol=1e-15)
    r = H.conj().T @ y
    assert np.allclose(orc.chol_solve(Lf, r), _cplx(g["x"], (2,)), atol=1e-15)
    beam = np.zeros((3, 1, 2), complex)
    beam[0, 0] = y
    xh, fails = orc.mmse(Hs[None], beam, s2, data_sym=[0])
    assert fails == 0 and np.allclose(xh[:, 0, 0], _cplx(g["x"], (2,)), atol=1e-15)


@pytest.mark.parametrize("n", [1, 2, 4, 16, 32])
def test_cholesky_reconstruction_and_shape(orc, n):
    A = crandn(2 * n + 3, n)
    G = A.conj().T @ A + 0.1 * np.eye(n)
    Lf, st = orc.cholesky(G)
    assert st == 0
    assert rel(Lf @ Lf.conj().T, G) < 1e-13
    assert np.all(np.triu(Lf, 1) == 0)
    d = np.diag(Lf)
    assert np.all(d.imag == 0) and np.all(d.real > 0)
    assert rel(Lf, np.linalg.cholesky(G)) < 1e-12                     # textbook/library special case


def test_cholesky_reads_only_lower_triangle(orc):
    A = crandn(9, 4)
    G = A.conj().T @ A + np.eye(4)
    G2 = G.copy()
    G2[np.triu_indices(4, 1)] = 99 + 7j
    assert np.array_equal(orc.cholesky(G)[0], orc.cholesky(G2)[0])


def test_cholesky_flags_bad_pivot(orc):
    G = np.array([[1, 2], [2, 1]], complex)                            # indefinite: pivot 2 is 1 - 4 < 0
    assert orc.cholesky(G)[1] == 2
    assert orc.cholesky(np.zeros((3, 3), complex))[1] == 1
    G = np.eye(3, dtype=complex)
    G[1, 1] = np.nan
    assert orc.cholesky(G)[1] == 2


def test_gram_definition(orc):
    Hs = crandn(3, 5)
    G = orc.gram(Hs, 0.25)
    H = Hs.T
    assert rel(G, H.conj().T @ H + 0.25 * np.eye(3)) < 1e-15
    assert np.allclose(G, G.conj().T)


# --------------------------------------------------------------------------------------------------- MMSE


def test_mmse_matches_explicit_inverse(orc):
    n_sc, L, B = 6, 3, 5
    Hs = crandn(n_sc, L, B)
    beam = crandn(14, n_sc, B)
    s2 = 0.3
    xh, fails = orc.mmse(Hs, beam, s2)
    assert fails == 0
    ds = orc.data_symbols()
    for a in range(n_sc):
        H = Hs[a].T
        Ginv = np.linalg.inv(H.conj().T @ H + s2 * np.eye(L))
        for d, s in enumerate(ds):
            assert rel(xh[:, d, a], Ginv @ H.conj().T @ beam[s, a]) < 1e-12


def test_mmse_closed_form_2x2_random(orc):
    rng = np.random.default_rng(9)
    for _ in range(20):
        H = crandn(4, 2, rng=rng)
        y = crandn(4, rng=rng)
        s2 = rng.uniform(0.01, 2)
        G = H.conj().T @ H + s2 * np.eye(2)
        a, b, d = G[0, 0], G[0, 1], G[1, 1]
        Ginv = np.array([[d, -b], [-np.conj(b), a]]) / (a * d - abs(b) ** 2)
        beam = np.zeros((1, 1, 4), complex)
        beam[0, 0] = y
        xh, _ = orc.mmse(H.T[None], beam, s2, data_sym=[0])
        assert rel(xh[:, 0, 0], Ginv @ H.conj().T @ y) < 1e-13


def test_mmse_noiseless_full_rank_recovers_symbols(orc):
    n_sc, L, B = 20, 4, 8
    Hs = crandn(n_sc, L, B)
    bits = RNG.integers(0, 2, (L, 12, n_sc, 4))
    x = synth.qam_map(bits, 4)
    beam = np.zeros((14, n_sc, B), complex)
    for d, s in enumerate(orc.data_symbols()):
        beam[s] = np.einsum("alb,la->ab", Hs, x[:, d, :])
    xh, fails = orc.mmse(Hs, beam, 0.0)
    assert fails == 0 and rel(xh, x) < 1e-12
    assert np.array_equal(orc.demap(xh, 4), synth.pack_bits(bits))


def test_mmse_sc_list_and_failure_count(orc):
    n_sc, L, B = 5, 2, 3
    Hs = crandn(n_sc, L, B)
    Hs[3] = 0                                                          # zero channel, sigma^2 = 0 -> singular
    beam = crandn(14, n_sc, B)
    xh, fails = orc.mmse(Hs, beam, 0.0, sc_list=[1, 3])
    assert fails == 12                                                 # every data symbol of subcarrier 3
    assert np.all(xh[:, :, 3] == 0) and np.all(xh[:, :, [0, 2, 4]] == 0) and np.any(xh[:, :, 1] != 0)


# ------------------------------------------------------------------------------------------------ demapper


@pytest.mark.parametrize("q", [2, 4])
def test_demap_inverts_gray_map(orc, q):
    bits = np.array(np.meshgrid(*[[0, 1]] * q, indexing="ij")).reshape(q, -1).T
    x = synth.qam_map(bits, q)
    assert np.array_equal(orc.demap(x, q), synth.pack_bits(bits))
    assert np.array_equal(orc.demap(x * 1.2 + 0.05 * (1 + 1j), q), synth.pack_bits(bits))


def test_demap_ties_go_to_bit_zero(orc):
    t = 2 / np.sqrt(10)
    x = np.array([0 + 0j, t + 1j * t, -t - 1j * t])
    assert list(orc.demap(x, 4)) == [0b0000, 0b0000, 0b0011]
    tf = float(np.float32(t))
    assert list(orc.demap(np.array([tf + 1j * tf]), 4, f32=True)) == [0]
    assert list(orc.demap(np.array([float(np.nextafter(np.float32(tf), np.float32(1))) + 0j]), 4, f32=True)) == [0b0100]


# ------------------------------------------------------------------------------------------ Table I model


def test_table1_counts_match_hand_worked_use_case(orc):
    g = _golden("table1_usecase_counts.txt")
    c = orc.op_counts(14, 2, 64, 4096, 32, 4)
    for k in ("ofdm", "bf", "mimo", "che", "ne"):
        assert c[k] == pytest.approx(float(g[k][0]), rel=1e-12)


# ------------------------------------------------------------------------------------------ whole chain


@pytest.mark.parametrize("q", [2, 4])
def test_slot_noiseless_flat_channel_recovers_bits(orc, q):
    cfg = synth.SMALL_FP32.with_(channel="flat", snr_db=300.0, qam_bits=q, n_beams=16)
    s = synth.make_slot(cfg, 0)
    xh, bits, fails = orc.run_slot(s)
    assert fails == 0
    assert rel(xh, s.x) < 1e-5                                         # complex64 input rounding only
    assert np.array_equal(bits, s.bits)


def test_slot_chain_equals_composition_of_stages(orc):
    cfg = synth.SMALL_FP32.with_(n_rx=8, n_beams=8, n_fft=64, n_sc=36, n_layers=2)
    s = synth.make_slot(cfg, 3)
    xh, bits, _ = orc.run_slot(s)
    freq = orc.ofdm_demod(s.time_as_complex128(), cfg.n_sc)
    beam = orc.beamform(freq, s.W)
    H = orc.chest_ls(beam, s.pilots, s.ports, cfg.comb)
    xh2, _ = orc.mmse(H, beam, s.noise_var)
    assert np.array_equal(xh, xh2)
    assert np.array_equal(bits, orc.demap(xh2, cfg.qam_bits))


def test_slot_deploy_pdp_decodes_well_at_30db(orc):
    """Sanity of the whole model at the deployment size: the oracle decodes a 30 dB PDP slot with a low
    bit-error rate vs the transmitted bits (LS + linear interpolation is the limiting error)."""
    s = synth.make_slot(synth.DEPLOY, 0)
    _, bits, fails = orc.run_slot(s)
    assert fails == 0
    assert np.mean(bits != s.bits) < 0.02


# ------------------------------------------------------------------------------------------ MU-MIMO


def test_mmse_active_all_layers_equals_plain_mmse(orc):
    n_sc, L, B = 6, 3, 5
    H, beam = crandn(n_sc, L, B), crandn(14, n_sc, B)
    x1, _ = orc.mmse_active(H, beam, np.ones((n_sc, L), bool), 0.3)
    x2, _ = orc.mmse(H, beam, 0.3)
    assert np.array_equal(x1, x2)


def test_mmse_active_detects_only_the_layers_present(orc):
    """A layer absent at a subcarrier neither receives an output nor enters the Gram there (Eq. 2 over the
    users that share the subcarrier)."""
    n_sc, L, B = 5, 4, 6
    H, beam = crandn(n_sc, L, B), crandn(14, n_sc, B)
    act = np.ones((n_sc, L), bool)
    act[1, 2] = act[3, 0] = act[3, 3] = False
    x, _ = orc.mmse_active(H, beam, act, 0.2)
    for a in range(n_sc):
        keep = np.flatnonzero(act[a])
        xr, _ = orc.mmse(H[a:a + 1][:, keep], beam[:, a:a + 1], 0.2)
        assert rel(x[keep][:, :, a], xr[:, :, 0]) < 1e-14
        assert np.all(x[~act[a]][:, :, a] == 0)
