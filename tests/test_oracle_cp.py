"""Pins of the oracle's cyclic-prefix removal and 7.5 kHz shift (TS 38.211 5.3.1 and 5.4; the receive chain of
the paper starts after them): the CP lengths make a 30 kHz slot last exactly 0.5 ms, a stream built from a known
grid with continuous-phase prefixes is demodulated back to the grid, and a delay shorter than the prefix turns
into the closed-form phase ramp exp(-2 pi i (bin + shift) d / N) on every subcarrier."""
import numpy as np
import pytest

RNG = np.random.default_rng(75)


def test_cp_lengths_make_a_half_millisecond_slot(orc):
    for n_fft in (4096, 2048, 1024, 512, 256, 128):
        fs = n_fft * 30e3                                  # sample rate of the n_fft-point symbol
        assert orc.slot_len(14, n_fft) / fs == pytest.approx(0.5e-3, abs=0)
        assert orc.cp_len(n_fft, 0) - orc.cp_len(n_fft, 1) == 64 * n_fft // 4096   # 16 kappa T_c longer
    assert orc.cp_len(4096, 0) == 352 and orc.cp_len(4096, 5) == 288


def bins(n_sc, n_fft):
    return (np.arange(n_sc) - n_sc // 2) % n_fft


def stream_of(grid, n_fft, shift, delay=0):
    """grid [S, R, n_sc] -> stream [R, slot_len] with continuous-phase prefixes (the transmitted waveform
    sampled at n' = -cp .. N-1 around each useful part), delayed by `delay` samples (zeros shifted in)."""
    S, R, n_sc = grid.shape
    k = bins(n_sc, n_fft)
    fshift = 0.25 if shift else 0.0
    out = []
    for s in range(S):
        cp = 352 * n_fft // 4096 if s == 0 else 288 * n_fft // 4096
        n = np.arange(-cp, n_fft)
        # sum_k X_k exp(2 pi i (k + fshift) n / N) / N
        ph = np.exp(2j * np.pi * np.outer(n, k + fshift) / n_fft) / n_fft       # [cp + N, n_sc]
        out.append(np.einsum("ra,na->rn", grid[s], ph))
    st = np.concatenate(out, axis=1)
    if delay:
        st = np.concatenate([np.zeros((R, delay), complex), st[:, :-delay]], axis=1)
    return st


@pytest.mark.parametrize("shift", [False, True])
def test_round_trip_from_a_known_grid(orc, shift):
    n_fft, n_sc, S, R = 512, 300, 14, 2
    grid = RNG.standard_normal((S, R, n_sc)) + 1j * RNG.standard_normal((S, R, n_sc))
    st = stream_of(grid, n_fft, shift)
    assert st.shape == (R, orc.slot_len(S, n_fft))
    got = orc.ofdm_demod_cp(st, S, n_fft, n_sc, shift=shift)
    assert np.allclose(got, grid, atol=1e-11)
    # the shift is not a no-op: demodulating without undoing it smears every subcarrier
    if shift:
        assert not np.allclose(orc.ofdm_demod_cp(st, S, n_fft, n_sc, shift=False), grid, atol=1e-3)


@pytest.mark.parametrize("shift", [False, True])
def test_delay_inside_the_prefix_is_a_phase_ramp(orc, shift):
    n_fft, n_sc, S, R = 256, 200, 14, 1
    d = 13                                                # < 288 * 256 / 4096 = 18 samples
    grid = RNG.standard_normal((S, R, n_sc)) + 1j * RNG.standard_normal((S, R, n_sc))
    got = orc.ofdm_demod_cp(stream_of(grid, n_fft, shift, delay=d), S, n_fft, n_sc, shift=shift)
    f = bins(n_sc, n_fft) + (0.25 if shift else 0.0)
    want = grid * np.exp(-2j * np.pi * f * d / n_fft)
    assert np.allclose(got[1:], want[1:], atol=1e-10)     # symbol 0: the delay reaches before the slot


def test_plain_copy_prefix_without_shift(orc):
    """Without the shift the prefix is a copy of the last cp samples of the IFFT output (the textbook form)."""
    n_fft, n_sc, S, R = 1024, 600, 14, 3
    grid = RNG.standard_normal((S, R, n_sc)) + 1j * RNG.standard_normal((S, R, n_sc))
    spec = np.zeros((S, R, n_fft), complex)
    spec[:, :, bins(n_sc, n_fft)] = grid
    t = np.fft.ifft(spec, axis=-1)
    parts = [np.concatenate([t[s][:, n_fft - orc.cp_len(n_fft, s):], t[s]], axis=1) for s in range(S)]
    got = orc.ofdm_demod_cp(np.concatenate(parts, axis=1), S, n_fft, n_sc)
    assert np.allclose(got, grid, atol=1e-11)


@pytest.mark.parametrize("shift", [False, True])
def test_generator_waveform_demodulates_to_the_plain_slot(orc, shift):
    """The signal generator's prefixed (and shifted) stream of a slot, demodulated by the oracle, gives the
    same grid as the plain slot with the same seed (up to the complex64 rounding of the stored samples)."""
    from paper_2210_09196_gb300 import synth
    cell = synth.SMALL_FP32
    plain = synth.make_slot(cell, 4)
    cp = synth.make_slot(cell.with_(cp=True, shift_7p5khz=shift), 4)
    assert cp.time_in.shape == (cell.n_rx, orc.slot_len(14, cell.n_fft)) and cp.time_in.flags["C_CONTIGUOUS"]
    f_plain = orc.ofdm_demod(plain.time_as_complex128(), cell.n_sc)
    f_cp = orc.ofdm_demod_cp(cp.time_as_complex128(), 14, cell.n_fft, cell.n_sc, shift=shift)
    assert np.max(np.abs(f_cp - f_plain)) < 1e-5 * np.max(np.abs(f_plain))
