"""The seeded input generator against the workload recipe it implements: orthonormal DFT beams (the noise
stays white after beamforming), unit-energy Gray constellations, the PDP channel's unit total tap power and
the configured SNR, the comb pilots, the deterministic seeding, and the ragged slot's drawing rules (PRB
ranges inside the cell's cap, at most N_B/2 layers overlapping anywhere, disjoint ports for overlapping
users, a pilot of every port inside its user's range)."""
import numpy as np
import pytest

from paper_2210_09196_gb300 import synth


def test_dft_beams_are_orthonormal():
    for cell in (synth.DEPLOY, synth.MASSIVE):
        W = synth.beam_matrix(cell).astype(np.complex128)
        assert np.allclose(W.conj().T @ W, np.eye(cell.n_beams), atol=1e-6)


def test_constellations_have_unit_energy_and_gray_labels():
    for q in (2, 4):
        bits = np.array([[(v >> k) & 1 for k in range(q)] for v in range(1 << q)])
        pts = synth.qam_map(bits, q)
        assert np.mean(np.abs(pts) ** 2) == pytest.approx(1.0, abs=1e-12)
        assert len(set(np.round(pts, 12))) == 1 << q
        # Gray: nearest neighbours differ in one bit
        for i, p in enumerate(pts):
            d = np.abs(pts - p)
            d[i] = np.inf
            for j in np.flatnonzero(np.isclose(d, d.min())):
                assert np.sum(bits[i] != bits[j]) == 1


def test_pdp_channel_power_and_snr():
    cell = synth.DEPLOY.with_(n_rx=32, n_beams=16, n_layers=4, n_fft=1024, n_sc=600)
    rng = np.random.default_rng(0)
    H = np.stack([synth._channel(cell, rng) for _ in range(40)])      # [draws, n_sc, R, L]
    assert np.mean(np.abs(H) ** 2) == pytest.approx(1.0, rel=0.05)    # unit total tap power per entry
    s = synth.make_slot(cell, 0)
    assert s.noise_var == pytest.approx(10 ** (-cell.snr_db / 10))


def test_comb_pilots_and_seeding():
    cell = synth.SMALL_FP32
    s = synth.make_slot(cell, 3)
    a = np.arange(cell.n_sc)
    for l in range(cell.n_layers):
        on = (a % cell.comb) == s.ports[l]
        assert np.all(s.pilots[l, :, ~on] == 0)
        assert np.allclose(np.abs(s.pilots[l, :, on]), 1.0, atol=1e-6)
    again = synth.make_slot(cell, 3)
    other = synth.make_slot(cell, 4)
    assert np.array_equal(s.time_in, again.time_in) and not np.array_equal(s.time_in, other.time_in)


def test_ragged_slot_drawing_rules():
    rs = synth.make_ragged_slot(n_cells=8, n_users=64, slot_index=0)
    assert len(rs.cells) == 8 and len(rs.users) == 64
    for c, cell in enumerate(rs.cells):
        assert cell.n_sc == 12 * int(np.floor(0.8 * cell.n_fft / 12))
        assert cell.n_beams == cell.n_rx // 2 and cell.comb == cell.n_beams // 2
        users = [u for u in rs.users if u.cell == c]
        load = np.zeros(cell.n_sc, dtype=int)
        for u in users:
            assert u.sc_start % 12 == 0 and u.sc_count % 12 == 0
            assert 0 <= u.sc_start and u.sc_start + u.sc_count <= cell.n_sc
            assert 1 <= u.n_layers <= 4 and u.port0 + u.n_layers <= cell.comb
            load[u.sc_start:u.sc_start + u.sc_count] += u.n_layers
            a = np.arange(u.sc_start, u.sc_start + u.sc_count)
            for p in range(u.port0, u.port0 + u.n_layers):
                assert np.any(a % cell.comb == p)
        assert load.max(initial=0) <= cell.comb
        for i, u in enumerate(users):
            for v in users[i + 1:]:
                if max(u.sc_start, v.sc_start) < min(u.sc_start + u.sc_count, v.sc_start + v.sc_count):
                    assert (u.port0 + u.n_layers <= v.port0) or (v.port0 + v.n_layers <= u.port0)
