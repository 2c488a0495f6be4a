"""GPU 3GPP type-1 DMRS (TS 38.211 5.2.1, 6.4.1.1): the Gold-sequence pilot generator equals the signal
generator's transmitted pilots bit for bit, and the chain with OCC-despread LS estimation (mean estimate, and
the estimate interpolated in time, and with the noise variance estimated from the CDM-group residuals) matches
the FP64 oracle chain (orc_chest_ls_type1 / orc_noise_est_type1 + Eq. 2) at 1e-4; the paths without type-1
support refuse such cells."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

CELL = synth.CellConfig("type1-16rx-512fft-4ue", n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4, qam_bits=4,
                        snr_db=30.0, channel="pdp", beam="dft", in_fp16=False, seed=12, dmrs="type1", n_id=41)


def nrel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n_id,n_scid,ports", [(41, 0, [0, 1, 2, 3]), (65535, 1, [3, 0]), (0, 0, [2])])
def test_pilot_generator_equals_transmitted_pilots(orc, n_id, n_scid, ports):
    cfg = host.cfg_for(CELL.with_(n_layers=len(ports), n_id=n_id), B.PUSCH_FORM_FP32, ports=ports)
    slots = [0, 7, 19, 3, 100]
    out = torch.empty((len(slots), len(ports), 2, CELL.n_sc), dtype=torch.complex64, device="cuda")
    B.pusch_dmrs_type1_pilots(cfg, len(slots), slots, n_id, n_scid, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    for i, sl in enumerate(slots):
        want = synth.dmrs_type1(n_id, n_scid, sl, ports, CELL.n_sc).astype(np.complex64)
        assert np.array_equal(got[i], want)
        assert np.array_equal(want, orc.dmrs_type1_pilots(n_id, n_scid, sl, ports, CELL.n_sc).astype(np.complex64))


def gpu_pilots(cfg, cell, n):
    p = torch.empty((n, cell.n_layers, 2, cell.n_sc), dtype=torch.complex64, device="cuda")
    B.pusch_dmrs_type1_pilots(cfg, n, [i % 20 for i in range(n)], cell.n_id, cell.n_scid, p)
    return p


def test_chain_with_type1_dmrs_matches_oracle(orc):
    n = 3
    slots = synth.make_slots(CELL, n)
    cfg = host.cfg_for(CELL, B.PUSCH_FORM_FP32)
    rx = host.Receiver(cfg, max_slots=n)
    x, b, st = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), gpu_pilots(cfg, CELL, n))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    e = p = 0.0
    for i, s in enumerate(slots):
        beam = orc.beamform(orc.ofdm_demod(s.time_as_complex128(), CELL.n_sc), s.W)
        xo, fails = orc.mmse(orc.chest_ls_type1(beam, s.pilots, s.ports), beam, s.noise_var)
        assert fails == 0
        xg = x[i].cpu().numpy().astype(np.complex128)
        assert nrel(xg, xo) < 1e-4
        e += np.sum(np.abs(xg - s.x) ** 2)
        p += np.sum(np.abs(s.x) ** 2)
    assert 10 * np.log10(e / p) < -20.0          # the oracle chain decodes this cell at about -25.6 dB
    rx.close()


def test_time_varying_estimate_with_type1_dmrs(orc):
    cell = CELL.with_(doppler_hz=300.0)
    n = 2
    slots = synth.make_slots(cell, n)
    cfg = host.cfg_for(cell, B.PUSCH_FORM_FP32, chol_every=4)
    rx = host.Receiver(cfg, max_slots=n)
    x, _, st = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), gpu_pilots(cfg, cell, n))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    for i, s in enumerate(slots):
        beam = orc.beamform(orc.ofdm_demod(s.time_as_complex128(), cell.n_sc), s.W)
        H0 = orc.chest_ls_type1_sym(beam, s.pilots, s.ports, 0)
        H1 = orc.chest_ls_type1_sym(beam, s.pilots, s.ports, 1)
        xo, fails = orc.mmse_tv(H0, H1, beam, s.noise_var, 4)
        assert fails == 0
        assert nrel(x[i].cpu().numpy().astype(np.complex128), xo) < 1e-4
    rx.close()


def test_paths_without_type1_support_refuse_it():
    rx = host.Receiver(host.cfg_for(CELL, B.PUSCH_FORM_FP32), max_slots=1)
    beam = rx.beam_buffer(1)
    grid = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    scale = torch.empty(1 << 12, dtype=torch.float32, device="cuda")
    with pytest.raises(B.PuschError) as ei:
        B.pusch_ls_grid(rx.h, 1, beam, torch.zeros((1, 4, 2, 300), dtype=torch.complex64, device="cuda"), grid, scale)
    assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED
    rx.close()
    rs = synth.make_ragged_slot(n_cells=2, n_users=4, slot_index=3)
    good = host.RaggedReceiver(rs, B.PUSCH_FORM_FP32)
    cells, users = list(good.cells), list(good.users)
    good.close()
    cells[0].dmrs_type = 1
    with pytest.raises(B.PuschError) as ei:
        B.pusch_batch_create(cells, users)
    assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED


def test_noise_estimate_type1_matches_oracle(orc):
    n = 2
    slots = synth.make_slots(CELL, n)
    cfg = host.cfg_for(CELL, B.PUSCH_FORM_FP32)
    rx = host.Receiver(cfg, max_slots=n)
    pil = gpu_pilots(cfg, CELL, n)
    beam = rx.beamform(rx.ofdm_fft(host.time_tensor(slots)), host.beam_tensor(slots[0].W))
    sig = rx.noise_estimate(beam, pil).cpu().numpy()
    for i, s in enumerate(slots):
        want = orc.noise_est_type1(beam[i].cpu().numpy().astype(np.complex128), s.pilots, s.ports)
        assert sig[i] == pytest.approx(want, rel=1e-5)
    rx.close()


def test_chain_type1_with_estimated_noise(orc):
    n = 2
    slots = synth.make_slots(CELL, n)
    cfg = host.cfg_for(CELL, B.PUSCH_FORM_FP32, noise_var=B.PUSCH_NOISE_ESTIMATE)
    rx = host.Receiver(cfg, max_slots=n)
    x, _, st = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), gpu_pilots(cfg, CELL, n))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    for i, s in enumerate(slots):
        beam = orc.beamform(orc.ofdm_demod(s.time_as_complex128(), CELL.n_sc), s.W)
        sig = orc.noise_est_type1(beam, s.pilots, s.ports)
        xo, fails = orc.mmse(orc.chest_ls_type1(beam, s.pilots, s.ports), beam, sig)
        assert fails == 0
        assert nrel(x[i].cpu().numpy().astype(np.complex128), xo) < 1e-4
    rx.close()
