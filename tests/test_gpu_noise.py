"""GPU noise-variance estimation (Section II NE) against the FP64 oracle, and the chain in the estimate mode
(PUSCH_NOISE_ESTIMATE) against the oracle chain fed the oracle's own estimate."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cell", [synth.SMALL_FP32, synth.DEPLOY.with_(snr_db=15.0)], ids=["small", "deploy15dB"])
def test_noise_estimate_matches_oracle(orc, cell):
    slots = synth.make_slots(cell, 2)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP32), max_slots=2)
    beam = rx.beamform(rx.ofdm_fft(host.time_tensor(slots)), host.beam_tensor(slots[0].W))
    sig = rx.noise_estimate(beam, host.pilot_tensor(slots)).cpu().numpy()
    sig2 = rx.noise_estimate(beam, host.pilot_tensor(slots)).cpu().numpy()
    assert np.array_equal(sig, sig2)                       # fixed reduction order
    for i, s in enumerate(slots):
        want = orc.noise_est(beam[i].cpu().numpy().astype(np.complex128), s.pilots, s.ports, cell.comb)
        assert sig[i] == pytest.approx(want, rel=1e-5)
        # the estimate tracks the configured noise: 10^(-SNR/10) per antenna, unchanged by orthonormal beams
        if cell.channel == "pdp":
            assert sig[i] == pytest.approx(s.noise_var, rel=0.1)
    rx.close()


def test_chain_with_estimated_noise_matches_oracle_chain(orc):
    cell = synth.SMALL_FP32
    slots = synth.make_slots(cell, 3)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP32, noise_var=B.PUSCH_NOISE_ESTIMATE), max_slots=3)
    x, b, st = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    x2, _, _ = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    assert torch.equal(x, x2)
    for i, s in enumerate(slots):
        freq = orc.ofdm_demod(s.time_as_complex128(), cell.n_sc)
        beam = orc.beamform(freq, s.W)
        sig = orc.noise_est(beam, s.pilots, s.ports, cell.comb)
        H = orc.chest_ls(beam, s.pilots, s.ports, cell.comb)
        xo, fails = orc.mmse(H, beam, sig)
        assert fails == 0
        xg = x[i].cpu().numpy().astype(np.complex128)
        assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-4
    rx.close()


def test_noalloc_chain_with_estimated_noise():
    cell = synth.SMALL_FP32
    slots = synth.make_slots(cell, 2)
    cfg = host.cfg_for(cell, B.PUSCH_FORM_FP32, noise_var=B.PUSCH_NOISE_ESTIMATE)
    rx = host.Receiver(cfg, max_slots=2)
    t, w, p = host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots)
    x, b, st = rx.slot(t, w, p)
    x2, b2, st2 = rx.xhat_buffer(2), rx.bits_buffer(2), rx.status_buffer()
    B.pusch_slot_noalloc(cfg, 2, t, w, p, x2, b2, st2)
    torch.cuda.synchronize()
    # the no-alloc chain stores the estimate and detects from it; the handle chain fuses the interpolation:
    # same arithmetic up to FP32 evaluation order
    xa, xb = x.cpu().numpy(), x2.cpu().numpy()
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xa) < 1e-5
    rx.close()


def test_batch_rejects_the_estimate_mode():
    rs = synth.make_ragged_slot(n_cells=2, n_users=4, slot_index=3)
    good = host.RaggedReceiver(rs, B.PUSCH_FORM_FP32)
    cells = list(good.cells)
    users = list(good.users)
    good.close()
    cells[1].noise_var = B.PUSCH_NOISE_ESTIMATE
    with pytest.raises(B.PuschError) as ei:
        B.pusch_batch_create(cells, users)
    assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED
