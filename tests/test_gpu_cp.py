"""GPU parity of cyclic-prefix removal and the 7.5 kHz shift (time input as one stream per antenna with NR
normal prefixes, TS 38.211 5.3.1 / 5.4): the FFT against the oracle's orc_ofdm_demod_cp (FP32: norm-relative
<= 1e-5), the whole chain at the deployment cell in the mixed form (EVM <= -40 dB against the FP64 chain), the
pipelined and the no-alloc chains reading the streams, and the configuration rules."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


def nrel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


CELLS = {
    "c64_512_cp": synth.SMALL_FP32.with_(cp=True),
    "c64_512_cp_shift": synth.SMALL_FP32.with_(cp=True, shift_7p5khz=True),
    "c64_512_shift_only": synth.SMALL_FP32.with_(shift_7p5khz=True),
    "f16_1024_cp_shift": synth.CellConfig("f16-32rx-1024", n_rx=32, n_fft=1024, n_sc=600, n_beams=16, n_layers=4,
                                          qam_bits=4, snr_db=30.0, channel="pdp", beam="dft", in_fp16=True, seed=8,
                                          cp=True, shift_7p5khz=True),
}


@pytest.mark.parametrize("name", list(CELLS))
def test_fft_with_prefixes_and_shift_matches_oracle(orc, name):
    cell = CELLS[name]
    slots = synth.make_slots(cell, 2)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP32), max_slots=2)
    freq = rx.ofdm_fft(host.time_tensor(slots)).cpu().numpy()
    for i, s in enumerate(slots):
        t = s.time_as_complex128()
        if cell.cp:
            want = orc.ofdm_demod_cp(t, 14, cell.n_fft, cell.n_sc, shift=cell.shift_7p5khz)
        else:  # shift only: undo it on each symbol, then the plain transform
            n = np.arange(cell.n_fft)
            want = orc.ofdm_demod(t * np.exp(-2j * np.pi * n / (4 * cell.n_fft)), cell.n_sc)
        assert nrel(freq[i], want) < 1e-5
    rx.close()


def test_deploy_chain_with_prefixes_and_shift(orc):
    cell = synth.DEPLOY.with_(cp=True, shift_7p5khz=True)
    slots = synth.make_slots(cell, 1)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_MIXED), max_slots=1)
    x, b, st = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    s = slots[0]
    freq = orc.ofdm_demod_cp(s.time_as_complex128(), 14, cell.n_fft, cell.n_sc, shift=True)
    beam = orc.beamform(freq, s.W)
    xo, fails = orc.mmse(orc.chest_ls(beam, s.pilots, s.ports, cell.comb), beam, s.noise_var)
    assert fails == 0
    xg = x[0].cpu().numpy().astype(np.complex128)
    evm = 10 * np.log10(np.sum(np.abs(xg - xo) ** 2) / np.sum(np.abs(xo) ** 2))
    assert evm <= -40.0, evm
    rx.close()


def test_pipelined_and_noalloc_chains_read_the_streams():
    cell = CELLS["c64_512_cp_shift"]
    n = 5
    slots = synth.make_slots(cell, n)
    cfg = host.cfg_for(cell, B.PUSCH_FORM_FP32)
    rx = host.Receiver(cfg, max_slots=n)
    t, w, p = host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots)
    x1, b1, s1 = (v.clone() for v in rx.slot(t, w, p))
    rx.set_pipeline(3)
    x, b, s = rx.slot(t, w, p)
    torch.cuda.synchronize()
    assert torch.equal(x, x1) and torch.equal(b, b1) and torch.equal(s, s1)
    x2, b2, s2 = rx.xhat_buffer(n), rx.bits_buffer(n), rx.status_buffer()
    B.pusch_slot_noalloc(cfg, n, t, w, p, x2, b2, s2)
    torch.cuda.synchronize()
    assert nrel(x2.cpu().numpy(), x1.cpu().numpy()) < 1e-5
    rx.close()


def test_batch_refuses_prefixed_cells():
    rs = synth.make_ragged_slot(n_cells=2, n_users=4, slot_index=3)
    good = host.RaggedReceiver(rs, B.PUSCH_FORM_FP32)
    cells, users = list(good.cells), list(good.users)
    good.close()
    for field in ("cp", "shift_7p5khz"):
        bad = [type(c)() for c in cells]
        for b_, c in zip(bad, cells):
            ctypes_copy(b_, c)
        setattr(bad[1], field, 1)
        with pytest.raises(B.PuschError) as ei:
            B.pusch_batch_create(bad, users)
        assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED


def ctypes_copy(dst, src):
    import ctypes
    ctypes.memmove(ctypes.addressof(dst), ctypes.addressof(src), ctypes.sizeof(src))
