"""Pipelined pusch_slot / pusch_slot_host (the batch as chunk runs alternating over two streams): every form
and mode gives bit-identical outputs and status words for every chunk count, including a batch with fewer
slots than chunks, the host-buffer path with per-chunk copies, and the stage profile of the chunk runs."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

SMALL = synth.SMALL_FP32
FP8_SMALL = synth.CellConfig("f8-16rx-512fft", n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4, qam_bits=2,
                             snr_db=25.0, channel="pdp", beam="dft", in_fp16=True, seed=31)
MODES = {
    "fp32": (SMALL, B.PUSCH_FORM_FP32, {}),
    "mixed": (SMALL, B.PUSCH_FORM_MIXED, {}),
    "fp8": (FP8_SMALL, B.PUSCH_FORM_FP8, {}),
    "estimate": (SMALL, B.PUSCH_FORM_FP32, dict(noise_var=B.PUSCH_NOISE_ESTIMATE)),
    "time_groups": (SMALL.with_(channel="pdp", beam="dft", doppler_hz=300.0), B.PUSCH_FORM_FP32, dict(chol_every=4)),
}


@pytest.mark.parametrize("mode", list(MODES))
def test_chunked_runs_are_bit_identical(mode):
    cell, form, kw = MODES[mode]
    n = 5
    slots = synth.make_slots(cell, n)
    rx = host.Receiver(host.cfg_for(cell, form, **kw), max_slots=n)
    t, w, p = host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots)
    x1, b1, s1 = (v.clone() for v in rx.slot(t, w, p))
    for k in (2, 3, 5, 16):
        rx.set_pipeline(k)
        x, b, s = rx.slot(t, w, p)
        torch.cuda.synchronize()
        assert torch.equal(x, x1) and torch.equal(b, b1) and torch.equal(s, s1), k
    # one slot with a chunk count above it runs as one chunk
    xs, bs, ss = rx.slot(t[:1], w, p[:1])
    torch.cuda.synchronize()
    assert torch.equal(xs[0], x1[0]) and torch.equal(bs[0], b1[0])
    rx.close()


def test_host_path_pipelined_equals_device_path():
    cell = SMALL
    n = 6
    slots = synth.make_slots(cell, n)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP32), max_slots=n)
    t, w, p = host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots)
    x1, b1, s1 = (v.clone() for v in rx.slot(t, w, p))
    th, ph = host.time_tensor(slots, "cpu", pin=True), host.pilot_tensor(slots, "cpu", pin=True)
    for k in (1, 3):
        rx.set_pipeline(k)
        out = (rx.xhat_buffer(n, "cpu").pin_memory(), rx.bits_buffer(n, "cpu").pin_memory(),
               rx.status_buffer("cpu").pin_memory())
        rx.slot_host(th, w, ph, out)
        assert torch.equal(out[0], x1.cpu()) and torch.equal(out[1], b1.cpu()) and torch.equal(out[2], s1.cpu())
    rx.close()


def test_profile_of_chunk_runs():
    cell = SMALL
    n = 4
    slots = synth.make_slots(cell, n)
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP32), max_slots=n)
    t, w, p = host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots)
    rx.set_pipeline(2)
    B.pusch_profile_start(rx.h, 3)
    for _ in range(4):                                   # the fourth call finds no records left: not timed
        rx.slot(t, w, p)
    ms, calls = B.pusch_profile_read(rx.h)
    assert calls == 3
    assert all(v > 0 for v in ms.values())
    rx.close()


def test_pipeline_arguments():
    rx = host.Receiver(host.cfg_for(SMALL, B.PUSCH_FORM_FP32), max_slots=2)
    for bad in (0, 17, -1):
        with pytest.raises(B.PuschError) as ei:
            rx.set_pipeline(bad)
        assert ei.value.code == B.PUSCH_ERR_ARG
    rx.set_pipeline(16)
    rx.set_pipeline(1)
    rx.close()
