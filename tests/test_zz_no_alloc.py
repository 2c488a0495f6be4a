"""pusch_slot_noalloc, the allocation-free variant of pusch_slot, called through the C ABI.

It is for callers that cannot allocate device memory (a real-time receiver thread that must not enter the
CUDA allocator, a plug-in whose framework owns all device memory, a stateless callback without a handle).
Its output must equal pusch_slot's on the same inputs, on two calls in a row (the static buffer keeps the
previous call's contents, which must not leak into the next call), within the tolerance the other GPU
tests use. This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def nrel(a, b):
    a = a.detach().cpu().numpy().astype(np.complex128)
    b = b.detach().cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def _bufs(rx, n):
    return rx.xhat_buffer(n), rx.bits_buffer(n), rx.status_buffer()


@pytest.mark.parametrize("form", [B.PUSCH_FORM_FP32, B.PUSCH_FORM_MIXED, B.PUSCH_FORM_FP8])
def test_noalloc_matches_pusch_slot_on_two_calls(form):
    # the small cell (16 antennas, 512-point FFT, 300 subcarriers); the FP8 form's E4M3 planes and block
    # scales are carved out of the static buffer like the other forms' intermediates
    cell = synth.SMALL_FP32
    slots = synth.make_slots(cell, 6)
    cfg = host.cfg_for(cell, form)
    rx = host.Receiver(cfg, max_slots=3)
    W = host.beam_tensor(slots[0].W)
    for call, group in enumerate((slots[:3], slots[3:])):
        t, p = host.time_tensor(group), host.pilot_tensor(group)
        ref = _bufs(rx, 3)
        B.pusch_slot(rx.h, 3, t, W, p, *ref)
        out = _bufs(rx, 3)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        B.pusch_slot_noalloc(cfg, 3, t, W, p, *out)
        torch.cuda.synchronize()
        if call == 1:   # the first call may load the library's device code; the second allocates nothing
            assert torch.cuda.mem_get_info()[0] == free_before
        assert nrel(out[0], ref[0]) <= TOL, f"call {call}"
        assert torch.equal(out[2], ref[2]), f"call {call}"
        mism = (out[1] != ref[1]).float().mean().item()
        assert mism == 0.0, f"call {call}: {mism}"
    rx.close()


def test_noalloc_rejects_sizes_beyond_its_buffer():
    cell = synth.DEPLOY
    cfg = host.cfg_for(cell, B.PUSCH_FORM_FP32)
    dummy = torch.empty(16, device="cuda")
    with pytest.raises(B.PuschError) as ei:
        B.pusch_slot_noalloc(cfg, 1, dummy, dummy, dummy, dummy, dummy)
    assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED
    assert "scratch" in B.pusch_last_error() or "scratch" in str(ei.value)
    small = host.cfg_for(synth.SMALL_FP32, B.PUSCH_FORM_FP32)
    with pytest.raises(B.PuschError) as ei:
        B.pusch_slot_noalloc(small, 1000, dummy, dummy, dummy, dummy, dummy)
    assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED
