"""Failure reporting through the C ABI on the GPU: the bounded-wait self-test expires on a barrier that nothing
completes, the kernel returns, and the expiry reaches the caller as PUSCH_ERR_TIMEOUT from pusch_status_check
and as PUSCH_STATUS_TIMEOUT in the next chain call's status words; numeric failures (Eq. 2's factorisation
meeting a non-positive pivot) come back as PUSCH_ERR_NUMERIC. No test faults, traps or hangs the GPU: the only
wait that expires is the self-test's, which issues no copy or MMA."""
import time

import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


def _rx(max_slots=2, **kw):
    return host.Receiver(host.cfg_for(synth.SMALL_FP32, **kw), max_slots=max_slots)


def test_selftest_wait_expires_and_is_reported():
    rx = _rx()
    t0 = time.time()
    B.pusch_selftest_wait(rx.h, 2000)
    torch.cuda.synchronize()            # the kernel gave up and returned
    assert time.time() - t0 < 10.0
    with pytest.raises(B.PuschError) as ei:
        B.pusch_status_check(rx.h)
    assert ei.value.code == B.PUSCH_ERR_TIMEOUT
    assert "0x4" in str(ei.value)
    B.pusch_status_check(rx.h)          # the check cleared the handle's error word
    rx.close()


def test_timeout_reaches_the_next_slot_status_and_the_context_stays_usable(orc):
    cell = synth.SMALL_FP32
    slots = synth.make_slots(cell, 2)
    args = (host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    rx = _rx()
    x0, b0, st0 = rx.slot(*args)
    torch.cuda.synchronize()
    assert list(st0.cpu().numpy()) == [0, 0, -1, 0]
    B.pusch_status_check(rx.h, st0)
    B.pusch_selftest_wait(rx.h, 1000)
    x1, b1, st1 = rx.slot(*args)
    torch.cuda.synchronize()
    s1 = st1.cpu().numpy().astype(np.int64) & 0xffffffff
    assert s1[0] & B.PUSCH_STATUS_TIMEOUT and s1[3] == 4
    with pytest.raises(B.PuschError) as ei:
        B.pusch_status_check(None, st1)
    assert ei.value.code == B.PUSCH_ERR_TIMEOUT
    # the chain itself ran normally: the same results as before the expired wait, and the next call is clean
    assert torch.equal(x1, x0) and torch.equal(b1, b0)
    x2, _, st2 = rx.slot(*args)
    torch.cuda.synchronize()
    assert list(st2.cpu().numpy()) == [0, 0, -1, 0]
    B.pusch_status_check(rx.h, st2)
    xo, _, _ = orc.run_slot(slots[0])
    xg = x2[0].cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) < 1e-5
    rx.close()


def test_timeout_reaches_the_detector_status_after_a_stage_call():
    """An expiry recorded by earlier work on the handle is reported by the next pusch_mmse_detect."""
    cell = synth.SMALL_FP32
    rx = _rx()
    H = torch.ones((1, cell.n_sc, cell.n_layers, cell.n_beams), dtype=torch.complex64, device="cuda")
    H += torch.eye(cell.n_layers, cell.n_beams, dtype=torch.complex64, device="cuda")
    beam = torch.ones((1, 14, cell.n_sc, cell.n_beams), dtype=torch.complex64, device="cuda")
    B.pusch_selftest_wait(rx.h, 500)
    x, b, st = rx.mmse_detect(H, beam)
    torch.cuda.synchronize()
    s = st.cpu().numpy().astype(np.int64) & 0xffffffff
    assert s[0] == B.PUSCH_STATUS_TIMEOUT and s[3] == 4
    rx.close()


def test_status_check_reports_numeric_failures():
    cell = synth.SMALL_FP32
    rx = _rx(noise_var=0.0)
    H = torch.zeros((1, cell.n_sc, cell.n_layers, cell.n_beams), dtype=torch.complex64, device="cuda")
    beam = torch.ones((1, 14, cell.n_sc, cell.n_beams), dtype=torch.complex64, device="cuda")
    x, b, st = rx.mmse_detect(H, beam)
    with pytest.raises(B.PuschError) as ei:
        B.pusch_status_check(rx.h, st)
    assert ei.value.code == B.PUSCH_ERR_NUMERIC
    assert f"{cell.n_sc} factorisation" in str(ei.value)
    rx.close()


def test_ragged_batch_status_carries_no_timeout():
    rs = synth.make_ragged_slot(n_cells=2, n_users=4, slot_index=1)
    rr = host.RaggedReceiver(rs)
    t, w, p = rr.pack(rs)
    out = rr.outputs()
    rr.run(t, w, p, out)
    B.pusch_status_check(None, out[2])
    assert int(out[2][3].item()) == 0
    rr.close()
