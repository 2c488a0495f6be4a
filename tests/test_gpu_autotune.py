"""pusch_autotune on a single-cell handle: it times the FFT, beamforming, detector and pipelining shapes, the
chain's results stay bit-identical under the chosen shapes, and a second handle takes every choice from the
cache file without timing anything."""
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cell,form,keys", [
    (synth.DEPLOY, B.PUSCH_FORM_MIXED, 4),          # tensor-core FFT and GEMM, 16-layer detector
    (synth.SMALL_FP32, B.PUSCH_FORM_FP32, 3),        # SIMT FFT and beamforming, 4-layer detector
], ids=["deploy-mixed", "small-fp32"])
def test_autotune_keeps_results_and_caches_choices(tmp_path, cell, form, keys):
    slots = synth.make_slots(cell, 2)
    args = (host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    rx = host.Receiver(host.cfg_for(cell, form), max_slots=2)
    x0, b0, st0 = rx.slot(*args)
    torch.cuda.synchronize()
    cache = tmp_path / "tune.txt"
    assert B.pusch_autotune(rx.h, cache) == keys
    x1, b1, st1 = rx.slot(*args)
    torch.cuda.synchronize()
    assert torch.equal(x1, x0) and torch.equal(b1, b0) and torch.equal(st1, st0)
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == keys and all(" | " in l for l in lines)
    rx2 = host.Receiver(host.cfg_for(cell, form), max_slots=2)
    assert B.pusch_autotune(rx2.h, cache) == 0
    x2, b2, _ = rx2.slot(*args)
    torch.cuda.synchronize()
    assert torch.equal(x2, x0) and torch.equal(b2, b0)
    rx.close()
    rx2.close()
