"""The benchmark's per-stage models on CPU: algorithmic bytes and FLOPs per launch (the roofline's numerators),
the kernel each stage runs, and the source files its traffic counters are keyed by.

The deployment cell (Section II: 3276 subcarriers, 14 symbols, 64 antennas, 32 beams, 16 single-layer users on a
16-subcarrier pilot comb) is worked out by hand here, so that a change of the model shows up as a changed
number, not as a silently different roofline."""
import importlib.util
import os

import pytest

pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_model_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_detection_flops_of_the_deployment_step():
    """Per subcarrier: Hermitian Gram 16*17/2*32 = 4352, right-hand sides 12*16*32 = 6144, Cholesky 16^3/6, two
    triangular solves 12*16^2 = 3072 complex MACs; 8 flop each, 3276 subcarriers, 16 slots."""
    b = _bench()
    from paper_2210_09196_gb300 import synth
    macs = 4352 + 6144 + 16 ** 3 / 6 + 3072
    assert b.stage_flops(synth.DEPLOY, 16)["detect"] == pytest.approx(8 * macs * 3276 * 16)
    assert round(b.stage_flops(synth.DEPLOY, 16)["detect"]) == 5975703552
    # beamforming: 14 symbols x 3276 subcarriers x 64 antennas x 32 beams complex MACs per slot
    assert b.stage_flops(synth.DEPLOY, 1)["beamform"] == 8.0 * 14 * 3276 * 64 * 32


def test_stage_bytes_with_the_estimate_interpolated_in_the_detector():
    """16 layers, 32 beams: the LS stage writes only the pilot table, the detector reads it (no estimate)."""
    b = _bench()
    from paper_2210_09196_gb300 import synth
    sb = b.stage_bytes(synth.DEPLOY, "mixed", 1)
    table = 16 * 205 * 32 * 8                       # 16 layers x ceil(3276 / 16) pilots x 32 beams x c64
    dmrs = 2 * 3276 * 32 * 8                        # the two DMRS symbols' beams
    pilots = 16 * 2 * 3276 * 8
    data = 12 * 3276 * 32 * 8                       # the 12 data symbols' beams
    out = 16 * 12 * 3276 * (8 + 1)                  # x-hat (c64) and one byte of bits per symbol
    assert sb["ls"] == dmrs + pilots + table
    assert sb["detect"] == data + table + out
    fft_in = 14 * 64 * 4096 * 4                     # FP16 complex time samples
    planes = 14 * 64 * 3276 * 4                     # FP16 re and im planes
    assert sb["fft"] == fft_in + planes
    assert sb["beamform"] == planes + 14 * 3276 * 32 * 8 + 64 * 32 * 8


def test_stage_bytes_with_the_interpolation_kernel():
    """8 layers (a class whose detector reads the estimate): the LS stage also writes the interpolated estimate
    and reads the table back, and the detector reads the estimate."""
    b = _bench()
    from paper_2210_09196_gb300 import synth
    cell = synth.DEPLOY.with_(n_layers=8)
    sb = b.stage_bytes(cell, "fp32", 1)
    table = 8 * 410 * 32 * 8                        # comb 8: ceil(3276 / 8) pilots per layer
    est = 3276 * 8 * 32 * 8
    assert sb["ls"] == 2 * 3276 * 32 * 8 + 8 * 2 * 3276 * 8 + 2 * table + est
    assert sb["detect"] == 12 * 3276 * 32 * 8 + est + 8 * 12 * 3276 * 9


def test_kernels_of_the_stages_and_their_sources():
    b = _bench()
    from paper_2210_09196_gb300 import synth
    assert b.kernel_of("fft", "mixed", synth.DEPLOY)[0] == "fft_tc_kernel"
    assert b.kernel_of("fft", "fp32", synth.DEPLOY)[0] == "fft_kernel"
    assert b.kernel_of("fft", "fp8", synth.MASSIVE)[0] == "fft_kernel"
    assert b.kernel_of("beamform", "mixed", synth.DEPLOY)[0] == "beamform_tc_kernel"
    assert b.kernel_of("beamform", "fp32", synth.DEPLOY)[0] == "beamform_tf32_kernel"
    assert b.kernel_of("detect", "mixed", synth.DEPLOY)[0] == "mmse_kernel"
    csrc = os.path.join(ROOT, "paper_2210_09196_gb300", "csrc")
    for stage, k in b.KERNELS.items():
        for name, src in (k.values() if isinstance(k, dict) else [k]):
            for part in src.split("+"):
                assert os.path.isfile(os.path.join(csrc, part)), (stage, name, part)
