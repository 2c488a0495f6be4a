"""GPU parity of the FP8 form: FFT output stored as E4M3 codes with one power-of-two scale per 128
subcarriers, W quantised to E4M3 per (beam, 128 antennas), beamforming as the block-scaled product of the two
quantised operands on tcgen05 with FP32 accumulation; estimation and detection FP32.

* FFT: the GPU's block exponents and codes equal the oracle's quantisation (orc_e4m3_quant_rows) of the
  oracle spectrum, except where the FP32 transform's rounding error can move a value across a decision
  (a scale boundary or a rounding midpoint); those differ by one grid step at most.
* Beamforming, quantisation-exact: the oracle's block-scaled product (orc_beamform_fp8) of the very codes and
  exponents the GPU wrote, and W, against the GPU beams: norm-relative <= 1e-5 (FP32 accumulation only).
* Whole chain at the 256-antenna massive cell: EVM against the FP64 oracle chain <= -25 dB (E4M3 keeps 3
  mantissa bits: about -30 dB is expected). Hard decisions: with the measured EVM as a Gaussian error of
  standard deviation sigma per component, a bit whose oracle value lies delta from its own decision threshold
  flips with probability Q(delta / sigma); the number of flipped bits must stay within five standard
  deviations of the sum of those probabilities, and no bit flips more than 6 sigma from its threshold.
"""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


def nrel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def decode_fp8(freq, cfg, n):
    """GPU FP8 FFT output -> (codes complex [n, S, R, n_sc] as E4M3 values, exps int [n, S, R, n_blk])."""
    S, R, n_sc = cfg.n_sym, cfg.n_rx, cfg.n_sc
    pitch = B.pusch_sc_pitch(cfg)
    n_blk = (n_sc + 127) // 128
    planes_b = n * S * R * 2 * pitch
    off = (planes_b + 255) // 256 * 256
    raw = freq.detach().cpu()
    pl = raw[:planes_b].view(torch.float8_e4m3fn).to(torch.float64).numpy().reshape(n, S, R, 2, pitch)
    sc = raw[off:off + n * S * n_blk * R * 4].view(torch.float32).numpy().reshape(n, S, n_blk, R)
    pads = raw[:planes_b].numpy().reshape(n, S, R, 2, pitch)[..., n_sc:]
    codes = pl[..., 0, :n_sc] + 1j * pl[..., 1, :n_sc]
    with np.errstate(divide="ignore", invalid="ignore"):
        exps = np.where(np.isfinite(sc), np.log2(sc), 128).round().astype(np.int32)
    return codes, np.transpose(exps, (0, 1, 3, 2)), pads


def bit_flip_check(xo, bits_gpu, bits_orc, sigma, qam_bits):
    """Bits that differ between the GPU's and the oracle's Gray decisions (3GPP TS 38.211 5.1.3/5.1.4) against a
    Gaussian error model of standard deviation sigma per component. Bit 0 / 1 is the sign of Re / Im (threshold
    0); for 16-QAM bit 2 / 3 compares |Re| / |Im| with 2 / sqrt(10). Returns (flipped bits, expected flips
    sum_i Q(delta_i / sigma), their variance, flips with delta > 6 sigma)."""
    from scipy.special import erfc
    t = 2.0 / np.sqrt(10.0)
    deltas = [np.abs(xo.real), np.abs(xo.imag)]
    if qam_bits == 4:
        deltas += [np.abs(np.abs(xo.real) - t), np.abs(np.abs(xo.imag) - t)]
    flips = expected = var = far = 0
    for j, dl in enumerate(deltas):
        mism = ((bits_gpu >> j) & 1) != ((bits_orc >> j) & 1)
        p = 0.5 * erfc(dl / (sigma * np.sqrt(2.0)))
        flips += int(mism.sum())
        expected += float(p.sum())
        var += float((p * (1 - p)).sum())
        far += int((mism & (dl > 6 * sigma)).sum())
    return flips, expected, var, far


FP8_SHAPES = [
    dict(n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4, qam_bits=2),
    dict(n_rx=48, n_fft=1024, n_sc=1000, n_beams=24, n_layers=8, qam_bits=4),
    dict(n_rx=144, n_fft=2048, n_sc=1638, n_beams=40, n_layers=16, qam_bits=4),   # partial last K chunk
    dict(n_rx=256, n_fft=4096, n_sc=3276, n_beams=64, n_layers=32, qam_bits=4),
]


@pytest.mark.parametrize("shape", FP8_SHAPES, ids=lambda d: f"R{d['n_rx']}sc{d['n_sc']}B{d['n_beams']}")
def test_fp8_fft_and_block_scaled_beamforming(orc, shape):
    n = 2
    cell = synth.CellConfig("f8", snr_db=25.0, channel="pdp", beam="dft", in_fp16=True, seed=31, **shape)
    slots = synth.make_slots(cell, n)
    cfg = host.cfg_for(cell, B.PUSCH_FORM_FP8)
    rx = host.Receiver(cfg, max_slots=n)
    freq = rx.ofdm_fft(host.time_tensor(slots))
    assert freq.numel() == B.pusch_freq_bytes(cfg, n)
    beam = rx.beamform(freq, host.beam_tensor(slots[0].W))
    torch.cuda.synchronize()
    codes, exps, pads = decode_fp8(freq, cfg, n)
    assert np.all(pads == 0)
    n_exp_diff = n_code_diff = 0
    for i, s in enumerate(slots):
        f_orc = orc.ofdm_demod(s.time_as_complex128(), cell.n_sc)
        c_orc, e_orc = orc.e4m3_quant_rows(f_orc)
        # exponents: a difference only where the block maximum sits within FP32 error of 448 * 2^e
        diff = np.argwhere(exps[i] != e_orc)
        for s_, r_, j in diff:
            blk = f_orc[s_, r_, 128 * j:128 * j + 128]
            amax = max(np.abs(blk.real).max(), np.abs(blk.imag).max())
            ratio = amax / (448.0 * 2.0 ** min(exps[i][s_, r_, j], e_orc[s_, r_, j]))
            assert abs(ratio - 1.0) < 1e-5, (s_, r_, j, ratio)
            assert abs(int(exps[i][s_, r_, j]) - int(e_orc[s_, r_, j])) == 1
        n_exp_diff += len(diff)
        # codes of blocks with equal exponents: equal except next to a rounding midpoint
        same = np.repeat(exps[i] == e_orc, 128, axis=-1)[..., :cell.n_sc]
        for part in (np.real, np.imag):
            g, o = part(codes[i]), part(c_orc)
            scaled = part(f_orc) / 2.0 ** np.repeat(e_orc, 128, axis=-1)[..., :cell.n_sc]
            bad = same & (g != o)
            if np.any(bad):
                # the exact value lies next to the midpoint of the two candidates: within the FP32 transform's
                # error, about 1e-6 of the block maximum (448 code units), with a 10x margin
                mid = 0.5 * (g[bad] + o[bad])
                step = np.abs(g[bad] - o[bad])
                assert np.all(np.abs(scaled[bad] - mid) <= 448.0 * 1e-5 + 1e-5 * np.abs(mid)), \
                    np.abs(scaled[bad] - mid).max()
                assert np.all(step <= 2.0 ** -3 * np.maximum(np.abs(mid), 2.0 ** -6) * 1.0001)
            n_code_diff += int(bad.sum())
        # beamforming: the oracle's block-scaled product of the GPU's own codes and exponents
        b_orc = orc.beamform_fp8(codes[i], exps[i], s.W)
        assert nrel(beam[i].cpu().numpy(), b_orc) < 1e-5
    total = n * 14 * cell.n_rx * cell.n_sc * 2
    assert n_code_diff <= 1e-3 * total, n_code_diff
    rx.close()


def test_fp8_config_rules():
    ok = synth.MASSIVE
    cfg = host.cfg_for(ok, B.PUSCH_FORM_FP8)
    h = B.pusch_create(cfg, 1)
    B.pusch_destroy(h)
    for bad in (ok.with_(n_rx=24), ok.with_(n_rx=1024), ok.with_(n_beams=12, n_layers=12)):
        with pytest.raises(B.PuschError) as ei:
            B.pusch_create(host.cfg_for(bad, B.PUSCH_FORM_FP8), 1)
        assert ei.value.code == B.PUSCH_ERR_UNSUPPORTED


def test_fp8_nonfinite_sample_flags_status():
    cell = synth.CellConfig("f8nan", n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4, qam_bits=2, snr_db=25.0,
                            channel="pdp", beam="dft", in_fp16=True, seed=3)
    s = synth.make_slot(cell, 0)
    t = host.time_tensor([s])
    t[0, 5, 3, 17, 0] = float("nan")                 # one time sample of a data symbol
    rx = host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_FP8), max_slots=1)
    x, b, st = rx.slot(t, host.beam_tensor(s.W), host.pilot_tensor([s]))
    torch.cuda.synchronize()
    assert int(st[0]) & B.PUSCH_STATUS_NONFINITE
    rx.close()


@pytest.fixture(scope="module")
def massive_slots():
    return synth.make_slots(synth.MASSIVE, 2)


@pytest.fixture(scope="module")
def massive_ref(orc, massive_slots):
    return [orc.run_slot(s) for s in massive_slots]


@pytest.mark.parametrize("form,evm_max", [(B.PUSCH_FORM_FP8, -25.0), (B.PUSCH_FORM_MIXED, -40.0)])
def test_massive_chain_vs_oracle(massive_slots, massive_ref, form, evm_max):
    cell = synth.MASSIVE
    n = len(massive_slots)
    rx = host.Receiver(host.cfg_for(cell, form), max_slots=n)
    x, b, st = rx.slot(host.time_tensor(massive_slots), host.beam_tensor(massive_slots[0].W),
                       host.pilot_tensor(massive_slots))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    for i, s in enumerate(massive_slots):
        xo, bo, fails = massive_ref[i]
        assert fails == 0
        xg = x[i].cpu().numpy().astype(np.complex128)
        err = xg - xo
        evm = 10 * np.log10(np.sum(np.abs(err) ** 2) / np.sum(np.abs(xo) ** 2))
        assert evm <= evm_max, evm
        sigma = np.sqrt(np.mean(np.abs(err) ** 2) / 2)
        flips, expected, var, far = bit_flip_check(xo, b[i].cpu().numpy(), bo, sigma, cell.qam_bits)
        print(f"\nform {form}: EVM {evm:.1f} dB, sigma {sigma:.4f}, flipped bits {flips} (expected {expected:.1f})")
        assert far == 0, far
        assert flips <= expected + 5.0 * np.sqrt(var) + 3.0, (flips, expected, var)
    rx.close()
