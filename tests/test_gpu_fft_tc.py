"""The mixed form's tensor-core FFT (4096 points, FP16 time samples; three radix-16 tcgen05 stages) against the
FP64 oracle's DFT, through pusch_ofdm_fft (Section II, Table I "OFDM dem.").

The operands of each stage are FP16, so the comparison is at the FP16 bar of the mixed form (norm-relative
<= 1e-3, i.e. better than -60 dB; the test prints the measured figure), on random rows, on single tones (the
energy lands in one bin), on an odd and a small active-band width (pads written as zero) and on more rows than
the persistent grid holds."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


def _planes(freq, n_sc):
    f = freq.detach().cpu().numpy().astype(np.float64)
    return f[..., 0, :n_sc] + 1j * f[..., 1, :n_sc]


def _rx(n_sc, n_rx=8, max_slots=2):
    cell = synth.CellConfig("fft", n_rx=n_rx, n_fft=4096, n_sc=n_sc, n_beams=8, n_layers=2, qam_bits=2, snr_db=30.0,
                            channel="pdp", beam="dft", in_fp16=True, seed=3)
    return cell, host.Receiver(host.cfg_for(cell, B.PUSCH_FORM_MIXED), max_slots=max_slots)


@pytest.mark.parametrize("n_sc", [3276, 3275, 100, 4096])
def test_tensor_core_fft_random_rows(orc, n_sc):
    cell, rx = _rx(n_sc)
    rng = np.random.default_rng(n_sc)
    x = (rng.standard_normal((2, 14, cell.n_rx, 4096)) + 1j * rng.standard_normal((2, 14, cell.n_rx, 4096))) * 0.02
    t16 = np.stack([x.real, x.imag], axis=-1).astype(np.float16)
    freq = rx.ofdm_fft(torch.from_numpy(t16).cuda())
    torch.cuda.synchronize()
    fr = freq.cpu().numpy()
    assert np.all(fr[..., n_sc:] == 0)
    xin = t16[..., 0].astype(np.float64) + 1j * t16[..., 1].astype(np.float64)
    err = ref = 0.0
    for i in range(2):
        fo = orc.ofdm_demod(xin[i], n_sc)
        fg = _planes(freq[i], n_sc)
        err += np.sum(np.abs(fg - fo) ** 2)
        ref += np.sum(np.abs(fo) ** 2)
        per_row = np.linalg.norm((fg - fo).reshape(-1, n_sc), axis=1) / np.linalg.norm(fo.reshape(-1, n_sc), axis=1)
        assert np.max(per_row) < 2e-3
    nrel = np.sqrt(err / ref)
    print(f"\nn_sc={n_sc}: tensor-core FFT vs FP64 DFT, norm-relative {nrel:.2e} ({20 * np.log10(nrel):.1f} dB)")
    assert nrel < 1e-3
    rx.close()


def test_tensor_core_fft_single_tones():
    cell, rx = _rx(3276, max_slots=1)
    n = np.arange(4096)
    x = np.zeros((1, 14, cell.n_rx, 4096), dtype=np.complex128)
    bins = {}
    for s in range(14):
        for r in range(cell.n_rx):
            k = (s * 613 + r * 97 + 5) % 4096
            bins[(s, r)] = k
            x[0, s, r] = 0.25 * np.exp(2j * np.pi * k * n / 4096)
    t16 = np.stack([x.real, x.imag], axis=-1).astype(np.float16)
    fg = _planes(rx.ofdm_fft(torch.from_numpy(t16).cuda())[0], 3276)
    torch.cuda.synchronize()
    for (s, r), k in bins.items():
        a = (k + 1638) % 4096
        row = fg[s, r]
        if a < 3276:
            assert abs(row[a] - 1024.0) < 2.0, (s, r, row[a])      # 4096 * 0.25 at the tone's bin
            rest = np.delete(row, a)
            assert np.max(np.abs(rest)) < 2.0
        else:                                                       # the tone is outside the active band
            assert np.max(np.abs(row)) < 2.0
    rx.close()


def test_tensor_core_fft_many_rows_equal_single_rows():
    """16 slots of 64 antennas (14,336 rows, several per persistent CTA) give the same rows as one slot at a
    time: each row's arithmetic does not depend on where it runs."""
    cell, rx = _rx(3276, n_rx=64, max_slots=16)
    rng = np.random.default_rng(7)
    t16 = (rng.standard_normal((16, 14, 64, 4096, 2)) * 0.02).astype(np.float16)
    td = torch.from_numpy(t16).cuda()
    full = rx.ofdm_fft(td)
    one = rx.ofdm_fft(td[5:6].contiguous())
    torch.cuda.synchronize()
    assert torch.equal(full[5], one[0])
    rx.close()
