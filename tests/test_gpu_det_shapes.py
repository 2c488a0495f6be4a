"""The detector's launch shapes (warps per CTA of the 12-data-symbol kernels, chosen by pusch_autotune or read
from its cache) against each other and against the FP64 oracle (Eq. 2 by Cholesky and two triangular solves,
Section V-C).

Every layer class (2, 4, 8, 16, 32 lanes per subcarrier) runs each of its warp counts on slots whose subcarrier
count is not a multiple of any CTA's subcarrier block, so that the last CTA is ragged and CTAs straddle slot
boundaries. The outputs must be bit-identical across the warp counts (each subcarrier's arithmetic does not
depend on where it runs) and within the FP32 form's 1e-5 norm-relative bar of the oracle."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

SIGMA2 = 0.05


def _case(nl, nb, n_sc, slots, seed):
    rng = np.random.default_rng(seed)
    H = (rng.standard_normal((slots, n_sc, nl, nb)) + 1j * rng.standard_normal((slots, n_sc, nl, nb))) / np.sqrt(2)
    y = (rng.standard_normal((slots, 14, n_sc, nb)) + 1j * rng.standard_normal((slots, 14, n_sc, nb))) / np.sqrt(2)
    return H.astype(np.complex64), y.astype(np.complex64)


def _warp_choices(nl, nb):
    """The default warps per CTA of a layer class, then the other counts of 1, 2, 4 and 8 whose tiles fit."""
    default = 4 if nl == 32 else 1
    ht = max(nl * ((nb + 3) & ~1), nl * (nl + 1) + nl // 2)
    ht += (2 - ht) & 15
    ys = nl if nl >= 16 and ((nb + 3) & ~1) < nl else (nb + 3) & ~1
    per_warp = (32 // nl) * (ht + 12 * ys) * 8
    return [default] + [w for w in (1, 2, 4, 8) if w != default and w * per_warp <= 227 * 1024]


@pytest.mark.parametrize("nl,nb,n_sc", [(2, 8, 77), (2, 64, 29), (4, 16, 301), (8, 16, 123), (8, 64, 31), (16, 32, 301), (16, 64, 45),
                                         (32, 48, 37), (32, 64, 41)], ids=lambda v: str(v))
def test_detector_warp_counts_bit_identical_and_at_parity(tmp_path, orc, nl, nb, n_sc):
    slots = 3
    H, y = _case(nl, nb, n_sc, slots, seed=nl * 1000 + nb + n_sc)
    cell = synth.SMALL_FP32.with_(n_rx=nb, n_beams=nb, n_layers=nl, n_sc=n_sc, n_fft=512 if n_sc <= 512 else 4096,
                                  qam_bits=4)
    cfg = host.cfg_for(cell, noise_var=SIGMA2)
    Hd, yd = torch.from_numpy(H).cuda(), torch.from_numpy(y).cuda()
    outs = {}
    for w in _warp_choices(nl, nb):
        rx = host.Receiver(cfg, max_slots=slots)
        cache = tmp_path / f"tune_{w}.txt"
        cache.write_text(f"slot-det form={B.PUSCH_FORM_FP32} n_layers={nl} n_beams={nb} n_sc={n_sc} slots={slots}"
                         f" | warps={w} ms=0\n")
        B.pusch_autotune(rx.h, cache)
        x, b, st = rx.mmse_detect(Hd, yd)
        torch.cuda.synchronize()
        outs[w] = (x.cpu(), b.cpu(), st.cpu())
        rx.close()
    ws = list(outs)
    for w in ws[1:]:
        assert torch.equal(outs[w][0], outs[ws[0]][0]), (ws[0], w)
        assert torch.equal(outs[w][1], outs[ws[0]][1]), (ws[0], w)
        assert torch.equal(outs[w][2], outs[ws[0]][2]), (ws[0], w)
    x = outs[ws[0]][0].numpy().astype(np.complex128)
    assert int(outs[ws[0]][2].numpy()[0]) == 0
    err = ref = 0.0
    for s in range(slots):
        xo, fails = orc.mmse(H[s].astype(np.complex128), y[s].astype(np.complex128), SIGMA2)
        assert fails == 0
        err += np.sum(np.abs(x[s] - xo) ** 2)
        ref += np.sum(np.abs(xo) ** 2)
    nrel = np.sqrt(err / ref)
    print(f"\nN_L={nl} N_B={nb} n_sc={n_sc}: warps per CTA {ws}, norm-relative error {nrel:.2e}")
    assert nrel <= 1e-5
