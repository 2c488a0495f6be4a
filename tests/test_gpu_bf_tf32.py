"""The plain FP32 form's beamforming on the tensor cores (three TF32 products per FP32 product, FP32 accumulation in
TMEM) against the FP64 oracle's Y = W^H X (Section II, Table I "BF"), through pusch_beamform.

Shapes cover one and several K chunks (16 antennas each), a ragged last subcarrier tile, 8 to 64 beams and the
deployment cell's 64 x 32 x 3276; inputs span several orders of magnitude across antennas, which a single TF32
product (10-bit mantissa) would resolve only to about 1e-3 but the split products hold to the FP32 bar (1e-5
norm-relative, and every beam row within 1e-5 of its own norm)."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_rx,n_beams,n_sc", [(16, 8, 8), (32, 24, 130), (48, 64, 1000), (128, 16, 777 * 2),
                                               (64, 32, 3276)], ids=lambda v: str(v))
def test_tf32_split_beamforming_at_fp32_parity(orc, n_rx, n_beams, n_sc):
    n = 2
    rng = np.random.default_rng(n_rx * 1000 + n_beams + n_sc)
    cell = synth.SMALL_FP32.with_(n_rx=n_rx, n_beams=n_beams, n_layers=min(4, n_beams), n_sc=n_sc,
                                  n_fft=4096 if n_sc > 2048 else 2048)
    rx = host.Receiver(host.cfg_for(cell), max_slots=n)
    scale = 10.0 ** rng.uniform(-3, 2, (1, 1, n_rx, 1))            # antenna powers over five decades
    X = (rng.standard_normal((n, 14, n_rx, n_sc)) + 1j * rng.standard_normal((n, 14, n_rx, n_sc))) * scale
    W = (rng.standard_normal((n_rx, n_beams)) + 1j * rng.standard_normal((n_rx, n_beams))) / np.sqrt(n_rx)
    freq = torch.from_numpy(X.astype(np.complex64)).cuda()
    beam = rx.beamform(freq, host.beam_tensor(W))
    torch.cuda.synchronize()
    Y = beam.cpu().numpy().astype(np.complex128)
    X32 = X.astype(np.complex64).astype(np.complex128)
    W32 = W.astype(np.complex64).astype(np.complex128)
    worst = 0.0
    for i in range(n):
        ref = orc.beamform(X32[i], W32)
        err = np.linalg.norm(Y[i] - ref) / np.linalg.norm(ref)
        row = np.abs(Y[i] - ref).max(axis=-1) / np.maximum(np.linalg.norm(ref, axis=-1), 1e-300)
        assert err < 1e-5, err
        assert row.max() < 1e-5, row.max()
        worst = max(worst, err)
    print(f"\nN_R={n_rx} N_B={n_beams} N_SC={n_sc}: norm-relative {worst:.2e}")
    rx.close()
