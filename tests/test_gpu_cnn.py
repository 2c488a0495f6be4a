"""Learned channel-estimate denoiser on the GPU: forward and backward kernels against the FP64 CNN oracle
(bfloat16 rounding emulated at the same points), Adam against its formula, training through the library
kernels, checkpoint resume, the LS fallback, and the post-MMSE EVM gain over plain LS."""
import math

import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import denoiser as D
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu


def nrel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def test_param_count():
    assert B.pusch_cnn_param_count() == D.PARAMS == 19682


@pytest.mark.parametrize("n,w", [(3, 37), (5, 300), (2, 256), (3, 264)])   # 256, 264: tensor-core 32 -> 32 layers
def test_forward_backward_match_oracle(orc, n, w):
    rng = np.random.default_rng(n * 1000 + w)
    p = D.init_params(seed=n)
    p[-(2 * 32 * 9 + 2):] *= 10.0                      # make the last layer matter
    x = rng.standard_normal((n, 2, 2, w)).astype(np.float32)
    tgt = rng.standard_normal((n, 2, 2, w)).astype(np.float32)
    dev = "cuda"
    pb = torch.from_numpy(p).to(dev).to(torch.bfloat16)
    xb = torch.from_numpy(x).to(dev).to(torch.bfloat16)
    y = torch.zeros((n, 2, 2, w), dtype=torch.float32, device=dev)
    acts = torch.zeros((3, n, 32, 2, w), dtype=torch.bfloat16, device=dev)
    B.pusch_cnn_forward(n, w, xb, pb, y, acts)
    grad = torch.zeros(D.PARAMS, dtype=torch.float32, device=dev)
    loss = torch.zeros(1, dtype=torch.float32, device=dev)
    work = torch.zeros(2 * n * 32 * 2 * w, dtype=torch.float32, device=dev)
    wflip = torch.zeros(D.PARAMS, dtype=torch.bfloat16, device=dev)
    tg = torch.from_numpy(tgt).to(dev)
    B.pusch_cnn_backward(n, w, xb, acts, pb, y, tg, grad, loss, work, wflip)
    torch.cuda.synchronize()
    yo, ao = orc.cnn_forward(p, x, bf16=True)
    assert nrel(y.cpu().numpy(), yo) < 2e-3
    assert nrel(acts.float().cpu().numpy(), ao) < 2e-3
    lo, go = orc.cnn_loss_grad(p, x, tgt, bf16=True)
    assert abs(float(loss) - lo) < 2e-3 * lo
    assert nrel(grad.cpu().numpy(), go) < 5e-3


def test_adam_matches_formula():
    dev = "cuda"
    rng = np.random.default_rng(3)
    p = rng.standard_normal(D.PARAMS).astype(np.float32)
    g = rng.standard_normal(D.PARAMS).astype(np.float32)
    m = rng.standard_normal(D.PARAMS).astype(np.float32) * 0.1
    v = np.abs(rng.standard_normal(D.PARAMS).astype(np.float32)) * 0.1
    P, G, Mt, V = (torch.from_numpy(a.copy()).to(dev) for a in (p, g, m, v))
    Pb = torch.zeros(D.PARAMS, dtype=torch.bfloat16, device=dev)
    B.pusch_cnn_adam(7, 1e-3, 0.9, 0.999, 1e-8, P, Pb, G, Mt, V)
    torch.cuda.synchronize()
    m2 = 0.9 * m + 0.1 * g
    v2 = 0.999 * v + 0.001 * g * g
    p2 = p - 1e-3 * (m2 / (1 - 0.9 ** 7)) / (np.sqrt(v2 / (1 - 0.999 ** 7)) + 1e-8)
    assert np.allclose(P.cpu().numpy(), p2, rtol=1e-5, atol=1e-7)
    # (1 - beta) is formed in float on the device, so the moments agree to float rounding
    assert np.allclose(Mt.cpu().numpy(), m2, rtol=1e-5, atol=1e-7) and np.allclose(V.cpu().numpy(), v2, rtol=1e-5,
                                                                                     atol=1e-7)
    assert torch.equal(Pb, P.to(torch.bfloat16))


@pytest.fixture(scope="module")
def trained(tmp_path_factory):
    gen = D.BeamDomainGenerator(seed=4)
    tr = D.Trainer(gen, slots_per_step=2, lr=2e-3, seed=0)
    before = tr.eval_loss(4)
    hist, secs = tr.fit(2500, log_every=100)
    after = tr.eval_loss(4)
    ck = tmp_path_factory.mktemp("ck") / "denoiser.pt"
    tr.save(ck)
    return tr, before, after, hist, ck


def test_training_reduces_loss(trained):
    tr, before, after, hist, _ = trained
    loss_cnn0, loss_ls = before
    loss_cnn1, loss_ls1 = after
    assert loss_cnn1 < 0.7 * loss_cnn0                 # learning happened
    assert loss_cnn1 < 0.8 * loss_ls1                   # and beats the interpolated LS grid it starts from
    assert all(np.isfinite(l) for _, l in hist)


def test_checkpoint_resumes(trained):
    tr, _, _, _, ck = trained
    tr2 = D.Trainer(D.BeamDomainGenerator(seed=9), slots_per_step=tr.n_slots, seed=123)
    tr2.load(ck)
    assert torch.equal(tr2.p, tr.p) and tr2.step == tr.step and torch.equal(tr2.pb, tr.pb)
    x = tr.x.clone()
    y1 = torch.zeros_like(tr.y)
    y2 = torch.zeros_like(tr.y)
    B.pusch_cnn_forward(tr.n, tr.gen.w, x, tr.pb, y1, tr.acts)
    B.pusch_cnn_forward(tr2.n, tr2.gen.w, x, tr2.pb, y2, tr2.acts)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    tr2.fit(5)
    assert tr2.step == tr.step + 5
    tr2.close()


def _chain(cell, seed=0):
    s = synth.make_slot(cell, seed)
    rx = host.Receiver(host.cfg_for(cell), max_slots=1)
    freq = rx.ofdm_fft(host.time_tensor([s]))
    beam = rx.beamform(freq, host.beam_tensor(s.W))
    pil = host.pilot_tensor([s])
    return s, rx, beam, pil


def test_identity_net_reproduces_ls_and_garbage_net_falls_back():
    cell = synth.DEPLOY.with_(n_rx=16, n_beams=16, n_layers=8, n_fft=1024, n_sc=600, snr_db=20.0)
    s, rx, beam, pil = _chain(cell)
    H_ls = rx.chest_ls(beam, pil)
    grids = cell.n_layers * cell.n_beams
    resid = torch.zeros(grids, device="cuda")
    flag = torch.zeros(grids, dtype=torch.uint8, device="cuda")
    zero = torch.zeros(D.PARAMS, dtype=torch.bfloat16, device="cuda")   # net = identity (residual only)
    H1 = rx.H_buffer(1)
    B.pusch_chest_cnn(rx.h, 1, beam, pil, zero, 2.0, H1, resid, flag)
    torch.cuda.synchronize()
    assert int(flag.sum()) == 0
    assert nrel(H1.cpu().numpy().view(np.float32), H_ls.cpu().numpy().view(np.float32)) < 1e-2
    assert float(resid.max()) < 0.6                    # the per-symbol LS rows against their own pilots
    garbage = (torch.randn(D.PARAMS, device="cuda") * 50).to(torch.bfloat16)
    H2 = rx.H_buffer(1)
    B.pusch_chest_cnn(rx.h, 1, beam, pil, garbage, 2.0, H2, resid, flag)
    torch.cuda.synchronize()
    assert int(flag.sum()) == grids                     # every grid falls back ...
    assert torch.equal(H2, H_ls)                        # ... to exactly the plain LS estimate
    rx.close()


def test_learned_estimator_gains_over_ls_after_mmse(trained):
    """Post-MMSE EVM against the transmitted symbols, learned vs plain LS estimator, same slots and kernels.
    At 0 dB the data-symbol noise dominates the EVM; from 10 dB the estimate does."""
    tr = trained[0]
    res = D.evaluate(tr.pb, [0.0, 10.0, 20.0], n_slots=1, kappa=2.0)
    assert res[0.0]["gain_db"] > 0.0, res
    assert res[10.0]["gain_db"] > 0.5 and res[20.0]["gain_db"] > 1.0, res
    for r in res.values():
        assert r["fallback_fraction"] < 0.2, res


def test_committed_weights_gain_over_ls():
    """The weight file trained on the generated-slot recipe (200k slot crops: delay spread 30-1000 ns, Doppler
    0-500 Hz, SNR -5..25 dB) improves the post-MMSE EVM over plain LS + interpolation on the evaluation cell
    (64 antennas, 32 beams, 16 layers, 16-QAM, 300 ns, 200 Hz Doppler), with few fallbacks."""
    from pathlib import Path
    path = Path(D.__file__).resolve().parent / "denoiser_c4.pt"
    if not path.exists():
        pytest.skip("no trained weight file")
    pb, meta = D.load_weights(path)
    assert meta["slots"] >= 200000
    res = D.evaluate(pb, [10.0, 20.0], n_slots=1, kappa=2.0)
    assert res[10.0]["gain_db"] > 1.0 and res[20.0]["gain_db"] > 2.0, res
    for r in res.values():
        assert r["fallback_fraction"] < 0.2, res
