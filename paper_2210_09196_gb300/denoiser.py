"""Training and use of the learned channel-estimate denoiser.

The network and every arithmetic step of training (forward, backward, Adam) run in libpusch's CUDA kernels
(pusch_cnn_forward / pusch_cnn_backward / pusch_cnn_adam). Its inputs are built by pusch_ls_grid, the same
kernel the receiver uses, from DMRS observations produced by a seeded beam-domain channel generator
(``BeamDomainGenerator``, transmitter/channel side only, in torch on the GPU for volume):

  * per (beam, layer) an independent channel with an exponential power-delay profile of 16 taps spanning
    three times a delay spread drawn from 30-1000 ns, each tap a Rayleigh fading process built as a sum of
    16 sinusoids with uniformly random arrival angles and phases (Clarke/Jakes Doppler spectrum; maximum
    Doppler drawn from 0-500 Hz), evaluated at the two DMRS symbols (symbols 2 and 11 of a 30 kHz slot);
  * QPSK pilots on a comb of 16 (layer l on subcarriers a % 16 == l), AWGN at an SNR drawn from -5..25 dB;
  * the target is the true channel at both DMRS symbols, in the grid's normalised units.

Checkpoints are torch files holding a version, the FP32 master parameters, the Adam moments, the step and
the generator seed; training resumes from them.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import binding as B

PARAMS = 19682
CH = (2, 32, 32, 32, 2)
_SYM_S = 1.0 / 30e3 * (1 + 0.0703125)   # OFDM symbol duration incl. the normal cyclic prefix (30 kHz)
_DMRS = (2, 11)


def init_params(seed: int = 0) -> np.ndarray:
    """He-normal weights, zero biases; the last layer is scaled by 0.1 so the net starts near identity."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(4):
        cin, cout = CH[k], CH[k + 1]
        w = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (cin * 9))
        if k == 3:
            w *= 0.1
        out += [w.ravel(), np.zeros(cout)]
    p = np.concatenate(out).astype(np.float32)
    assert p.size == PARAMS
    return p


class BeamDomainGenerator:
    """Seeded beam-domain DMRS observations for denoiser training (no receiver arithmetic)."""

    def __init__(self, width: int = 256, n_layers: int = 16, n_beams: int = 16, seed: int = 4, device="cuda",
                 snr_db=(-5.0, 25.0), delay_spread_s=(30e-9, 1000e-9), doppler_hz=(0.0, 500.0), n_fft: int = 4096,
                 scs_hz: float = 30e3):
        self.w, self.L, self.B = width, n_layers, n_beams
        self.dev = torch.device(device)
        self.g = torch.Generator(device=self.dev)
        self.g.manual_seed(seed)
        self.seed = seed
        self.snr, self.ds, self.fd = snr_db, delay_spread_s, doppler_hz
        self.ts = 1.0 / (n_fft * scs_hz)
        self.n_fft = n_fft

    def _u(self, shape, lo, hi):
        return lo + (hi - lo) * torch.rand(shape, generator=self.g, device=self.dev)

    def _n(self, shape):
        return torch.randn(shape, generator=self.g, device=self.dev)

    def batch(self, n_slots: int):
        """-> beam [n, 14, w, B] c64 (only the DMRS symbols filled), pilots [n, L, 2, w] c64,
        H [n, L, B, 2, w] c64 (true channel at the two DMRS symbols), noise variance per slot [n]."""
        n, w, L, Bm = n_slots, self.w, self.L, self.B
        taps = 16
        G = (n, L, Bm)
        tau = self._u(G, *self.ds)                                            # delay spread per grid
        step = 3.0 * tau / (taps - 1)                                         # tap spacing
        i = torch.arange(taps, device=self.dev, dtype=torch.float32)
        delay = torch.round(i * step[..., None] / self.ts)                    # samples
        pw = torch.exp(-i * step[..., None] / tau[..., None])
        pw = pw / pw.sum(-1, keepdim=True)
        fd = self._u(G, *self.fd)
        M = 16
        alpha = self._u(G + (taps, M), 0.0, 2 * math.pi)
        phi = self._u(G + (taps, M), 0.0, 2 * math.pi)
        t = torch.tensor([s * _SYM_S for s in _DMRS], device=self.dev)
        arg = 2 * math.pi * fd[..., None, None, None] * torch.cos(alpha)[..., None] * t + phi[..., None]
        h = torch.exp(1j * arg).sum(-2) / math.sqrt(M)                        # [n, L, B, taps, 2]
        h = h * torch.sqrt(pw)[..., None]
        off = torch.randint(0, self.n_fft - w, (n, 1, 1, 1, 1), generator=self.g, device=self.dev)
        a = torch.arange(w, device=self.dev)
        k = (a + off).float()                                                 # [n,1,1,1,w]
        ph = torch.exp(-2j * math.pi * delay[..., None] * k / self.n_fft)   # [n, L, B, taps, w]
        H = torch.einsum("nlbts,nlbtw->nlbsw", h.to(torch.complex64), ph.to(torch.complex64))  # [n,L,B,2,w]
        snr = self._u((n,), *self.snr)
        nv = 10.0 ** (-snr / 10.0)
        bits = torch.randint(0, 2, (n, L, 2, w, 2), generator=self.g, device=self.dev).float()
        p = ((1 - 2 * bits[..., 0]) + 1j * (1 - 2 * bits[..., 1])) / math.sqrt(2.0)
        comb = (a[None, :] % L) == torch.arange(L, device=self.dev)[:, None]  # [L, w]
        p = (p * comb[None, :, None, :]).to(torch.complex64)                  # [n, L, 2, w]
        # subcarrier a carries layer a % L's pilot
        lay = a % L
        Hs = H.permute(0, 3, 4, 1, 2)                                         # [n, 2, w, L, B]
        Hsel = Hs[:, :, a, lay, :]                                            # [n, 2, w, B]
        psel = p.permute(0, 2, 3, 1)[:, :, a, lay]                             # [n, 2, w]
        noise = (self._n((n, 2, w, Bm)) + 1j * self._n((n, 2, w, Bm))) * torch.sqrt(nv / 2)[:, None, None, None]
        y = Hsel * psel[..., None] + noise.to(torch.complex64)
        beam = torch.zeros((n, 14, w, Bm), dtype=torch.complex64, device=self.dev)
        beam[:, _DMRS[0]] = y[:, 0]
        beam[:, _DMRS[1]] = y[:, 1]
        return beam, p.contiguous(), H.contiguous(), nv


class Trainer:
    """Adam on the FP32 master parameters; forward, backward and the update run in libpusch kernels."""

    def __init__(self, gen: BeamDomainGenerator, slots_per_step: int = 1, lr: float = 1e-3, seed: int = 0,
                 device="cuda"):
        self.gen, self.n_slots, self.lr = gen, slots_per_step, lr
        self.dev = torch.device(device)
        L, Bm, w = gen.L, gen.B, gen.w
        cfg = B.make_cfg(n_rx=Bm, n_fft=max(64, 1 << (w - 1).bit_length()), n_sc=w, n_beams=Bm, n_layers=L, comb=L,
                         noise_var=1.0)
        self.h = B.pusch_create(cfg, slots_per_step)
        self.n = slots_per_step * L * Bm
        n = self.n
        self.p = torch.from_numpy(init_params(seed)).to(self.dev)
        self.pb = self.p.to(torch.bfloat16)
        self.m = torch.zeros_like(self.p)
        self.v = torch.zeros_like(self.p)
        self.grad = torch.zeros_like(self.p)
        self.wflip = torch.zeros(PARAMS, dtype=torch.bfloat16, device=self.dev)
        self.x = torch.zeros((n, 2, 2, w), dtype=torch.bfloat16, device=self.dev)
        self.scale = torch.zeros(n, dtype=torch.float32, device=self.dev)
        self.y = torch.zeros((n, 2, 2, w), dtype=torch.float32, device=self.dev)
        self.acts = torch.zeros((3, n, 32, 2, w), dtype=torch.bfloat16, device=self.dev)
        self.work = torch.zeros(2 * n * 32 * 2 * w, dtype=torch.float32, device=self.dev)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.dev)
        self.step = 0

    def close(self):
        if self.h:
            B.pusch_destroy(self.h)
            self.h = None

    def make_batch(self):
        """(grid, target) of one step: the receiver's LS grid and the true channel in its units."""
        beam, pil, H, _ = self.gen.batch(self.n_slots)
        B.pusch_ls_grid(self.h, self.n_slots, beam, pil, self.x, self.scale)
        # target [slot, L, B, ch, row, w] in the grid's units (divide by the grid's scale)
        T = H / self.scale.view(self.n_slots, self.gen.L, self.gen.B, 1, 1)
        tgt = torch.stack([T.real, T.imag], dim=3).reshape(self.n, 2, 2, self.gen.w).contiguous()
        return tgt

    def train_step(self, lr=None):
        tgt = self.make_batch()
        n, w = self.n, self.gen.w
        B.pusch_cnn_forward(n, w, self.x, self.pb, self.y, self.acts)
        B.pusch_cnn_backward(n, w, self.x, self.acts, self.pb, self.y, tgt, self.grad, self.loss, self.work, self.wflip)
        self.step += 1
        B.pusch_cnn_adam(self.step, self.lr if lr is None else lr, 0.9, 0.999, 1e-8, self.p, self.pb, self.grad, self.m,
                         self.v)
        return self.loss

    def eval_loss(self, n_batches: int = 4):
        """Mean loss of the current net and of the plain per-symbol LS grid (identity) on fresh batches."""
        n, w = self.n, self.gen.w
        tot = ident = 0.0
        for _ in range(n_batches):
            tgt = self.make_batch()
            B.pusch_cnn_forward(n, w, self.x, self.pb, self.y, self.acts)
            torch.cuda.synchronize()
            tot += float(((self.y - tgt) ** 2).mean())
            ident += float(((self.x.float() - tgt) ** 2).mean())
        return tot / n_batches, ident / n_batches

    def fit(self, steps: int, log_every: int = 0):
        hist = []
        t0 = time.time()
        for k in range(steps):
            lr = self.lr * 0.5 * (1 + math.cos(math.pi * min(1.0, self.step / max(steps, 1))))
            loss = self.train_step(lr)
            if log_every and (k % log_every == 0 or k == steps - 1):
                hist.append((self.step, float(loss)))
        torch.cuda.synchronize()
        return hist, time.time() - t0

    def state(self):
        return {"version": 1, "params": self.p.cpu(), "m": self.m.cpu(), "v": self.v.cpu(), "step": self.step,
                "gen_seed": self.gen.seed}

    def save(self, path):
        torch.save(self.state(), path)

    def load(self, path):
        st = torch.load(path, map_location="cpu")
        if st.get("version") != 1 or st["params"].numel() != PARAMS:
            raise ValueError("not a denoiser checkpoint of this version")
        self.p.copy_(st["params"].to(self.dev))
        self.pb.copy_(self.p.to(torch.bfloat16))
        self.m.copy_(st["m"].to(self.dev))
        self.v.copy_(st["v"].to(self.dev))
        self.step = int(st["step"])


def evaluate(params_bf16, snrs_db, n_slots: int = 2, kappa: float = 2.0, cell=None, device="cuda"):
    """Post-MMSE EVM (vs the transmitted symbols) of the plain LS estimator and of the learned estimator on
    the same slots of the evaluation cell (default synth.DENOISE_EVAL: 64 antennas, 32 DFT beams, 16 layers,
    4096-point FFT, 3276 subcarriers, 16-QAM, 300 ns delay spread, 200 Hz Doppler), per SNR.
    Both paths share the FFT, beamforming and MMSE kernels; only the estimator differs."""
    from . import host, synth
    cell = synth.DENOISE_EVAL if cell is None else cell
    out = {}
    for snr in snrs_db:
        c = cell.with_(snr_db=float(snr))
        rx = host.Receiver(host.cfg_for(c, B.PUSCH_FORM_FP32), max_slots=1, device=device)
        e_ls = e_cnn = ref = 0.0
        fb = []
        for k in range(n_slots):
            s = synth.make_slot(c, 1000 + k)
            freq = rx.ofdm_fft(host.time_tensor([s], device))
            beam = rx.beamform(freq, host.beam_tensor(s.W, device))
            pil = host.pilot_tensor([s], device)
            H_ls = rx.chest_ls(beam, pil)
            x_ls, _, _ = rx.mmse_detect(H_ls, beam)
            H_c = rx.H_buffer(1)
            grids = c.n_layers * c.n_beams
            resid = torch.zeros(grids, dtype=torch.float32, device=device)
            flag = torch.zeros(grids, dtype=torch.uint8, device=device)
            B.pusch_chest_cnn(rx.h, 1, beam, pil, params_bf16, kappa, H_c, resid, flag)
            x_c, _, _ = rx.mmse_detect(H_c, beam)
            torch.cuda.synchronize()
            truth = s.x
            e_ls += float(np.sum(np.abs(x_ls[0].cpu().numpy() - truth) ** 2))
            e_cnn += float(np.sum(np.abs(x_c[0].cpu().numpy() - truth) ** 2))
            ref += float(np.sum(np.abs(truth) ** 2))
            fb.append(float(flag.float().mean()))
        rx.close()
        evm_ls, evm_cnn = 10 * np.log10(e_ls / ref), 10 * np.log10(e_cnn / ref)
        out[float(snr)] = {"evm_ls_db": round(evm_ls, 2), "evm_cnn_db": round(evm_cnn, 2),
                           "gain_db": round(evm_ls - evm_cnn, 2), "fallback_fraction": round(float(np.mean(fb)), 4)}
    return out


def save_weights(tr: "Trainer", path, slots_trained: int, seconds: float) -> None:
    """The trained network for use: FP32 parameters and how they were made (no optimiser state)."""
    torch.save({"version": 1, "params": tr.p.cpu(), "step": tr.step, "slots": int(slots_trained),
                "slots_per_step": tr.n_slots, "gen_seed": tr.gen.seed, "seconds": round(float(seconds), 1),
                "recipe": {"width": tr.gen.w, "layers": tr.gen.L, "beams": tr.gen.B, "snr_db": list(tr.gen.snr),
                           "delay_spread_s": list(tr.gen.ds), "doppler_hz": list(tr.gen.fd)}}, path)


def load_weights(path, device="cuda"):
    """(bfloat16 parameters on the device, metadata) of a file written by save_weights."""
    st = torch.load(path, map_location="cpu")
    if st.get("version") != 1 or st["params"].numel() != PARAMS:
        raise ValueError("not a denoiser weight file of this version")
    meta = {k: v for k, v in st.items() if k != "params"}
    return st["params"].to(device).to(torch.bfloat16), meta


def train(slots: int, slots_per_step: int = 8, lr: float = 2e-3, seed: int = 4, checkpoint=None,
          checkpoint_every: int = 2000, resume: bool = False, log_every: int = 1000):
    """Trains on `slots` generated slot crops (each: 16 layers x 16 beams of 256 subcarriers, fresh channel, delay
    spread, Doppler and SNR draws), slots_per_step per Adam step with a cosine learning-rate decay; checkpoints
    (optimiser state included) every checkpoint_every steps and resumes from `checkpoint` when resume is set."""
    gen = BeamDomainGenerator(seed=seed)
    tr = Trainer(gen, slots_per_step=slots_per_step, lr=lr, seed=0)
    steps = max(1, slots // slots_per_step)
    if resume and checkpoint is not None:
        import os
        if os.path.exists(checkpoint):
            tr.load(checkpoint)
            # the generator resumes at a fresh seed derived from the step, so no draw repeats
            tr.gen.g.manual_seed(seed * 1000003 + tr.step)
    t0 = time.time()
    hist = []
    while tr.step < steps:
        lr_t = tr.lr * 0.5 * (1 + math.cos(math.pi * tr.step / steps))
        loss = tr.train_step(lr_t)
        if log_every and tr.step % log_every == 0:
            hist.append((tr.step, float(loss)))
            print(f"step {tr.step}/{steps} loss {float(loss):.5f} {time.time() - t0:.0f} s", flush=True)
        if checkpoint is not None and tr.step % checkpoint_every == 0:
            tr.save(checkpoint)
    torch.cuda.synchronize()
    return tr, hist, time.time() - t0


def _main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="train or evaluate the learned channel-estimate denoiser")
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--slots", type=int, default=200000)
    t.add_argument("--slots-per-step", type=int, default=8)
    t.add_argument("--lr", type=float, default=2e-3)
    t.add_argument("--seed", type=int, default=4)
    t.add_argument("--out", required=True)
    t.add_argument("--checkpoint", default=None)
    t.add_argument("--resume", action="store_true")
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", required=True)
    e.add_argument("--snr", type=float, nargs="+", default=[-5.0, 0.0, 10.0, 20.0, 25.0])
    e.add_argument("--slots", type=int, default=2)
    a = ap.parse_args(argv)
    if a.cmd == "train":
        tr, hist, secs = train(a.slots, a.slots_per_step, a.lr, a.seed, a.checkpoint, resume=a.resume)
        save_weights(tr, a.out, tr.step * tr.n_slots, secs)
        loss, ident = tr.eval_loss(8)
        print(f"trained {tr.step} steps ({tr.step * tr.n_slots} slots) in {secs:.0f} s; loss {loss:.5f}, "
              f"per-symbol LS grid {ident:.5f}", flush=True)
        tr.close()
    else:
        pb, meta = load_weights(a.weights)
        import json
        print(json.dumps({"weights": meta, "evm": evaluate(pb, a.snr, n_slots=a.slots)}), flush=True)


if __name__ == "__main__":
    _main()
