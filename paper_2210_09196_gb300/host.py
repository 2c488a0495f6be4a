"""Host-side helpers around the binding: device buffers in the layouts of include/pusch.h and a small
``Receiver`` object owning one handle. Marshalling only -- no receive-chain arithmetic happens here.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def cfg_for(cell, form: int = B.PUSCH_FORM_FP32, noise_var: float | None = None, loading: float = 0.0,
            ports=None, chol_every: int = 0) -> B.pusch_cell_cfg:
    """pusch_cell_cfg for a generator CellConfig (paper_2210_09196_gb300.synth)."""
    nv = float(10.0 ** (-cell.snr_db / 10.0)) if noise_var is None else float(noise_var)
    return B.make_cfg(n_rx=cell.n_rx, n_fft=cell.n_fft, n_sc=cell.n_sc, n_beams=cell.n_beams,
                      n_layers=cell.n_layers, comb=cell.comb, ports=ports, qam_bits=cell.qam_bits,
                      in_fp16=cell.in_fp16, form=form, noise_var=nv, loading=loading, chol_every=chol_every,
                      cp=getattr(cell, "cp", False), shift_7p5khz=getattr(cell, "shift_7p5khz", False),
                      dmrs_type=1 if getattr(cell, "dmrs", "comb") == "type1" else 0)


def time_tensor(slots, device="cuda", pin=False) -> torch.Tensor:
    """Stack the slots' time samples: complex64 [n, S, R, N] or float16 [n, S, R, N, 2]."""
    arr = np.stack([s.time_in for s in slots])
    t = torch.from_numpy(arr)
    if device == "cpu":
        return t.pin_memory() if pin else t
    return t.to(device)


def pilot_tensor(slots, device="cuda", pin=False) -> torch.Tensor:
    t = torch.from_numpy(np.stack([s.pilots for s in slots]))
    if device == "cpu":
        return t.pin_memory() if pin else t
    return t.to(device)


def beam_tensor(W, device="cuda") -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(W, dtype=np.complex64)).to(device)


class Receiver:
    """One pusch handle plus the output buffers of the stage and chain entry points."""

    def __init__(self, cfg: B.pusch_cell_cfg, max_slots: int, device="cuda"):
        self.cfg = cfg
        self.max_slots = max_slots
        self.device = torch.device(device)
        self.h = B.pusch_create(cfg, max_slots)
        self.n_data = cfg.n_sym - 2
        self.pitch = B.pusch_sc_pitch(cfg)

    def close(self):
        if self.h:
            B.pusch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- buffer factories (layouts of include/pusch.h, leading [n_slots])
    def freq_buffer(self, n):
        c = self.cfg
        if c.form == B.PUSCH_FORM_FP8:   # E4M3 planes + block scales, one byte buffer (include/pusch.h)
            return torch.empty(B.pusch_freq_bytes(c, n), dtype=torch.uint8, device=self.device)
        if c.form == B.PUSCH_FORM_MIXED:
            return torch.empty((n, c.n_sym, c.n_rx, 2, self.pitch), dtype=torch.float16, device=self.device)
        return torch.empty((n, c.n_sym, c.n_rx, c.n_sc), dtype=torch.complex64, device=self.device)

    def beam_buffer(self, n):
        c = self.cfg
        return torch.empty((n, c.n_sym, c.n_sc, c.n_beams), dtype=torch.complex64, device=self.device)

    def H_buffer(self, n):
        c = self.cfg
        return torch.empty((n, c.n_sc, c.n_layers, c.n_beams), dtype=torch.complex64, device=self.device)

    def xhat_buffer(self, n, device=None):
        c = self.cfg
        return torch.empty((n, c.n_layers, self.n_data, c.n_sc), dtype=torch.complex64,
                           device=self.device if device is None else device)

    def bits_buffer(self, n, device=None):
        c = self.cfg
        return torch.empty((n, c.n_layers, self.n_data, c.n_sc), dtype=torch.uint8,
                           device=self.device if device is None else device)

    def status_buffer(self, device=None):
        return torch.zeros(4, dtype=torch.int32, device=self.device if device is None else device)

    # --- stage calls
    def ofdm_fft(self, time_in, freq=None, stream=None):
        n = time_in.shape[0]
        freq = self.freq_buffer(n) if freq is None else freq
        B.pusch_ofdm_fft(self.h, n, time_in, freq, stream)
        return freq

    def freq_slots(self, freq) -> int:
        """Slots held by an FFT output buffer (the FP8 form's byte buffer carries no slot dimension)."""
        if self.cfg.form != B.PUSCH_FORM_FP8:
            return freq.shape[0]
        for n in range(self.max_slots + 1):
            if B.pusch_freq_bytes(self.cfg, n) == freq.numel():
                return n
        raise ValueError("buffer size matches no slot count of this cell's FP8 layout")

    def beamform(self, freq, W, beam=None, stream=None):
        n = self.freq_slots(freq)
        beam = self.beam_buffer(n) if beam is None else beam
        B.pusch_beamform(self.h, n, freq, W, beam, stream)
        return beam

    def chest_ls(self, beam, pilots, H=None, stream=None):
        n = beam.shape[0]
        H = self.H_buffer(n) if H is None else H
        B.pusch_chest_ls(self.h, n, beam, pilots, H, stream)
        return H

    def set_pipeline(self, n_chunks: int):
        """Run pusch_slot / pusch_slot_host batches as n_chunks runs over two streams (1 = one run)."""
        B.pusch_set_pipeline(self.h, n_chunks)

    def noise_estimate(self, beam, pilots, stream=None):
        n = beam.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=self.device)
        B.pusch_noise_estimate(self.h, n, beam, pilots, out, stream)
        return out

    def mmse_detect(self, H, beam, stream=None):
        n = H.shape[0]
        x, b, st = self.xhat_buffer(n), self.bits_buffer(n), self.status_buffer()
        B.pusch_mmse_detect(self.h, n, H, beam, x, b, st, stream)
        return x, b, st

    def slot(self, time_in, W, pilots, out=None, stream=None):
        n = time_in.shape[0]
        x, b, st = (self.xhat_buffer(n), self.bits_buffer(n), self.status_buffer()) if out is None else out
        B.pusch_slot(self.h, n, time_in, W, pilots, x, b, st, stream)
        return x, b, st

    def slot_host(self, time_in_host, W, pilots_host, out_host, stream=None):
        x, b, st = out_host
        B.pusch_slot_host(self.h, time_in_host.shape[0], time_in_host, W, pilots_host, x, b, st, stream)
        return x, b, st


class RaggedReceiver:
    """One pusch_batch for a generated ragged multi-cell slot (synth.RaggedSlot) and its packed buffers."""

    def __init__(self, rs, form: int = B.PUSCH_FORM_MIXED, device="cuda"):
        self.cells = []
        for c in rs.cells:
            cfg = B.make_cfg(n_rx=c.n_rx, n_fft=c.n_fft, n_sc=c.n_sc, n_beams=c.n_beams, n_layers=1, comb=c.comb,
                             ports=[0], in_fp16=True, form=form, noise_var=c.noise_var)
            self.cells.append(cfg)
        self.users = [B.pusch_user_desc(u.cell, u.sc_start, u.sc_count, u.n_layers, u.port0, u.qam_bits)
                      for u in rs.users]
        self.h = B.pusch_batch_create(self.cells, self.users)
        self.sizes = B.pusch_batch_sizes(self.h)
        self.device = torch.device(device)
        self.n_data = 12

    def close(self):
        if self.h:
            B.pusch_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def pack(self, rs):
        """Concatenated device buffers (time_in, W, pilots) of a ragged slot."""
        t = torch.from_numpy(np.concatenate([x.reshape(-1, 2) for x in rs.time_in])).to(self.device)
        w = torch.from_numpy(np.concatenate([x.reshape(-1) for x in rs.W])).to(self.device)
        p = torch.from_numpy(np.concatenate([x.reshape(-1) for x in rs.pilots])).to(self.device)
        assert t.shape[0] == self.sizes[0] and w.numel() == self.sizes[1] and p.numel() == self.sizes[2]
        return t, w, p

    def outputs(self):
        x = torch.empty(self.sizes[3], dtype=torch.complex64, device=self.device)
        b = torch.empty(self.sizes[4], dtype=torch.uint8, device=self.device)
        s = torch.zeros(4, dtype=torch.int32, device=self.device)
        return x, b, s

    def run(self, t, w, p, out, stream=None):
        B.pusch_batch_run(self.h, t, w, p, *out, stream=stream)
        return out

    def autotune(self, t, w, p, out, cache_path=None, stream=None) -> int:
        """Times the batch's launch shapes on these buffers (or loads them from cache_path)."""
        return B.pusch_batch_autotune(self.h, t, w, p, *out, cache_path=cache_path, stream=stream)

    def tuning(self) -> dict:
        return B.pusch_batch_tuning(self.h, len(self.cells))

    def split(self, flat, rs):
        """Per-user [n_layers, 12, sc_count] views of a packed output."""
        res, o = [], 0
        for u in rs.users:
            n = u.n_layers * self.n_data * u.sc_count
            res.append(flat[o:o + n].reshape(u.n_layers, self.n_data, u.sc_count))
            o += n
        return res
