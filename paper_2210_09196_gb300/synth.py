"""Seeded synthetic PUSCH slots (transmitter + channel side only).

This module produces the inputs of the receive chain of "Efficient Parallelization of 5G-PUSCH on a Scalable
RISC-V Many-core Processor" (arXiv 2210.09196): time-domain samples per (symbol, antenna), the beam matrix W,
the DMRS pilots and the noise variance, plus the ground truth (channel, symbols, bits) for quality metrics.

It holds none of the receiver's arithmetic: no FFT of received samples, no beamforming, no channel
estimation, no detection and no demapping. The transmitter's OFDM modulation uses ``numpy.fft.ifft``.
Both the CUDA path and the FP64 oracle consume exactly the arrays returned here.

Model (Section II, Eq. 1, Fig. 2):
  * OFDMA grid of N_SC active subcarriers x 14 symbols, block-type DMRS on symbols 2 and 11 (two whole
    pilot OFDM symbols per slot, Section II); the 12 remaining symbols carry data.
  * Active subcarrier a sits at FFT bin (a - N_SC//2) mod N_F (centred band, DC included, no CP).
  * N_L single-layer users; user l sends its QPSK pilot on the subcarriers a with a % comb == port[l]
    (frequency comb of size comb = N_L) and nothing on the other REs of the DMRS symbols.
  * Antenna-domain received RE: X[s, r, a] = sum_l Hant[a, r, l] t_l[s, a] + n,  n ~ CN(0, sigma^2),
    sigma^2 = 10^(-SNR/10) with unit-variance channel entries and unit-energy symbols.
  * Time samples: x[s, r, :] = ifft(spectrum) (numpy's 1/N_F normalisation), so the receiver's
    unnormalised forward FFT returns X exactly; optionally rounded to complex FP16.
  * Beam matrix W [N_R, N_B]: identity, or DFT columns W[r, b] = exp(-2 pi i r b / N_R) / sqrt(N_R).
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass, field

import numpy as np

N_SYM = 14
DMRS_SYMBOLS = (2, 11)
DATA_SYMBOLS = tuple(s for s in range(N_SYM) if s not in DMRS_SYMBOLS)

_SCS_HZ = 30e3


@dataclass(frozen=True)
class CellConfig:
    """One cell's slot shape. Names follow the paper's notation (N_R, N_SC, N_B, N_L)."""

    name: str
    n_rx: int            # N_R receive antennas
    n_fft: int           # N_F FFT size
    n_sc: int            # N_SC active subcarriers
    n_beams: int         # N_B beams
    n_layers: int        # N_L single-layer users detected jointly
    qam_bits: int        # 2 = QPSK, 4 = 16-QAM
    snr_db: float
    channel: str         # "iid" (CN(0,1) per subcarrier), "flat" (CN(0,1), same on every subcarrier)
                         # or "pdp" (16-tap exponential power-delay profile)
    beam: str            # "identity" or "dft"
    in_fp16: bool        # time samples stored as complex FP16
    delay_spread_s: float = 300e-9
    n_taps: int = 16
    tap_spacing_s: float = 60e-9
    doppler_hz: float = 0.0  # > 0: each tap fades over the slot (sum of 16 sinusoids, Clarke/Jakes spectrum)
    seed: int = 0
    dmrs: str = "comb"       # "comb": layer l's QPSK pilots on subcarriers a % n_layers == l (seeded draws);
                             # "type1": 3GPP type-1 DMRS, ports 0..3 (n_layers <= 4), Gold sequence of (n_id, n_scid)
    n_id: int = 0
    n_scid: int = 0
    cp: bool = False         # time input as one stream per antenna with NR normal cyclic prefixes
    shift_7p5khz: bool = False  # spectrum shifted up by 7.5 kHz (a quarter subcarrier) before transmission

    @property
    def comb(self) -> int:
        return self.n_layers

    def with_(self, **kw) -> "CellConfig":
        return dataclasses.replace(self, **kw)


# Workload presets. Sizes follow the paper's use case (Section II: 100 MHz, 30 kHz SCS, 3276 subcarriers,
# 14 symbols, 2 pilot symbols, 64 antennas, 32 beams) and the small/massive variants around it.
SMALL_FP32 = CellConfig("small-16rx-512fft-4ue", n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4,
                        qam_bits=2, snr_db=20.0, channel="iid", beam="identity", in_fp16=False, seed=1)
DEPLOY = CellConfig("deploy-64rx-4096fft-32beam-16ue", n_rx=64, n_fft=4096, n_sc=3276, n_beams=32,
                    n_layers=16, qam_bits=4, snr_db=30.0, channel="pdp", beam="dft", in_fp16=True, seed=2)
MASSIVE = CellConfig("massive-256rx-4096fft-64beam-32ue", n_rx=256, n_fft=4096, n_sc=3276, n_beams=64,
                     n_layers=32, qam_bits=4, snr_db=25.0, channel="pdp", beam="dft", in_fp16=True, seed=5)

# Evaluation cell of the learned estimator (the deployment cell with a fading channel): 300 ns delay
# spread, 200 Hz maximum Doppler; the SNR is swept by the caller.
DENOISE_EVAL = DEPLOY.with_(name="denoise-64rx-4096fft-32beam-16ue-doppler", doppler_hz=200.0, seed=4)

PRESETS = {"small": SMALL_FP32, "deploy": DEPLOY, "massive": MASSIVE, "denoise": DENOISE_EVAL}


def active_bins(n_sc: int, n_fft: int) -> np.ndarray:
    """FFT bin of each active subcarrier a: (a - n_sc//2) mod n_fft."""
    a = np.arange(n_sc)
    return (a - n_sc // 2) % n_fft


def beam_matrix(cfg: CellConfig) -> np.ndarray:
    """W [N_R, N_B] complex64: identity, or the first N_B orthonormal DFT columns."""
    if cfg.beam == "identity":
        if cfg.n_beams != cfg.n_rx:
            raise ValueError("identity beamforming needs n_beams == n_rx")
        return np.eye(cfg.n_rx, dtype=np.complex64)
    r = np.arange(cfg.n_rx)[:, None]
    b = np.arange(cfg.n_beams)[None, :]
    return (np.exp(-2j * np.pi * r * b / cfg.n_rx) / np.sqrt(cfg.n_rx)).astype(np.complex64)


def qam_map(bits: np.ndarray, qam_bits: int) -> np.ndarray:
    """Gray mapping of 3GPP TS 38.211 5.1.3 (QPSK) / 5.1.4 (16-QAM); bits[..., q] -> complex128."""
    b = bits.astype(np.int64)
    if qam_bits == 2:
        return ((1 - 2 * b[..., 0]) + 1j * (1 - 2 * b[..., 1])) / np.sqrt(2.0)
    if qam_bits == 4:
        re = (1 - 2 * b[..., 0]) * (2 - (1 - 2 * b[..., 2]))
        im = (1 - 2 * b[..., 1]) * (2 - (1 - 2 * b[..., 3]))
        return (re + 1j * im) / np.sqrt(10.0)
    raise ValueError("qam_bits must be 2 or 4")


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """bits[..., q] (0/1) -> one byte per symbol, bit j of the byte = b_j."""
    q = bits.shape[-1]
    out = np.zeros(bits.shape[:-1], dtype=np.uint8)
    for j in range(q):
        out |= (bits[..., j].astype(np.uint8) << j)
    return out


def _channel(cfg: CellConfig, rng: np.random.Generator) -> np.ndarray:
    """Antenna-domain channel Hant [N_SC, N_R, N_L] complex128, unit average power per entry."""
    R, L, n_sc = cfg.n_rx, cfg.n_layers, cfg.n_sc
    if cfg.channel == "iid":
        return (rng.standard_normal((n_sc, R, L)) + 1j * rng.standard_normal((n_sc, R, L))) / np.sqrt(2.0)
    if cfg.channel == "flat":
        h = (rng.standard_normal((R, L)) + 1j * rng.standard_normal((R, L))) / np.sqrt(2.0)
        return np.broadcast_to(h, (n_sc, R, L)).copy()
    if cfg.channel == "pdp":
        ts = 1.0 / (cfg.n_fft * _SCS_HZ)
        i = np.arange(cfg.n_taps)
        delays = np.round(i * cfg.tap_spacing_s / ts)                      # samples
        power = np.exp(-i * cfg.tap_spacing_s / cfg.delay_spread_s)
        power = power / power.sum()
        taps = (rng.standard_normal((R, L, cfg.n_taps)) + 1j * rng.standard_normal((R, L, cfg.n_taps)))
        taps *= np.sqrt(power / 2.0)
        k = (np.arange(n_sc) - n_sc // 2)[:, None]                       # signed frequency index
        F = np.exp(-2j * np.pi * k * delays[None, :] / cfg.n_fft)         # [N_SC, taps]
        return np.einsum("at,rlt->arl", F, taps)
    raise ValueError(f"unknown channel model {cfg.channel}")


_SYM_S = 1.0 / _SCS_HZ * (1 + 0.0703125)  # OFDM symbol duration with the normal cyclic prefix


def _channel_per_symbol(cfg: CellConfig, rng: np.random.Generator):
    """Time-varying PDP channel: list of 14 arrays Hant_s [N_SC, R, L]. Tap i of (r, l) is
    sqrt(p_i / M) sum_m exp(j (2 pi f_d cos(alpha_m) t + phi_m)) with uniformly random alpha, phi (M = 16)."""
    R, L, n_sc = cfg.n_rx, cfg.n_layers, cfg.n_sc
    ts = 1.0 / (cfg.n_fft * _SCS_HZ)
    i = np.arange(cfg.n_taps)
    delays = np.round(i * cfg.tap_spacing_s / ts)
    power = np.exp(-i * cfg.tap_spacing_s / cfg.delay_spread_s)
    power = power / power.sum()
    M = 16
    alpha = rng.uniform(0, 2 * np.pi, (R, L, cfg.n_taps, M))
    phi = rng.uniform(0, 2 * np.pi, (R, L, cfg.n_taps, M))
    k = (np.arange(n_sc) - n_sc // 2)[:, None]
    F = np.exp(-2j * np.pi * k * delays[None, :] / cfg.n_fft)                   # [N_SC, taps]
    out = []
    for s in range(N_SYM):
        t = s * _SYM_S
        taps = np.exp(1j * (2 * np.pi * cfg.doppler_hz * np.cos(alpha) * t + phi)).sum(-1) / np.sqrt(M)
        taps = taps * np.sqrt(power)                                              # [R, L, taps]
        out.append(np.matmul(F, taps.reshape(R * L, -1).T).reshape(n_sc, R, L))
    return out


@dataclass
class Slot:
    cfg: CellConfig
    time_in: np.ndarray      # [S, N_R, N_F] complex64, or [S, N_R, N_F, 2] float16 when cfg.in_fp16; with cfg.cp
                             # one stream per antenna, [N_R, slot_len] (or [N_R, slot_len, 2])
    W: np.ndarray            # [N_R, N_B] complex64
    pilots: np.ndarray       # [N_L, 2, N_SC] complex64 (zero off the layer's comb)
    ports: np.ndarray        # [N_L] int32 comb offsets
    noise_var: float
    H_beam: np.ndarray = field(repr=False)   # truth: [N_SC, N_L, N_B] complex128 = (W^H Hant)^T per subcarrier
    x: np.ndarray = field(repr=False)        # truth: [N_L, 12, N_SC] complex128 transmitted data symbols
    bits: np.ndarray = field(repr=False)     # truth: [N_L, 12, N_SC] uint8 packed (bit j = b_j)

    def time_as_complex128(self) -> np.ndarray:
        """The exact values the receiver sees, widened to complex128."""
        t = self.time_in
        if t.dtype == np.float16:
            return t[..., 0].astype(np.float64) + 1j * t[..., 1].astype(np.float64)
        return t.astype(np.complex128)


def make_slot(cfg: CellConfig, slot_index: int = 0, seed: int | None = None) -> Slot:
    """Generate one slot deterministically from (seed, slot_index)."""
    rng = np.random.default_rng([cfg.seed if seed is None else seed, slot_index])
    R, L, n_sc, N = cfg.n_rx, cfg.n_layers, cfg.n_sc, cfg.n_fft
    q = cfg.qam_bits
    if L > cfg.n_beams:
        raise ValueError("more layers than beams")
    comb = cfg.comb
    ports = np.arange(L, dtype=np.int32) % comb

    if cfg.doppler_hz > 0 and cfg.channel == "pdp":
        Hsym = _channel_per_symbol(cfg, rng)                             # 14 x [N_SC, R, L]
        Hant = Hsym[DMRS_SYMBOLS[0]]
    else:
        Hant = _channel(cfg, rng)                                        # [N_SC, R, L]
        Hsym = None
    W = beam_matrix(cfg)
    noise_var = float(10.0 ** (-cfg.snr_db / 10.0))

    # DMRS: QPSK on each layer's comb, zero elsewhere (or the 3GPP type-1 sequence of the slot).
    pb = rng.integers(0, 2, size=(L, 2, n_sc, 2))
    pil = qam_map(pb, 2)
    a = np.arange(n_sc)
    mask = (a[None, :] % comb) == ports[:, None]                          # [L, N_SC]
    pil = pil * mask[:, None, :]
    if cfg.dmrs == "type1":
        if L > 4:
            raise ValueError("type-1 DMRS carries at most 4 ports")
        pil = dmrs_type1(cfg.n_id, cfg.n_scid, slot_index % 20, ports, n_sc)
    pilots = pil.astype(np.complex64)

    bits = rng.integers(0, 2, size=(L, len(DATA_SYMBOLS), n_sc, q)).astype(np.uint8)
    x = qam_map(bits, q)                                                  # [L, 12, N_SC]

    # Transmitted grid t[l, s, a]; the pilots as the receiver knows them (complex64) are what is sent.
    t = np.zeros((L, N_SYM, n_sc), dtype=np.complex128)
    for j, s in enumerate(DMRS_SYMBOLS):
        t[:, s, :] = pilots[:, j, :].astype(np.complex128)
    for j, s in enumerate(DATA_SYMBOLS):
        t[:, s, :] = x[:, j, :]

    if Hsym is None:
        X = np.matmul(Hant, np.ascontiguousarray(t.transpose(2, 0, 1))).transpose(2, 1, 0)   # [S, R, N_SC]
    else:
        X = np.stack([np.einsum("arl,la->ra", Hsym[s], t[:, s, :]) for s in range(N_SYM)])
    noise = (rng.standard_normal(X.shape) + 1j * rng.standard_normal(X.shape)) * np.sqrt(noise_var / 2.0)
    X = X + noise

    spec = np.zeros((N_SYM, R, N), dtype=np.complex128)
    spec[:, :, active_bins(n_sc, N)] = X
    time = np.fft.ifft(spec, axis=-1)
    if cfg.cp or cfg.shift_7p5khz:
        time = _waveform(time, cfg.cp, cfg.shift_7p5khz)
    if cfg.in_fp16:
        time_in = np.stack([time.real, time.imag], axis=-1).astype(np.float16)
    else:
        time_in = time.astype(np.complex64)

    H_beam = np.matmul(W.astype(np.complex128).conj().T, Hant).transpose(0, 2, 1)   # [N_SC, L, B]
    return Slot(cfg=cfg, time_in=time_in, W=W, pilots=pilots, ports=ports, noise_var=noise_var,
                H_beam=H_beam, x=x, bits=pack_bits(bits))


def gold_bits(c_init: int, n: int) -> np.ndarray:
    """c(0..n) of the length-31 Gold sequence of TS 38.211 5.2.1 (the transmitter's copy of the definition)."""
    total = 1600 + n + 31
    x1 = [0] * total
    x2 = [0] * total
    x1[0] = 1
    for i in range(31):
        x2[i] = (c_init >> i) & 1
    for k in range(total - 31):
        x1[k + 31] = x1[k + 3] ^ x1[k]
        x2[k + 31] = x2[k + 3] ^ x2[k + 2] ^ x2[k + 1] ^ x2[k]
    return np.array([x1[k + 1600] ^ x2[k + 1600] for k in range(n)], dtype=np.uint8)


def dmrs_type1(n_id: int, n_scid: int, slot: int, ports, n_sc: int, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """Transmitted type-1 DMRS [L, 2, n_sc] (TS 38.211 6.4.1.1): port p on subcarriers k = 4n + 2k' + p // 2 with
    w_f(k') r(2n + k'), w_f = (1, -1) for odd p, r(m) = ((1 - 2c(2m)) + i (1 - 2c(2m + 1))) / sqrt 2 from
    c_init = (2^17 (14 slot + l + 1)(2 n_id + 1) + 2 n_id + n_scid) mod 2^31 of DMRS symbol l."""
    ports = list(ports)
    out = np.zeros((len(ports), 2, n_sc), dtype=np.complex128)
    for j, sym in enumerate(dmrs):
        c_init = ((1 << 17) * (14 * slot + sym + 1) * (2 * n_id + 1) + 2 * n_id + n_scid) % (1 << 31)
        c = gold_bits(c_init, n_sc + 2).astype(np.float64)
        for li, p in enumerate(ports):
            delta = p // 2
            k = np.arange(delta, n_sc, 2)
            m = (k - delta) // 2
            w = np.where((p % 2 == 1) & (m % 2 == 1), -1.0, 1.0)
            out[li, j, k] = w * ((1 - 2 * c[2 * m]) + 1j * (1 - 2 * c[2 * m + 1])) / np.sqrt(2)
    return out


def cp_lengths(n_fft: int) -> tuple[int, int]:
    """NR normal cyclic prefix at 30 kHz (TS 38.211 5.3.1): samples of symbol 0 and of the other symbols."""
    return 352 * n_fft // 4096, 288 * n_fft // 4096


def _waveform(time: np.ndarray, cp: bool, shift: bool) -> np.ndarray:
    """[S, R, N] periodic symbols -> the transmitted samples: with cp, [R, slot_len] streams where each symbol is
    preceded by its cyclic prefix; with shift, every sample multiplied by exp(2 pi i n' / (4 N)), n' counted from
    the start of its symbol's useful part (negative inside the prefix), as the 7.5 kHz shift of TS 38.211 5.4."""
    S, R, N = time.shape
    cp0, cp1 = cp_lengths(N) if cp else (0, 0)
    parts = []
    for s in range(S):
        c = cp0 if s == 0 else cp1
        n = np.arange(-c, N)
        x = time[s][:, n % N]
        if shift:
            x = x * np.exp(2j * np.pi * n / (4 * N))
        parts.append(x)
    return np.ascontiguousarray(np.concatenate(parts, axis=1) if cp else np.stack(parts))


def make_slots(cfg: CellConfig, n: int, first: int = 0, seed: int | None = None) -> list[Slot]:
    return [make_slot(cfg, first + i, seed) for i in range(n)]


# ------------------------------------------------------------------------------------------------------------
# Ragged multi-cell batches: several cells (antennas 32 or 64, FFT 2048 or 4096), each with users on seeded
# random contiguous PRB ranges, 1-4 layers, QPSK or 16-QAM and their own SNR. A cell's DMRS comb has N_B/2
# ports; overlapping users get disjoint contiguous port ranges (see _draw_users).

@dataclass
class RaggedCell:
    n_rx: int
    n_fft: int
    n_sc: int
    n_beams: int
    noise_var: float
    comb: int = 1                 # DMRS comb size = number of ports of the cell (N_B / 2)


@dataclass
class RaggedUser:
    cell: int
    sc_start: int
    sc_count: int
    n_layers: int
    port0: int
    qam_bits: int
    snr_db: float


@dataclass
class RaggedSlot:
    cells: list
    users: list
    time_in: list = field(repr=False)       # per cell [14, n_rx, n_fft, 2] float16
    W: list = field(repr=False)             # per cell [n_rx, n_beams] complex64
    pilots: list = field(repr=False)        # per user [n_layers, 2, sc_count] complex64 (zero off its comb)
    x: list = field(repr=False)             # per user [n_layers, 12, sc_count] complex128 (truth)
    bits: list = field(repr=False)          # per user [n_layers, 12, sc_count] uint8 packed (truth)

    def time_as_complex128(self, c: int) -> np.ndarray:
        t = self.time_in[c]
        return t[..., 0].astype(np.float64) + 1j * t[..., 1].astype(np.float64)


RAGGED_SEED = 3


def _draw_users(rng, cells, n_users, max_tries=10000):
    """Users are drawn one at a time. A cell's comb (port count) is N_B/2; a user takes the lowest contiguous
    ports that no user overlapping its range already uses. The user is redrawn while its range would make
    more than N_B/2 layers overlap, no such ports exist, or its range misses a pilot of one of its ports."""
    cell_of = [int(rng.integers(0, len(cells))) for _ in range(n_users)]
    for cell in cells:
        cell.comb = cell.n_beams // 2
    out = []
    placed = [[] for _ in cells]  # (a0, a1, p0, L)
    for c in cell_of:
        cell = cells[c]
        cap = cell.comb
        n_prb_max = cell.n_sc // 12
        for _ in range(max_tries):
            n_prb = int(rng.integers(1, n_prb_max + 1))
            a0 = 12 * int(rng.integers(0, n_prb_max - n_prb + 1))
            a1 = a0 + 12 * n_prb
            L = int(rng.integers(1, 5))
            used = np.zeros(cap, dtype=bool)
            load = np.zeros(a1 - a0, dtype=np.int64)
            for (b0, b1, q0, K) in placed[c]:
                lo, hi = max(a0, b0), min(a1, b1)
                if lo < hi:
                    used[q0:q0 + K] = True
                    load[lo - a0:hi - a0] += K
            if L > cap or load.max(initial=0) + L > cap:
                continue
            p0 = next((p for p in range(cap - L + 1) if not used[p:p + L].any()), None)
            if p0 is None:
                continue
            a = np.arange(a0, a1)
            if not all(np.any(a % cap == p) for p in range(p0, p0 + L)):
                continue
            placed[c].append((a0, a1, p0, L))
            out.append(RaggedUser(cell=c, sc_start=a0, sc_count=a1 - a0, n_layers=L, port0=p0,
                                  qam_bits=int(rng.choice([2, 4])), snr_db=float(rng.uniform(5.0, 25.0))))
            break
        else:
            raise RuntimeError("could not draw a valid user")
    return out


def make_ragged_slot(n_cells: int = 8, n_users: int = 64, slot_index: int = 0, seed: int = RAGGED_SEED,
                     cell_shapes=None, users=None) -> RaggedSlot:
    """One slot of a ragged multi-cell batch (the noise variance of every cell is 10^-2.5; a user's SNR sets
    its channel power). `users` (a list of RaggedUser) replaces the random user draw."""
    rng = np.random.default_rng([seed, slot_index])
    cells = []
    for c in range(n_cells):
        if cell_shapes is not None:
            n_rx, n_fft = cell_shapes[c % len(cell_shapes)]
        else:
            n_rx, n_fft = int(rng.choice([32, 64])), int(rng.choice([2048, 4096]))
        n_sc = 12 * int(np.floor(0.8 * n_fft / 12))
        cells.append(RaggedCell(n_rx=n_rx, n_fft=n_fft, n_sc=n_sc, n_beams=n_rx // 2, noise_var=10 ** -2.5))
    if users is None:
        users = _draw_users(rng, cells, n_users)
    else:
        for c in cells:
            c.comb = c.n_beams // 2

    time_in, Ws = [], []
    X = [np.zeros((N_SYM, c.n_rx, c.n_sc), dtype=np.complex128) for c in cells]
    pilots, xs, bitss = [], [], []
    for u in users:
        cell = cells[u.cell]
        ccfg = CellConfig("u", n_rx=cell.n_rx, n_fft=cell.n_fft, n_sc=cell.n_sc, n_beams=cell.n_beams,
                          n_layers=u.n_layers, qam_bits=u.qam_bits, snr_db=u.snr_db, channel="pdp", beam="dft",
                          in_fp16=True)
        Hant = _channel(ccfg, rng)[u.sc_start:u.sc_start + u.sc_count]            # [n, R, L]
        gain = np.sqrt(10.0 ** (u.snr_db / 10.0) * cell.noise_var)
        Hant = Hant * gain
        a = np.arange(u.sc_start, u.sc_start + u.sc_count)
        pb = rng.integers(0, 2, size=(u.n_layers, 2, u.sc_count, 2))
        pil = qam_map(pb, 2)
        ports = u.port0 + np.arange(u.n_layers)
        mask = (a[None, :] % cell.comb) == ports[:, None]
        pil = (pil * mask[:, None, :]).astype(np.complex64)
        bits = rng.integers(0, 2, size=(u.n_layers, len(DATA_SYMBOLS), u.sc_count, u.qam_bits)).astype(np.uint8)
        x = qam_map(bits, u.qam_bits)
        t = np.zeros((u.n_layers, N_SYM, u.sc_count), dtype=np.complex128)
        for j, s in enumerate(DMRS_SYMBOLS):
            t[:, s, :] = pil[:, j, :].astype(np.complex128)
        for j, s in enumerate(DATA_SYMBOLS):
            t[:, s, :] = x[:, j, :]
        X[u.cell][:, :, u.sc_start:u.sc_start + u.sc_count] += np.matmul(
            Hant, np.ascontiguousarray(t.transpose(2, 0, 1))).transpose(2, 1, 0)
        pilots.append(pil)
        xs.append(x)
        bitss.append(pack_bits(bits))
    for c, cell in enumerate(cells):
        Xc = X[c] + (rng.standard_normal(X[c].shape) + 1j * rng.standard_normal(X[c].shape)) * np.sqrt(
            cell.noise_var / 2.0)
        spec = np.zeros((N_SYM, cell.n_rx, cell.n_fft), dtype=np.complex128)
        spec[:, :, active_bins(cell.n_sc, cell.n_fft)] = Xc
        tm = np.fft.ifft(spec, axis=-1)
        time_in.append(np.stack([tm.real, tm.imag], axis=-1).astype(np.float16))
        r = np.arange(cell.n_rx)[:, None]
        b = np.arange(cell.n_beams)[None, :]
        Ws.append((np.exp(-2j * np.pi * r * b / cell.n_rx) / np.sqrt(cell.n_rx)).astype(np.complex64))
    return RaggedSlot(cells=cells, users=users, time_in=time_in, W=Ws, pilots=pilots, x=xs, bits=bitss)
