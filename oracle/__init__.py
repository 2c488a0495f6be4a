"""FP64 CPU oracle of the PUSCH receive hot path (arXiv 2210.09196) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
package. The product path (``paper_2210_09196_gb300``) never imports it and shares no code with it.

This module is argument marshalling around ``pusch_oracle.c`` (plain C, double precision), which carries the
definitions and their citations. Arrays are numpy complex128 in the layouts documented in the C file.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "pusch_oracle.c"
_BUILD = _HERE / "_build"
_LIB_PATH = _BUILD / "liboracle.so"
_lib = None

DMRS_SYMBOLS = (2, 11)


def build(force: bool = False) -> Path:
    """Compile the oracle with gcc (portable C99, no architecture flags)."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB_PATH.exists() or _LIB_PATH.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _BUILD / f"liboracle.{os.getpid()}.so"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", str(_SRC), "-o", str(tmp), "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB_PATH))
        P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
        sig = {
            "orc_dft": (None, [P, I, P]),
            "orc_fft": (I, [P, I, P]),
            "orc_ofdm_demod": (I, [P, I, I, I, I, P, I, P]),
            "orc_cp_len": (I, [I, I]),
            "orc_gold": (I, [ctypes.c_uint32, I, P]),
            "orc_dmrs_cinit": (ctypes.c_uint32, [I, I, I, I]),
            "orc_dmrs_type1_pilots": (I, [I, I, I, P, I, P, I, P]),
            "orc_chest_ls_type1": (I, [P, I, I, I, P, I, P, P, P]),
            "orc_chest_ls_type1_sym": (I, [P, I, I, I, P, I, P, P, I, P]),
            "orc_noise_est_type1": (D, [P, I, I, I, P, I, P, P]),
            "orc_slot_len": (ctypes.c_longlong, [I, I]),
            "orc_ofdm_demod_cp": (I, [P, I, I, I, I, I, P]),
            "orc_beamform": (None, [P, P, I, I, I, I, P]),
            "orc_chest_ls": (I, [P, I, I, I, P, I, P, P, I, P, P, P]),
            "orc_gram": (None, [P, I, I, D, P]),
            "orc_cholesky": (I, [P, I, P]),
            "orc_chol_solve": (None, [P, I, P, P]),
            "orc_mmse": (I, [P, P, I, I, I, P, I, D, D, P, I, P]),
            "orc_mmse_active": (I, [P, P, P, I, I, I, P, I, D, D, P]),
            "orc_demap": (None, [P, LL, I, I, P]),
            "orc_cnn_param_count": (I, []),
            "orc_round_bf16": (D, [D]),
            "orc_cnn_forward": (None, [P, P, I, I, I, P, P]),
            "orc_cnn_loss_grad": (D, [P, P, P, I, I, I, P]),
            "orc_op_counts": (None, [I, I, I, I, I, I, P]),
            "orc_slot": (I, [P, I, I, I, I, P, I, P, I, P, P, I, I, D, D, P, P]),
            "orc_noise_est": (D, [P, I, I, I, P, I, P, P, I]),
            "orc_chest_ls_sym": (I, [P, I, I, I, P, I, P, P, I, I, P]),
            "orc_mmse_tv": (I, [P, P, P, I, I, I, P, P, I, D, D, I, P]),
            "orc_e4m3_round": (D, [D]),
            "orc_e4m3_round_array": (None, [P, LL, P]),
            "orc_e4m3_block_exp": (I, [D]),
            "orc_e4m3_quant_rows": (None, [P, LL, I, P, P]),
            "orc_beamform_fp8": (None, [P, P, P, I, I, I, I, P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _c128(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def dft(x) -> np.ndarray:
    x = _c128(x)
    X = np.empty_like(x)
    lib().orc_dft(_p(x), x.size, _p(X))
    return X


def fft(x) -> np.ndarray:
    x = _c128(x)
    X = np.empty_like(x)
    if lib().orc_fft(_p(x), x.size, _p(X)) != 0:
        raise ValueError("orc_fft needs a power-of-two length")
    return X


def gold(c_init: int, n: int) -> np.ndarray:
    """c(0..n) of the TS 38.211 5.2.1 sequence for c_init, as uint8 bits."""
    c = np.zeros(n, dtype=np.uint8)
    if lib().orc_gold(int(c_init), n, _p(c)) != 0:
        raise ValueError("orc_gold failed")
    return c


def dmrs_cinit(n_id: int, n_scid: int, slot: int, sym: int) -> int:
    return int(lib().orc_dmrs_cinit(n_id, n_scid, slot, sym))


def dmrs_type1_pilots(n_id: int, n_scid: int, slot: int, ports, n_sc: int, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """[L, 2, n_sc] type-1 DMRS values of the layers' ports (0..3) on the two DMRS symbols."""
    ports = _i32(ports)
    out = np.zeros((ports.size, 2, n_sc), dtype=np.complex128)
    if lib().orc_dmrs_type1_pilots(n_id, n_scid, slot, _p(_i32(dmrs)), ports.size, _p(ports), n_sc, _p(out)) != 0:
        raise ValueError("orc_dmrs_type1_pilots failed")
    return out


def chest_ls_type1(beam, pilots, ports, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """beam [S, N_SC, B], pilots [L, 2, N_SC] (type 1) -> H [N_SC, L, B]."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    L = pilots.shape[0]
    H = np.zeros((n_sc, L, B), dtype=np.complex128)
    rc = lib().orc_chest_ls_type1(_p(beam), S, n_sc, B, _p(_i32(dmrs)), L, _p(_i32(ports)), _p(pilots), _p(H))
    if rc != 0:
        raise ValueError(f"orc_chest_ls_type1 failed ({rc})")
    return H


def chest_ls_type1_sym(beam, pilots, ports, j: int, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """The type-1 estimate of DMRS symbol j alone: [N_SC, L, B]."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    L = pilots.shape[0]
    H = np.zeros((n_sc, L, B), dtype=np.complex128)
    rc = lib().orc_chest_ls_type1_sym(_p(beam), S, n_sc, B, _p(_i32(dmrs)), L, _p(_i32(ports)), _p(pilots), int(j),
                                      _p(H))
    if rc != 0:
        raise ValueError(f"orc_chest_ls_type1_sym failed ({rc})")
    return H


def noise_est_type1(beam, pilots, ports, dmrs=DMRS_SYMBOLS) -> float:
    """sigma^2 from the type-1 DMRS residuals (degrees-of-freedom normalised)."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    return float(lib().orc_noise_est_type1(_p(beam), S, n_sc, B, _p(_i32(dmrs)), pilots.shape[0], _p(_i32(ports)),
                                           _p(pilots)))


def cp_len(n_fft: int, sym: int) -> int:
    """Normal cyclic-prefix length (samples) of symbol sym of a 30 kHz slot."""
    return int(lib().orc_cp_len(n_fft, sym))


def slot_len(n_sym: int, n_fft: int) -> int:
    return int(lib().orc_slot_len(n_sym, n_fft))


def ofdm_demod_cp(stream, n_sym: int, n_fft: int, n_sc: int, shift: bool = False) -> np.ndarray:
    """stream [R, slot_len] (cyclic prefixes included) -> freq [S, R, N_SC]."""
    stream = _c128(stream)
    R = stream.shape[0]
    if stream.shape[1] != slot_len(n_sym, n_fft):
        raise ValueError("stream length is not the slot length")
    freq = np.zeros((n_sym, R, n_sc), dtype=np.complex128)
    rc = lib().orc_ofdm_demod_cp(_p(stream), n_sym, R, n_fft, n_sc, int(bool(shift)), _p(freq))
    if rc != 0:
        raise ValueError(f"orc_ofdm_demod_cp failed ({rc})")
    return freq


def ofdm_demod(time, n_sc: int, pairs=None) -> np.ndarray:
    """time [S, R, N_F] -> freq [S, R, N_SC] (only the listed (symbol, antenna) rows when pairs is given)."""
    time = _c128(time)
    S, R, N = time.shape
    freq = np.zeros((S, R, n_sc), dtype=np.complex128)
    if pairs is None:
        rc = lib().orc_ofdm_demod(_p(time), S, R, N, n_sc, None, 0, _p(freq))
    else:
        pr = _i32(pairs).reshape(-1, 2)
        rc = lib().orc_ofdm_demod(_p(time), S, R, N, n_sc, _p(pr), pr.shape[0], _p(freq))
    if rc != 0:
        raise ValueError(f"orc_ofdm_demod failed ({rc})")
    return freq


def beamform(freq, W) -> np.ndarray:
    """freq [S, R, N_SC], W [R, B] -> beam [S, N_SC, B] = W^H x."""
    freq, W = _c128(freq), _c128(W)
    S, R, n_sc = freq.shape
    B = W.shape[1]
    beam = np.empty((S, n_sc, B), dtype=np.complex128)
    lib().orc_beamform(_p(freq), _p(W), S, R, n_sc, B, _p(beam))
    return beam


def chest_ls(beam, pilots, ports, comb: int, sc_start=None, sc_count=None, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """beam [S, N_SC, B], pilots [L, 2, N_SC] -> H [N_SC, L, B] (zeros outside each layer's range)."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    L = pilots.shape[0]
    st = _i32(np.zeros(L) if sc_start is None else sc_start)
    ct = _i32(np.full(L, n_sc) if sc_count is None else sc_count)
    H = np.zeros((n_sc, L, B), dtype=np.complex128)
    rc = lib().orc_chest_ls(_p(beam), S, n_sc, B, _p(_i32(dmrs)), L, _p(pilots), _p(_i32(ports)), comb,
                            _p(st), _p(ct), _p(H))
    if rc != 0:
        raise ValueError(f"orc_chest_ls: layer {-rc - 1} has no pilot in its range")
    return H


def noise_est(beam, pilots, ports, comb: int, dmrs=DMRS_SYMBOLS) -> float:
    """beam [S, N_SC, B], pilots [L, 2, N_SC] -> sigma2_hat (Section II NE; see orc_noise_est)."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    L = pilots.shape[0]
    v = lib().orc_noise_est(_p(beam), S, n_sc, B, _p(_i32(dmrs)), L, _p(pilots), _p(_i32(ports)), comb)
    if v < 0:
        raise ValueError("orc_noise_est: no pilot subcarrier")
    return float(v)


def gram(Hs, load: float) -> np.ndarray:
    """Hs [L, B] (row l = column l of H) -> G = H^H H + load I."""
    Hs = _c128(Hs)
    L, B = Hs.shape
    G = np.empty((L, L), dtype=np.complex128)
    lib().orc_gram(_p(Hs), L, B, load, _p(G))
    return G


def cholesky(G):
    """Returns (L, status); status = 0 or the 1-based index of the first non-positive pivot."""
    G = _c128(G)
    n = G.shape[0]
    L = np.empty_like(G)
    st = lib().orc_cholesky(_p(G), n, _p(L))
    return L, int(st)


def chol_solve(L, r) -> np.ndarray:
    L, r = _c128(L), _c128(r)
    x = np.empty_like(r)
    lib().orc_chol_solve(_p(L), L.shape[0], _p(r), _p(x))
    return x


def data_symbols(n_sym: int = 14, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    return np.array([s for s in range(n_sym) if s not in dmrs], dtype=np.int32)


def mmse(H, beam, noise_var: float, loading: float = 0.0, sc_list=None, data_sym=None):
    """H [N_SC, L, B], beam [S, N_SC, B] -> (xhat [L, n_data, N_SC], n_failed)."""
    H, beam = _c128(H), _c128(beam)
    n_sc, L, B = H.shape
    S = beam.shape[0]
    ds = data_symbols(S) if data_sym is None else _i32(data_sym)
    xhat = np.zeros((L, ds.size, n_sc), dtype=np.complex128)
    if sc_list is None:
        fails = lib().orc_mmse(_p(H), _p(beam), n_sc, B, L, _p(ds), ds.size, noise_var, loading, None, 0, _p(xhat))
    else:
        sl = _i32(sc_list)
        fails = lib().orc_mmse(_p(H), _p(beam), n_sc, B, L, _p(ds), ds.size, noise_var, loading, _p(sl), sl.size,
                               _p(xhat))
    return xhat, int(fails)


def chest_ls_sym(beam, pilots, ports, comb: int, j: int, dmrs=DMRS_SYMBOLS) -> np.ndarray:
    """The estimate of DMRS symbol j alone: beam [S, N_SC, B], pilots [L, 2, N_SC] -> H [N_SC, L, B]."""
    beam, pilots = _c128(beam), _c128(pilots)
    S, n_sc, B = beam.shape
    L = pilots.shape[0]
    H = np.zeros((n_sc, L, B), dtype=np.complex128)
    rc = lib().orc_chest_ls_sym(_p(beam), S, n_sc, B, _p(_i32(dmrs)), L, _p(pilots), _p(_i32(ports)), comb, int(j),
                                _p(H))
    if rc != 0:
        raise ValueError(f"orc_chest_ls_sym: layer {-rc - 1} has no pilot")
    return H


def mmse_tv(H0, H1, beam, noise_var: float, K: int, loading: float = 0.0, dmrs=DMRS_SYMBOLS, data_sym=None):
    """Eq. 2 with the estimate interpolated in time between the DMRS symbols and factorised every K data
    symbols -> (xhat [L, n_data, N_SC], n_failed)."""
    H0, H1, beam = _c128(H0), _c128(H1), _c128(beam)
    n_sc, L, B = H0.shape
    ds = data_symbols(beam.shape[0], dmrs) if data_sym is None else _i32(data_sym)
    xhat = np.zeros((L, ds.size, n_sc), dtype=np.complex128)
    fails = lib().orc_mmse_tv(_p(H0), _p(H1), _p(beam), n_sc, B, L, _p(_i32(dmrs)), _p(ds), ds.size, noise_var,
                              loading, int(K), _p(xhat))
    return xhat, int(fails)


def mmse_active(H, beam, active, noise_var: float, loading: float = 0.0, data_sym=None):
    """H [N_SC, L, B], beam [S, N_SC, B], active [N_SC, L] (bool) -> (xhat [L, n_data, N_SC], n_failed);
    entries of layers inactive at a subcarrier are zero."""
    H, beam = _c128(H), _c128(beam)
    act = np.ascontiguousarray(active, dtype=np.uint8)
    n_sc, L, B = H.shape
    ds = data_symbols(beam.shape[0]) if data_sym is None else _i32(data_sym)
    xhat = np.zeros((L, ds.size, n_sc), dtype=np.complex128)
    fails = lib().orc_mmse_active(_p(H), _p(beam), _p(act), n_sc, B, L, _p(ds), ds.size, noise_var, loading, _p(xhat))
    return xhat, int(fails)


def demap(x, qam_bits: int, f32: bool = False) -> np.ndarray:
    x = _c128(x)
    bits = np.empty(x.shape, dtype=np.uint8)
    lib().orc_demap(_p(x), x.size, qam_bits, 1 if f32 else 0, _p(bits))
    return bits


def op_counts(n_symb: int, n_pilot: int, n_r: int, n_sc: int, n_b: int, n_l: int) -> dict:
    out = np.zeros(5, dtype=np.float64)
    lib().orc_op_counts(n_symb, n_pilot, n_r, n_sc, n_b, n_l, _p(out))
    return dict(zip(("ofdm", "bf", "mimo", "che", "ne"), out.tolist()))


def slot(time, W, pilots, ports, comb: int, n_sc: int, qam_bits: int, noise_var: float, loading: float = 0.0,
         dmrs=DMRS_SYMBOLS):
    """The whole chain for one slot -> (xhat [L, 12, N_SC], bits [L, 12, N_SC], n_failed)."""
    time, W, pilots = _c128(time), _c128(W), _c128(pilots)
    S, R, N = time.shape
    B = W.shape[1]
    L = pilots.shape[0]
    n_data = S - 2
    xhat = np.zeros((L, n_data, n_sc), dtype=np.complex128)
    bits = np.zeros((L, n_data, n_sc), dtype=np.uint8)
    rc = lib().orc_slot(_p(time), S, R, N, n_sc, _p(W), B, _p(_i32(dmrs)), L, _p(pilots), _p(_i32(ports)), comb,
                        qam_bits, noise_var, loading, _p(xhat), _p(bits))
    if rc < 0:
        raise ValueError(f"orc_slot failed ({rc})")
    return xhat, bits, rc


def run_slot(s, loading: float = 0.0):
    """Convenience: run the chain on a generated slot object (paper_2210_09196_gb300.synth.Slot)."""
    return slot(s.time_as_complex128(), s.W, s.pilots, s.ports, s.cfg.comb, s.cfg.n_sc, s.cfg.qam_bits,
                s.noise_var, loading)


# ---------------------------------------------------------------------------------------- denoiser CNN

def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def cnn_param_count() -> int:
    return int(lib().orc_cnn_param_count())


def round_bf16(v) -> np.ndarray:
    f = np.vectorize(lambda t: lib().orc_round_bf16(float(t)))
    return f(np.asarray(v, dtype=np.float64))


def cnn_forward(params, x, bf16: bool = False):
    """params (packed), x [n, 2, 2, w] -> (y [n, 2, 2, w], activations [3, n, 32, 2, w])."""
    params, x = _f64(params), _f64(x)
    n, _, _, w = x.shape
    y = np.empty_like(x)
    acts = np.empty((3, n, 32, 2, w))
    lib().orc_cnn_forward(_p(params), _p(x), n, w, 1 if bf16 else 0, _p(y), _p(acts))
    return y, acts


def cnn_loss_grad(params, x, target, bf16: bool = False):
    """(mean squared error, d loss / d params)."""
    params, x, target = _f64(params), _f64(x), _f64(target)
    n, _, _, w = x.shape
    g = np.empty_like(params)
    loss = lib().orc_cnn_loss_grad(_p(params), _p(x), _p(target), n, w, 1 if bf16 else 0, _p(g))
    return float(loss), g


# ------------------------------------------------------------------------------------ FP8 E4M3 form

def e4m3_round(v) -> np.ndarray:
    """Nearest E4M3 value (ties to even, saturating at +-448) of every element."""
    x = _f64(v)
    y = np.empty_like(x)
    lib().orc_e4m3_round_array(_p(x), x.size, _p(y))
    return y


def e4m3_block_exp(amax: float) -> int:
    return int(lib().orc_e4m3_block_exp(float(amax)))


def e4m3_quant_rows(x):
    """x complex [..., n] -> (codes complex [..., n] (E4M3 values, scale not applied), exps int [..., n_blk])."""
    x = _c128(x)
    n = x.shape[-1]
    rows = x.size // n if n else 0
    codes = np.empty_like(x)
    exps = np.empty(x.shape[:-1] + ((n + 127) // 128,), dtype=np.int32)
    lib().orc_e4m3_quant_rows(_p(x), rows, n, _p(codes), _p(exps))
    return codes, exps


def beamform_fp8(codes, exps, W) -> np.ndarray:
    """codes [n_sym, n_rx, n_sc] (E4M3 values), exps [n_sym, n_rx, ceil(n_sc/128)], W [n_rx, n_beams]
    -> beam [n_sym, n_sc, n_beams] of the FP8 form's block-scaled product."""
    codes, exps, W = _c128(codes), _i32(exps), _c128(W)
    n_sym, n_rx, n_sc = codes.shape
    n_beams = W.shape[1]
    assert exps.shape == (n_sym, n_rx, (n_sc + 127) // 128) and W.shape[0] == n_rx
    beam = np.empty((n_sym, n_sc, n_beams), dtype=np.complex128)
    lib().orc_beamform_fp8(_p(codes), _p(exps), _p(W), n_sym, n_rx, n_sc, n_beams, _p(beam))
    return beam
