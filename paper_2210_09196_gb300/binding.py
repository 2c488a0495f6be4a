"""Thin ctypes binding of libpusch (include/pusch.h): argument marshalling only.

Every computation runs in the CUDA kernels of libpusch.so. There is no CPU or PyTorch fallback: if the
library is missing or cannot be loaded, every entry point raises.

Functions keep the C names. Buffers may be passed as torch tensors (their ``data_ptr()`` is used; device
tensors for device pointers, CPU tensors for the host buffers of ``pusch_slot_host``) or as raw integer
addresses. ``stream`` may be a ``torch.cuda.Stream``, an integer cudaStream_t or None (the current torch
stream).
"""
from __future__ import annotations

import ctypes
from pathlib import Path

_PKG = Path(__file__).resolve().parent
LIB_PATH = _PKG / "_build" / "libpusch.so"

PUSCH_OK = 0
PUSCH_ERR_ARG = -1
PUSCH_ERR_CUDA = -2
PUSCH_ERR_NUMERIC = -3
PUSCH_ERR_TIMEOUT = -4
PUSCH_ERR_UNSUPPORTED = -5

PUSCH_FORM_FP32 = 0
PUSCH_FORM_MIXED = 1
PUSCH_FORM_FP8 = 2

PUSCH_NOISE_ESTIMATE = -1.0

PUSCH_STATUS_PIVOT = 0x1
PUSCH_STATUS_NONFINITE = 0x2
PUSCH_STATUS_TIMEOUT = 0x4

# every symbol include/pusch.h declares
EXPORTS = (
    "pusch_create", "pusch_destroy", "pusch_workspace_size", "pusch_sc_pitch", "pusch_freq_bytes", "pusch_ofdm_fft",
    "pusch_beamform",
    "pusch_chest_ls", "pusch_noise_estimate", "pusch_mmse_detect", "pusch_slot", "pusch_slot_host",
    "pusch_set_pipeline", "pusch_dmrs_type1_pilots", "pusch_last_error", "pusch_version",
    "pusch_slot_noalloc", "pusch_profile_start", "pusch_profile_read",
    "pusch_batch_create", "pusch_batch_destroy", "pusch_batch_sizes", "pusch_batch_run", "pusch_batch_autotune",
    "pusch_batch_tuning",
    "pusch_cnn_param_count", "pusch_cnn_forward", "pusch_cnn_backward", "pusch_cnn_adam", "pusch_ls_grid",
    "pusch_chest_cnn", "pusch_status_check", "pusch_selftest_wait", "pusch_autotune",
)


class PuschError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed with status {code}: {msg}")
        self.code = code


class pusch_cell_cfg(ctypes.Structure):
    _fields_ = [
        ("n_rx", ctypes.c_int), ("n_fft", ctypes.c_int), ("n_sc", ctypes.c_int), ("n_beams", ctypes.c_int),
        ("n_layers", ctypes.c_int), ("comb", ctypes.c_int), ("port", ctypes.c_int * 32),
        ("qam_bits", ctypes.c_int), ("in_fp16", ctypes.c_int), ("form", ctypes.c_int), ("n_sym", ctypes.c_int),
        ("dmrs_sym", ctypes.c_int * 2), ("noise_var", ctypes.c_float), ("loading", ctypes.c_float),
        ("chol_every", ctypes.c_int),
        ("cp", ctypes.c_int),
        ("shift_7p5khz", ctypes.c_int),
        ("dmrs_type", ctypes.c_int),
    ]


class pusch_user_desc(ctypes.Structure):
    _fields_ = [("cell", ctypes.c_int), ("sc_start", ctypes.c_int), ("sc_count", ctypes.c_int),
                ("n_layers", ctypes.c_int), ("port0", ctypes.c_int), ("qam_bits", ctypes.c_int)]


def make_cfg(*, n_rx, n_fft, n_sc, n_beams, n_layers, comb=None, ports=None, qam_bits=2, in_fp16=False,
             form=PUSCH_FORM_FP32, noise_var=0.0, loading=0.0, n_sym=14, dmrs_sym=(2, 11),
             chol_every=0, cp=False, shift_7p5khz=False, dmrs_type=0) -> pusch_cell_cfg:
    c = pusch_cell_cfg()
    c.n_rx, c.n_fft, c.n_sc, c.n_beams, c.n_layers = n_rx, n_fft, n_sc, n_beams, n_layers
    c.comb = n_layers if comb is None else comb
    ports = list(range(n_layers)) if ports is None else list(ports)
    for i, p in enumerate(ports[:32]):
        c.port[i] = int(p)
    c.qam_bits, c.in_fp16, c.form, c.n_sym = qam_bits, int(bool(in_fp16)), int(form), n_sym
    c.dmrs_sym[0], c.dmrs_sym[1] = dmrs_sym
    c.noise_var, c.loading = float(noise_var), float(loading)
    c.chol_every = int(chol_every)
    c.cp, c.shift_7p5khz = int(bool(cp)), int(bool(shift_7p5khz))
    c.dmrs_type = int(dmrs_type)
    return c


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"libpusch.so is not built ({LIB_PATH}); run __graft_entry__.build() first")
        L = ctypes.CDLL(str(LIB_PATH))
        P, I = ctypes.c_void_p, ctypes.c_int
        sig = {
            "pusch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(pusch_cell_cfg), I]),
            "pusch_destroy": (I, [P]),
            "pusch_workspace_size": (I, [ctypes.POINTER(pusch_cell_cfg), I, ctypes.POINTER(ctypes.c_size_t)]),
            "pusch_sc_pitch": (I, [ctypes.POINTER(pusch_cell_cfg)]),
            "pusch_freq_bytes": (ctypes.c_size_t, [ctypes.POINTER(pusch_cell_cfg), I]),
            "pusch_ofdm_fft": (I, [P, I, P, P, P]),
            "pusch_beamform": (I, [P, I, P, P, P, P]),
            "pusch_chest_ls": (I, [P, I, P, P, P, P]),
            "pusch_noise_estimate": (I, [P, I, P, P, P, P]),
            "pusch_mmse_detect": (I, [P, I, P, P, P, P, P, P]),
            "pusch_slot": (I, [P, I, P, P, P, P, P, P, P]),
            "pusch_slot_host": (I, [P, I, P, P, P, P, P, P, P]),
            "pusch_slot_noalloc": (I, [ctypes.POINTER(pusch_cell_cfg), I, P, P, P, P, P, P, P]),
            "pusch_profile_start": (I, [P, I]),
            "pusch_set_pipeline": (I, [P, I]),
            "pusch_dmrs_type1_pilots": (I, [P, I, P, I, I, P, P]),
            "pusch_profile_read": (I, [P, ctypes.POINTER(ctypes.c_float), I, ctypes.POINTER(I)]),
            "pusch_batch_create": (I, [ctypes.POINTER(P), ctypes.POINTER(pusch_cell_cfg), I,
                                       ctypes.POINTER(pusch_user_desc), I]),
            "pusch_batch_destroy": (I, [P]),
            "pusch_batch_sizes": (I, [P, ctypes.POINTER(ctypes.c_size_t)]),
            "pusch_batch_run": (I, [P, P, P, P, P, P, P, P]),
            "pusch_batch_autotune": (I, [P, P, P, P, P, P, P, ctypes.c_char_p, P, ctypes.POINTER(I)]),
            "pusch_batch_tuning": (I, [P, ctypes.POINTER(I), I]),
            "pusch_cnn_param_count": (I, []),
            "pusch_cnn_forward": (I, [I, I, P, P, P, P, P]),
            "pusch_cnn_backward": (I, [I, I, P, P, P, P, P, P, P, P, P, P]),
            "pusch_cnn_adam": (I, [I, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, P, P, P, P, P,
                                   P]),
            "pusch_ls_grid": (I, [P, I, P, P, P, P, P]),
            "pusch_chest_cnn": (I, [P, I, P, P, P, ctypes.c_float, P, P, P, P]),
            "pusch_status_check": (I, [P, P, P]),
            "pusch_autotune": (I, [P, ctypes.c_char_p, P, ctypes.POINTER(I)]),
            "pusch_selftest_wait": (I, [P, ctypes.c_uint, P]),
            "pusch_last_error": (ctypes.c_char_p, []),
            "pusch_version": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Address of a buffer: None, a raw address (int), or a tensor, which must be contiguous (the C ABI takes
    dense row-major buffers)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "is_contiguous") and not x.is_contiguous():
        raise ValueError("buffers passed to libpusch must be contiguous tensors")
    return x.data_ptr()


def _stream(s):
    if s is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(s, int):
        return s
    return s.cuda_stream


def _check(code: int, where: str):
    if code != PUSCH_OK:
        raise PuschError(code, where, lib().pusch_last_error().decode())


def pusch_version() -> str:
    return lib().pusch_version().decode()


def pusch_last_error() -> str:
    return lib().pusch_last_error().decode()


def pusch_sc_pitch(cfg: pusch_cell_cfg) -> int:
    return lib().pusch_sc_pitch(ctypes.byref(cfg))


def pusch_freq_bytes(cfg: pusch_cell_cfg, n_slots: int) -> int:
    return int(lib().pusch_freq_bytes(ctypes.byref(cfg), int(n_slots)))


def pusch_workspace_size(cfg: pusch_cell_cfg, max_slots: int) -> int:
    out = ctypes.c_size_t()
    _check(lib().pusch_workspace_size(ctypes.byref(cfg), max_slots, ctypes.byref(out)), "pusch_workspace_size")
    return out.value


def pusch_create(cfg: pusch_cell_cfg, max_slots: int) -> int:
    h = ctypes.c_void_p()
    _check(lib().pusch_create(ctypes.byref(h), ctypes.byref(cfg), max_slots), "pusch_create")
    return h.value


def pusch_destroy(h) -> None:
    _check(lib().pusch_destroy(h), "pusch_destroy")


def pusch_ofdm_fft(h, n_slots, time_in, freq_out, stream=None) -> None:
    _check(lib().pusch_ofdm_fft(h, n_slots, _ptr(time_in), _ptr(freq_out), _stream(stream)), "pusch_ofdm_fft")


def pusch_beamform(h, n_slots, freq_in, W, beam_out, stream=None) -> None:
    _check(lib().pusch_beamform(h, n_slots, _ptr(freq_in), _ptr(W), _ptr(beam_out), _stream(stream)),
           "pusch_beamform")


def pusch_chest_ls(h, n_slots, beam, pilots, H_hat, stream=None) -> None:
    _check(lib().pusch_chest_ls(h, n_slots, _ptr(beam), _ptr(pilots), _ptr(H_hat), _stream(stream)),
           "pusch_chest_ls")


def pusch_noise_estimate(h, n_slots, beam, pilots, sigma2=None, stream=None) -> None:
    _check(lib().pusch_noise_estimate(h, n_slots, _ptr(beam), _ptr(pilots), _ptr(sigma2), _stream(stream)),
           "pusch_noise_estimate")


def pusch_mmse_detect(h, n_slots, H_hat, beam, x_hat, bits, status=None, stream=None) -> None:
    _check(lib().pusch_mmse_detect(h, n_slots, _ptr(H_hat), _ptr(beam), _ptr(x_hat), _ptr(bits), _ptr(status),
                                   _stream(stream)), "pusch_mmse_detect")


def pusch_slot(h, n_slots, time_in, W, pilots, x_hat, bits, status=None, stream=None) -> None:
    _check(lib().pusch_slot(h, n_slots, _ptr(time_in), _ptr(W), _ptr(pilots), _ptr(x_hat), _ptr(bits), _ptr(status),
                            _stream(stream)), "pusch_slot")


def pusch_slot_host(h, n_slots, time_in_host, W, pilots_host, x_hat_host, bits_host, status_host=None,
                    stream=None) -> None:
    _check(lib().pusch_slot_host(h, n_slots, _ptr(time_in_host), _ptr(W), _ptr(pilots_host), _ptr(x_hat_host),
                                 _ptr(bits_host), _ptr(status_host), _stream(stream)), "pusch_slot_host")


def pusch_slot_noalloc(cfg: pusch_cell_cfg, n_slots, time_in, W, pilots, x_hat, bits, status=None,
                       stream=None) -> None:
    """pusch_slot without a handle and without device allocation (static library buffer)."""
    _check(lib().pusch_slot_noalloc(ctypes.byref(cfg), n_slots, _ptr(time_in), _ptr(W), _ptr(pilots), _ptr(x_hat),
                                    _ptr(bits), _ptr(status), _stream(stream)), "pusch_slot_noalloc")


def pusch_status_check(h, status=None, stream=None) -> None:
    """Waits for the stream and raises PuschError (code PUSCH_ERR_TIMEOUT or PUSCH_ERR_NUMERIC) if the status
    words or the handle's kernel error word report a failure."""
    _check(lib().pusch_status_check(h, _ptr(status), _stream(stream)), "pusch_status_check")


def pusch_autotune(h, cache_path=None, stream=None) -> int:
    """Tunes the handle's launch shapes (or reads them from cache_path); returns the number of keys timed."""
    n = ctypes.c_int(0)
    path = None if cache_path is None else str(cache_path).encode()
    _check(lib().pusch_autotune(h, path, _stream(stream), ctypes.byref(n)), "pusch_autotune")
    return n.value


def pusch_selftest_wait(h, limit_us: int, stream=None) -> None:
    _check(lib().pusch_selftest_wait(h, int(limit_us), _stream(stream)), "pusch_selftest_wait")


SLOT_STAGES = ("fft", "beamform", "ls", "detect")


def pusch_dmrs_type1_pilots(cfg, n_slots, slot_numbers, n_id, n_scid, pilots, stream=None) -> None:
    sl = (ctypes.c_int * max(1, n_slots))(*[int(v) for v in slot_numbers])
    _check(lib().pusch_dmrs_type1_pilots(ctypes.byref(cfg), n_slots, sl, n_id, n_scid, _ptr(pilots), _stream(stream)),
           "pusch_dmrs_type1_pilots")


def pusch_set_pipeline(h, n_chunks: int) -> None:
    _check(lib().pusch_set_pipeline(h, n_chunks), "pusch_set_pipeline")


def pusch_profile_start(h, max_calls: int) -> None:
    _check(lib().pusch_profile_start(h, max_calls), "pusch_profile_start")


def pusch_profile_read(h) -> tuple[dict, int]:
    """(summed milliseconds per pusch_slot stage, number of timed calls)."""
    ms = (ctypes.c_float * len(SLOT_STAGES))()
    n = ctypes.c_int()
    _check(lib().pusch_profile_read(h, ms, len(SLOT_STAGES), ctypes.byref(n)), "pusch_profile_read")
    return dict(zip(SLOT_STAGES, list(ms))), n.value


def pusch_batch_create(cells, users) -> int:
    """cells: sequence of pusch_cell_cfg; users: sequence of pusch_user_desc."""
    ca = (pusch_cell_cfg * len(cells))(*cells)
    ua = (pusch_user_desc * len(users))(*users)
    b = ctypes.c_void_p()
    _check(lib().pusch_batch_create(ctypes.byref(b), ca, len(cells), ua, len(users)), "pusch_batch_create")
    return b.value


def pusch_batch_destroy(b) -> None:
    _check(lib().pusch_batch_destroy(b), "pusch_batch_destroy")


def pusch_batch_sizes(b) -> list:
    out = (ctypes.c_size_t * 5)()
    _check(lib().pusch_batch_sizes(b, out), "pusch_batch_sizes")
    return list(out)


def pusch_batch_run(b, time_in, W, pilots, x_hat, bits, status=None, stream=None) -> None:
    _check(lib().pusch_batch_run(b, _ptr(time_in), _ptr(W), _ptr(pilots), _ptr(x_hat), _ptr(bits), _ptr(status),
                                 _stream(stream)), "pusch_batch_run")


def pusch_batch_autotune(b, time_in, W, pilots, x_hat, bits, status=None, cache_path=None, stream=None) -> int:
    """Returns the number of keys that were timed (0 when every choice came from the cache)."""
    n = ctypes.c_int(0)
    path = None if cache_path is None else str(cache_path).encode()
    _check(lib().pusch_batch_autotune(b, _ptr(time_in), _ptr(W), _ptr(pilots), _ptr(x_hat), _ptr(bits), _ptr(status),
                                      path, _stream(stream), ctypes.byref(n)), "pusch_batch_autotune")
    return n.value


def pusch_batch_tuning(b, n_cells: int) -> dict:
    n = 11 + 2 * n_cells
    arr = (ctypes.c_int * n)()
    _check(lib().pusch_batch_tuning(b, arr, n), "pusch_batch_tuning")
    v = list(arr)
    return {"branches": v[0],
            "detector": {2 << c: {"warps": v[1 + 2 * c], "ctas_per_sm": v[2 + 2 * c]} for c in range(5)},
            "beamform": [{"chunk_rows": v[11 + 2 * c], "staged": v[12 + 2 * c]} for c in range(n_cells)]}


def pusch_cnn_param_count() -> int:
    return lib().pusch_cnn_param_count()


def pusch_cnn_forward(n, w, x, params_bf16, y, acts, stream=None) -> None:
    _check(lib().pusch_cnn_forward(n, w, _ptr(x), _ptr(params_bf16), _ptr(y), _ptr(acts), _stream(stream)),
           "pusch_cnn_forward")


def pusch_cnn_backward(n, w, x, acts, params_bf16, y, target, grad, loss, work, wflip, stream=None) -> None:
    _check(lib().pusch_cnn_backward(n, w, _ptr(x), _ptr(acts), _ptr(params_bf16), _ptr(y), _ptr(target), _ptr(grad),
                                    _ptr(loss), _ptr(work), _ptr(wflip), _stream(stream)), "pusch_cnn_backward")


def pusch_cnn_adam(step, lr, beta1, beta2, eps, params, params_bf16, grad, m, v, stream=None) -> None:
    _check(lib().pusch_cnn_adam(step, lr, beta1, beta2, eps, _ptr(params), _ptr(params_bf16), _ptr(grad), _ptr(m),
                                _ptr(v), _stream(stream)), "pusch_cnn_adam")


def pusch_ls_grid(h, n_slots, beam, pilots, grid, scale, stream=None) -> None:
    _check(lib().pusch_ls_grid(h, n_slots, _ptr(beam), _ptr(pilots), _ptr(grid), _ptr(scale), _stream(stream)),
           "pusch_ls_grid")


def pusch_chest_cnn(h, n_slots, beam, pilots, params_bf16, kappa, H_hat, resid=None, fallback=None,
                    stream=None) -> None:
    _check(lib().pusch_chest_cnn(h, n_slots, _ptr(beam), _ptr(pilots), _ptr(params_bf16), kappa, _ptr(H_hat),
                                 _ptr(resid), _ptr(fallback), _stream(stream)), "pusch_chest_cnn")
