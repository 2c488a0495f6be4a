"""CPU-side checks of the C ABI: the library builds and loads, exports every symbol include/pusch.h
declares, and rejects invalid configurations on the host (these paths make no CUDA call)."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def B():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2210_09196_gb300 import binding
    return binding


def declared_functions():
    text = (ROOT / "include" / "pusch.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pusch_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_stage_and_chain_entry_points():
    names = declared_functions()
    for n in ("pusch_ofdm_fft", "pusch_beamform", "pusch_chest_ls", "pusch_mmse_detect", "pusch_slot"):
        assert n in names


def test_library_exports_every_declared_symbol(B):
    lib = ctypes.CDLL(str(B.LIB_PATH))
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(B.EXPORTS)


def test_version_and_pitch(B):
    assert "sm_103a" in B.pusch_version()
    cfg = B.make_cfg(n_rx=64, n_fft=4096, n_sc=3276, n_beams=32, n_layers=16)
    assert B.pusch_sc_pitch(cfg) == 3328                  # FP32 form: the mixed form's planes, 64-element rows
    cfg8 = B.make_cfg(n_rx=64, n_fft=4096, n_sc=3276, n_beams=32, n_layers=16, form=B.PUSCH_FORM_FP8)
    assert B.pusch_sc_pitch(cfg8) == 3328                 # 128-byte rows of E4M3 codes
    cfgm = B.make_cfg(n_rx=64, n_fft=4096, n_sc=3200, n_beams=32, n_layers=16, form=B.PUSCH_FORM_MIXED)
    assert B.pusch_sc_pitch(cfgm) == 3200


def _good(**kw):
    from paper_2210_09196_gb300 import binding as B
    base = dict(n_rx=16, n_fft=512, n_sc=300, n_beams=16, n_layers=4, qam_bits=2, noise_var=0.01)
    base.update(kw)
    return B.make_cfg(**base)


@pytest.mark.parametrize("bad,code", [
    (dict(n_fft=500), -5), (dict(n_fft=8192), -5), (dict(n_sc=0), -1), (dict(n_sc=600), -1),
    (dict(n_beams=65), -5), (dict(n_layers=17), -1), (dict(n_layers=33, n_beams=64), -1),
    (dict(qam_bits=3), -1), (dict(noise_var=-0.5), -1), (dict(noise_var=float("nan")), -1),
    (dict(comb=0), -1), (dict(ports=[0, 1, 2, 4]), -1), (dict(dmrs_sym=(2, 2)), -1), (dict(dmrs_sym=(2, 14)), -1),
    (dict(n_sym=2), -1), (dict(form=7), -1), (dict(n_rx=0), -5), (dict(chol_every=-1), -1),
    (dict(chol_every=13), -1),
])
def test_invalid_configs_are_rejected_on_the_host(B, bad, code):
    cfg = _good(**bad)
    out = ctypes.c_size_t()
    rc = B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out))
    assert rc == code
    assert B.pusch_last_error()
    h = ctypes.c_void_p(123)
    assert B.lib().pusch_create(ctypes.byref(h), ctypes.byref(cfg), 1) == code
    assert h.value is None


def test_prefix_needs_512_points(B):
    out = ctypes.c_size_t()
    cfg = _good(n_fft=256, n_sc=200, cp=True)
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == B.PUSCH_ERR_UNSUPPORTED
    cfg = _good(cp=True, shift_7p5khz=True)
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == 0
    cfg.cp = 2
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == B.PUSCH_ERR_ARG


@pytest.mark.parametrize("bad,code", [
    (dict(n_layers=5, n_beams=16), -1), (dict(ports=[0, 1, 1, 2]), -1), (dict(ports=[0, 1, 2, 4]), -1),
    (dict(n_sc=302), -1),
])
def test_type1_dmrs_rules(B, bad, code):
    kw = dict(dmrs_type=1, ports=[0, 1, 2, 3])
    kw.update(bad)
    cfg = _good(**kw)
    out = ctypes.c_size_t()
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == code


def test_type1_noise_estimate_mode_is_accepted(B):
    cfg = _good(dmrs_type=1, ports=[0, 1, 2, 3], noise_var=B.PUSCH_NOISE_ESTIMATE)
    out = ctypes.c_size_t()
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == 0


def test_type1_pilot_generator_arguments(B):
    ok = _good(dmrs_type=1, ports=[0, 1, 2, 3])
    comb = _good()
    sl = (ctypes.c_int * 1)(0)
    assert B.lib().pusch_dmrs_type1_pilots(ctypes.byref(comb), 1, sl, 0, 0, 16, None) == B.PUSCH_ERR_ARG
    assert B.lib().pusch_dmrs_type1_pilots(ctypes.byref(ok), 1, sl, 70000, 0, 16, None) == B.PUSCH_ERR_ARG
    assert B.lib().pusch_dmrs_type1_pilots(ctypes.byref(ok), 1, sl, 0, 2, 16, None) == B.PUSCH_ERR_ARG
    sl[0] = 160
    assert B.lib().pusch_dmrs_type1_pilots(ctypes.byref(ok), 1, sl, 0, 0, 16, None) == B.PUSCH_ERR_ARG
    assert B.lib().pusch_dmrs_type1_pilots(ctypes.byref(ok), 0, None, 0, 0, None, None) == B.PUSCH_OK


def test_noise_estimate_mode_is_accepted(B):
    cfg = _good(noise_var=B.PUSCH_NOISE_ESTIMATE)
    out = ctypes.c_size_t()
    assert B.lib().pusch_workspace_size(ctypes.byref(cfg), 1, ctypes.byref(out)) == 0


def test_workspace_size(B):
    cfg = _good()
    n = B.pusch_workspace_size(cfg, 2)
    # FFT out + beams + LS pilot table + interpolated estimate
    per_slot = 14 * 16 * 300 * 8 + 14 * 300 * 16 * 8 + 4 * 75 * 16 * 8 + 300 * 4 * 16 * 8
    assert n >= 2 * per_slot and n < 2 * per_slot + 64 * 1024


def test_workspace_size_of_the_time_varying_estimate(B):
    """chol_every = 4 over 12 data symbols: two LS tables (one per DMRS symbol) and three estimates."""
    n0 = B.pusch_workspace_size(_good(), 2)
    n4 = B.pusch_workspace_size(_good(chol_every=4), 2)
    assert n4 - n0 >= 2 * (4 * 75 * 16 * 8 + 2 * 300 * 4 * 16 * 8)
    assert n4 - n0 < 2 * (4 * 75 * 16 * 8 + 2 * 300 * 4 * 16 * 8) + 64 * 1024


def test_null_handle_and_bad_batch_rejected(B):
    L = B.lib()
    assert L.pusch_ofdm_fft(None, 1, 1, 1, None) == B.PUSCH_ERR_ARG
    assert L.pusch_slot(None, 1, 1, 1, 1, 1, 1, None, None) == B.PUSCH_ERR_ARG
    assert L.pusch_destroy(None) == B.PUSCH_OK
    assert L.pusch_set_pipeline(None, 2) == B.PUSCH_ERR_ARG
    with pytest.raises(B.PuschError):
        B.pusch_ofdm_fft(None, 1, 1, 1, stream=0)


def test_binding_rejects_non_contiguous_buffers(B):
    torch = pytest.importorskip("torch")
    t = torch.zeros((4, 6), dtype=torch.complex64).t()
    with pytest.raises(ValueError):
        B._ptr(t)
    c = t.contiguous()
    assert B._ptr(c) == c.data_ptr()


def test_header_compiles_as_c99(tmp_path):
    """The boundary is a C ABI: the public header must compile as strict C99, not only as CUDA C++."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = Path(__file__).resolve().parents[1]
    src = tmp_path / "abi.c"
    src.write_text('#include "include/pusch.h"\n'
                   "int main(void) { pusch_cell_cfg c; c.dmrs_type = 1; c.cp = 0; (void)c;\n"
                   "  return pusch_version() != 0 ? 0 : 1; }\n")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", f"-I{root}",
                        str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_status_and_selftest_arguments_are_checked_on_the_host(B):
    L = B.lib()
    assert L.pusch_selftest_wait(None, 1000, None) == B.PUSCH_ERR_ARG
    assert L.pusch_selftest_wait(123, 0, None) == B.PUSCH_ERR_ARG          # limit below 1 us
    assert L.pusch_selftest_wait(123, 2000000, None) == B.PUSCH_ERR_ARG    # limit above 1 s
    assert "limit_us" in B.pusch_last_error()


def test_noalloc_refuses_the_time_varying_estimate_on_the_host(B):
    """chol_every > 0 needs a handle: refused before any CUDA call (the pointers are never touched)."""
    cfg = _good(chol_every=4)
    rc = B.lib().pusch_slot_noalloc(ctypes.byref(cfg), 1, 16, 16, 16, 16, 16, None, None)
    assert rc == B.PUSCH_ERR_UNSUPPORTED
    assert "chol_every" in B.pusch_last_error()


def test_autotune_rejects_a_null_handle(B):
    n = ctypes.c_int(7)
    assert B.lib().pusch_autotune(None, None, None, ctypes.byref(n)) == B.PUSCH_ERR_ARG
