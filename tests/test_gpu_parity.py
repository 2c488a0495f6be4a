"""GPU parity: every stage of the CUDA path, called through the C ABI, against the FP64 oracle on the same
seeded inputs. Plain FP32 form: norm-relative error <= 1e-5 per stage (each stage fed the same inputs on
both sides), hard decisions identical except where the oracle's symbol sits on a decision threshold
within the observed error."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import binding as B
from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def nrel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def c128(t):
    return t.detach().cpu().numpy().astype(np.complex128)


def bits_agree(bits_gpu, x_orc, x_gpu, q, f32=True):
    """Hard decisions of the GPU vs the oracle's decisions on the oracle's symbols; a mismatch is allowed
    only where the oracle component lies within 4x the observed error of a threshold (tie-ambiguous)."""
    import oracle
    b_orc = oracle.demap(x_orc, q)
    mism = bits_gpu != b_orc
    if not mism.any():
        return 0, 0
    err = np.max(np.abs(x_gpu - x_orc))
    thr = [0.0] if q == 2 else [0.0, 2 / np.sqrt(10)]
    comp = np.minimum(np.min([np.abs(np.abs(x_orc.real) - t) for t in thr], axis=0),
                      np.min([np.abs(np.abs(x_orc.imag) - t) for t in thr], axis=0))
    ambiguous = comp <= 4 * err + 1e-7
    hard = mism & ~ambiguous
    return int(mism.sum()), int(hard.sum())


@pytest.fixture(scope="module")
def small_slots():
    return synth.make_slots(synth.SMALL_FP32, 3)


def run_stages(rx, slots, W):
    t = host.time_tensor(slots)
    p = host.pilot_tensor(slots)
    Wt = host.beam_tensor(W)
    freq = rx.ofdm_fft(t)
    beam = rx.beamform(freq, Wt)
    H = rx.chest_ls(beam, p)
    x, b, st = rx.mmse_detect(H, beam)
    torch.cuda.synchronize()
    return freq, beam, H, x, b, st


def test_small_slot_each_stage_fp32(orc, small_slots):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=len(small_slots))
    freq, beam, H, x, b, st = run_stages(rx, small_slots, small_slots[0].W)
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    for i, s in enumerate(small_slots):
        f_orc = orc.ofdm_demod(s.time_as_complex128(), cell.n_sc)
        assert nrel(c128(freq[i]), f_orc) < TOL
        fg = c128(freq[i])
        assert nrel(c128(beam[i]), orc.beamform(fg, s.W)) < TOL
        bg = c128(beam[i])
        assert nrel(c128(H[i]), orc.chest_ls(bg, s.pilots, s.ports, cell.comb)) < TOL
        Hg = c128(H[i])
        xo, fails = orc.mmse(Hg, bg, s.noise_var)
        assert fails == 0
        xg = c128(x[i])
        assert nrel(xg, xo) < TOL
        # the detector's own decisions, taken in single precision on its own symbols, are bit-exact
        assert np.array_equal(b[i].cpu().numpy(), orc.demap(xg, cell.qam_bits, f32=True))
        mism, hard = bits_agree(b[i].cpu().numpy(), xo, xg, cell.qam_bits)
        assert hard == 0
    rx.close()


def test_small_slot_chain_vs_oracle_chain(orc, small_slots):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=len(small_slots))
    x, b, st = rx.slot(host.time_tensor(small_slots), host.beam_tensor(small_slots[0].W),
                       host.pilot_tensor(small_slots))
    torch.cuda.synchronize()
    assert list(st.cpu().numpy()) == [0, 0, -1, 0]
    for i, s in enumerate(small_slots):
        xo, bo, fails = orc.run_slot(s)
        xg = c128(x[i])
        assert nrel(xg, xo) < TOL
        _, hard = bits_agree(b[i].cpu().numpy(), xo, xg, cell.qam_bits)
        assert hard == 0
    rx.close()


# shapes: several tiles and ragged tails in every dimension; FFT sizes 64..4096; every layer class
SHAPES = [
    dict(n_rx=5, n_fft=64, n_sc=37, n_beams=5, n_layers=1, qam_bits=2),
    dict(n_rx=8, n_fft=128, n_sc=100, n_beams=8, n_layers=2, qam_bits=4),
    dict(n_rx=33, n_fft=256, n_sc=255, n_beams=12, n_layers=3, qam_bits=4),
    dict(n_rx=16, n_fft=512, n_sc=512, n_beams=16, n_layers=8, qam_bits=2),
    dict(n_rx=40, n_fft=1024, n_sc=601, n_beams=24, n_layers=7, qam_bits=4),
    dict(n_rx=64, n_fft=2048, n_sc=1638, n_beams=40, n_layers=16, qam_bits=4),
    dict(n_rx=70, n_fft=4096, n_sc=3276, n_beams=64, n_layers=32, qam_bits=4),
    # the 16- and 32-lane classes with padded lanes (identity rows), odd beam counts (8-byte staging) and
    # beam counts whose row stride is below the lane count (the data-symbol rows padded to it). Square or
    # nearly square H is avoided: its Gram matrices reach condition numbers near 1e4, where a plain FP32
    # Cholesky (LAPACK) is itself 2e-5 from the FP64 result; these shapes stay below 2e-6 there.
    dict(n_rx=12, n_fft=256, n_sc=200, n_beams=12, n_layers=9, qam_bits=2),
    dict(n_rx=24, n_fft=512, n_sc=300, n_beams=15, n_layers=12, qam_bits=4),
    dict(n_rx=20, n_fft=512, n_sc=333, n_beams=20, n_layers=17, qam_bits=4),
    dict(n_rx=48, n_fft=1024, n_sc=720, n_beams=33, n_layers=25, qam_bits=2),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda d: f"R{d['n_rx']}N{d['n_fft']}sc{d['n_sc']}B{d['n_beams']}L{d['n_layers']}")
@pytest.mark.parametrize("in_fp16", [False, True])
def test_stage_parity_over_shapes(orc, shape, in_fp16):
    cell = synth.CellConfig("t", snr_db=25.0, channel="pdp", beam="dft", in_fp16=in_fp16, seed=11, **shape)
    slots = synth.make_slots(cell, 2)
    rx = host.Receiver(host.cfg_for(cell), max_slots=2)
    freq, beam, H, x, b, st = run_stages(rx, slots, slots[0].W)
    assert st.cpu().numpy()[0] == 0
    rng = np.random.default_rng(0)
    for i, s in enumerate(slots):
        pairs = [(int(a), int(r)) for a, r in zip(rng.integers(0, 14, 6), rng.integers(0, cell.n_rx, 6))]
        f_orc = orc.ofdm_demod(s.time_as_complex128(), cell.n_sc, pairs=pairs)
        fg = c128(freq[i])
        for (sy, r) in pairs:
            assert nrel(fg[sy, r], f_orc[sy, r]) < TOL
        bg = c128(beam[i])
        assert nrel(bg, orc.beamform(fg, s.W)) < TOL
        Hg = c128(H[i])
        assert nrel(Hg, orc.chest_ls(bg, s.pilots, s.ports, cell.comb)) < TOL
        sc = np.unique(np.concatenate([[0, cell.n_sc - 1], rng.integers(0, cell.n_sc, 40)]))
        xo, fails = orc.mmse(Hg, bg, s.noise_var, sc_list=sc)
        assert fails == 0
        xg = c128(x[i])
        assert nrel(xg[:, :, sc], xo[:, :, sc]) < TOL
    rx.close()


def test_fused_chain_equals_staged_estimation_and_detection(orc, small_slots):
    """pusch_slot forms the estimate inside the detector; it must equal pusch_chest_ls + pusch_mmse_detect."""
    for cell in (synth.SMALL_FP32, synth.DEPLOY.with_(n_rx=16, n_beams=16, n_layers=8, n_fft=1024, n_sc=600)):
        slots = small_slots if cell is synth.SMALL_FP32 else synth.make_slots(cell, 2)
        rx = host.Receiver(host.cfg_for(cell), max_slots=len(slots))
        freq, beam, H, x, b, st = run_stages(rx, slots, slots[0].W)
        x2, b2, st2 = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
        torch.cuda.synchronize()
        assert nrel(c128(x2), c128(x)) < 1e-6
        assert torch.equal(st, st2)
        assert (b2 != b).float().mean().item() < 1e-4
        rx.close()


@pytest.mark.parametrize("nl,nb,n_sc", [(16, 32, 300), (12, 32, 123), (32, 64, 77), (16, 64, 64), (20, 32, 45)],
                         ids=lambda v: str(v))
def test_detector_interpolating_from_the_pilot_table_is_bit_identical(orc, nl, nb, n_sc):
    """With 16 or 32 lanes per subcarrier and 32 or 64 beams, pusch_slot's detector interpolates the estimate
    from the LS table at the pilots while it stages (Section II: linear interpolation between a layer's pilot
    subcarriers), so the interpolated estimate never goes through memory. Its x-hat, bits and status must be
    bit-identical to pusch_chest_ls (which writes the interpolated estimate) followed by pusch_mmse_detect, over
    ragged last CTAs, slot boundaries, padded layers (12 and 20 layers) and the held edges before the first and
    after the last pilot."""
    cell = synth.DEPLOY.with_(n_rx=nb, n_beams=nb, n_layers=nl, n_fft=512, n_sc=n_sc)
    slots = synth.make_slots(cell, 3)
    rx = host.Receiver(host.cfg_for(cell), max_slots=len(slots))
    freq, beam, H, x, b, st = run_stages(rx, slots, slots[0].W)
    x2, b2, st2 = rx.slot(host.time_tensor(slots), host.beam_tensor(slots[0].W), host.pilot_tensor(slots))
    torch.cuda.synchronize()
    assert torch.equal(x2, x) and torch.equal(b2, b) and torch.equal(st2, st)
    assert int(st2.cpu().numpy()[0]) == 0
    for i, s in enumerate(slots):   # and the chain against the oracle's estimate + Eq. 2 on sampled subcarriers
        Ho = orc.chest_ls(c128(beam[i]), s.pilots, s.ports, cell.comb)
        sc = np.array([0, 1, n_sc // 2, n_sc - 2, n_sc - 1])
        xo, fails = orc.mmse(Ho, c128(beam[i]), s.noise_var, sc_list=sc)
        assert fails == 0
        assert nrel(c128(x2[i])[:, :, sc], xo[:, :, sc]) < TOL
    rx.close()


def test_profile_hooks_time_pusch_slot(orc, small_slots):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=3)
    args = (host.time_tensor(small_slots), host.beam_tensor(small_slots[0].W), host.pilot_tensor(small_slots))
    B.pusch_profile_start(rx.h, 2)
    for _ in range(3):
        rx.slot(*args)
    ms, n = B.pusch_profile_read(rx.h)
    assert n == 2 and all(v > 0 for v in ms.values()) and set(ms) == {"fft", "beamform", "ls", "detect"}
    ms, n = B.pusch_profile_read(rx.h)
    assert n == 0 and all(v == 0 for v in ms.values())
    rx.close()


def test_zero_slots_is_a_no_op(orc):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=1)
    t = torch.empty(0, device="cuda")
    B.pusch_slot(rx.h, 0, t, t, t, t, t, None)
    B.pusch_ofdm_fft(rx.h, 0, t, t)
    torch.cuda.synchronize()
    with pytest.raises(B.PuschError):
        B.pusch_slot(rx.h, 2, t, t, t, t, t, None)  # more than max_slots
    rx.close()


def test_singular_gram_sets_pivot_status(orc):
    # zero channel estimate and sigma^2 = 0: every Gram is singular -> pivot flag, count, first index
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell, noise_var=0.0), max_slots=2)
    H = torch.zeros((2, cell.n_sc, cell.n_layers, cell.n_beams), dtype=torch.complex64, device="cuda")
    H[0, 7:] = 1.0  # slot 0: subcarriers >= 7 have rank-1 H (singular for 4 layers); 0..6 are zero
    beam = torch.ones((2, 14, cell.n_sc, cell.n_beams), dtype=torch.complex64, device="cuda")
    x, b, st = rx.mmse_detect(H, beam)
    torch.cuda.synchronize()
    stat = st.cpu().numpy().astype(np.int64) & 0xffffffff
    assert stat[0] & B.PUSCH_STATUS_PIVOT
    assert stat[1] == 2 * cell.n_sc
    assert stat[2] == 0
    assert np.all(np.isfinite(x.cpu().numpy()))
    rx.close()


def test_nonfinite_input_flags_status(orc):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=1)
    s = synth.make_slot(cell, 0)
    t = host.time_tensor([s])
    t[0, 5, 3, 17] = complex(float("nan"), 0.0)
    x, b, st = rx.slot(t, host.beam_tensor(s.W), host.pilot_tensor([s]))
    torch.cuda.synchronize()
    assert st.cpu().numpy()[0] & (B.PUSCH_STATUS_NONFINITE | B.PUSCH_STATUS_PIVOT)
    rx.close()


def test_diagonal_loading_matches_oracle(orc):
    cell = synth.SMALL_FP32
    s = synth.make_slot(cell, 1)
    rx = host.Receiver(host.cfg_for(cell, loading=0.5), max_slots=1)
    freq, beam, H, x, b, st = run_stages(rx, [s], s.W)
    xo, _ = orc.mmse(c128(H[0]), c128(beam[0]), s.noise_var, loading=0.5)
    assert nrel(c128(x[0]), xo) < TOL
    rx.close()


def test_deterministic_reruns(orc, small_slots):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=3)
    args = (host.time_tensor(small_slots), host.beam_tensor(small_slots[0].W), host.pilot_tensor(small_slots))
    x1, b1, _ = rx.slot(*args)
    x2, b2, _ = rx.slot(*args)
    torch.cuda.synchronize()
    assert torch.equal(x1, x2) and torch.equal(b1, b2)
    rx.close()


def test_host_buffer_entry_point_equals_device_entry_point(orc, small_slots):
    cell = synth.SMALL_FP32
    rx = host.Receiver(host.cfg_for(cell), max_slots=3)
    W = host.beam_tensor(small_slots[0].W)
    xd, bd, sd = rx.slot(host.time_tensor(small_slots), W, host.pilot_tensor(small_slots))
    out = (rx.xhat_buffer(3, "cpu").pin_memory(), rx.bits_buffer(3, "cpu").pin_memory(),
           rx.status_buffer("cpu").pin_memory())
    xh, bh, sh = rx.slot_host(host.time_tensor(small_slots, "cpu", pin=True), W,
                              host.pilot_tensor(small_slots, "cpu", pin=True), out)
    torch.cuda.synchronize()
    assert torch.equal(xh, xd.cpu()) and torch.equal(bh, bd.cpu()) and torch.equal(sh, sd.cpu())
    rx.close()
