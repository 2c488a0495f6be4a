"""Pins of the FP64 CNN oracle (learned channel-estimate denoiser): parameter count of the literal 4-layer
net, closed forms, a library correlation special case, bfloat16 rounding, and finite-difference gradients
over every layer."""
import numpy as np
import pytest

RNG = np.random.default_rng(77)
CH = [2, 32, 32, 32, 2]


def offsets():
    out, off = [], 0
    for k in range(4):
        w = CH[k + 1] * CH[k] * 9
        out.append((off, off + w, off + w + CH[k + 1]))   # W start, b start, end
        off += w + CH[k + 1]
    return out


def test_parameter_count(orc):
    # 2*32*9+32 + 2*(32*32*9+32) + 32*2*9+2 = 19682 (the 4-layer net; "~30k" in the workload text would need
    # a fifth 32->32 layer)
    assert orc.cnn_param_count() == 19682 == offsets()[-1][2]


def test_zero_weights_is_identity_plus_last_bias(orc):
    p = np.zeros(orc.cnn_param_count())
    x = RNG.standard_normal((3, 2, 2, 9))
    y, _ = orc.cnn_forward(p, x)
    assert np.array_equal(y, x)
    o = offsets()
    p[o[3][1]:o[3][2]] = [0.5, -0.25]
    y, _ = orc.cnn_forward(p, x)
    assert np.allclose(y[:, 0], x[:, 0] + 0.5) and np.allclose(y[:, 1], x[:, 1] - 0.25)


def test_conv_matches_library_correlation(orc):
    """Layers 1-3 carry channel 0/1 through (positive inputs, centre taps = 1); layer 4 applies random 3x3
    kernels: the output must equal scipy's zero-padded 2-D correlation plus the residual."""
    signal = pytest.importorskip("scipy.signal")
    p = np.zeros(orc.cnn_param_count())
    o = offsets()
    for k in range(3):
        W = p[o[k][0]:o[k][1]].reshape(CH[k + 1], CH[k], 3, 3)
        W[0, 0, 1, 1] = 1.0
        W[1, 1, 1, 1] = 1.0
    W4 = RNG.standard_normal((2, 32, 3, 3))
    W4[:, 2:] = 0.0
    p[o[3][0]:o[3][1]] = W4.ravel()
    x = np.abs(RNG.standard_normal((2, 2, 2, 11)))
    y, acts = orc.cnn_forward(p, x)
    for s in range(2):
        for co in range(2):
            want = x[s, co].copy()
            for ci in range(2):
                want += signal.correlate2d(x[s, ci], W4[co, ci], mode="same", boundary="fill")
            assert np.allclose(y[s, co], want, atol=1e-12)
    assert np.allclose(acts[0][:, :2], x) and np.all(acts[0][:, 2:] == 0)


def test_relu_cuts_negative_paths(orc):
    p = np.zeros(orc.cnn_param_count())
    o = offsets()
    for k in range(3):
        W = p[o[k][0]:o[k][1]].reshape(CH[k + 1], CH[k], 3, 3)
        W[0, 0, 1, 1] = 1.0
    W4 = p[o[3][0]:o[3][1]].reshape(2, 32, 3, 3)
    W4[0, 0, 1, 1] = 1.0
    x = RNG.standard_normal((1, 2, 2, 6))
    y, _ = orc.cnn_forward(p, x)
    assert np.allclose(y[0, 0], x[0, 0] + np.maximum(x[0, 0], 0)) and np.allclose(y[0, 1], x[0, 1])


def test_bf16_rounding(orc):
    vals = [1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.0 - 2 ** -7, 3.14159, 1e-30, 65504.0]
    want = [1.0, 1.0, 1.015625, -2.0, 3.140625, None, 65536.0]
    got = orc.round_bf16(vals)
    for g, w in zip(got, want):
        if w is not None:
            assert g == w
    torch = pytest.importorskip("torch")
    v = RNG.standard_normal(1000) * 10.0 ** RNG.integers(-5, 5, 1000)
    ref = torch.tensor(v, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(orc.round_bf16(v), ref)


@pytest.mark.parametrize("bf16", [False, True])
def test_gradients_match_finite_differences(orc, bf16):
    n_p = orc.cnn_param_count()
    p = RNG.standard_normal(n_p) * 0.15
    x = RNG.standard_normal((2, 2, 2, 6))
    t = RNG.standard_normal((2, 2, 2, 6))
    loss, g = orc.cnn_loss_grad(p, x, t)
    o = offsets()
    picks = []
    for k in range(4):
        picks += list(RNG.integers(o[k][0], o[k][1], 4)) + [int(RNG.integers(o[k][1], o[k][2]))]
    eps = 1e-6
    for i in picks:
        q = p.copy()
        q[i] += eps
        lp, _ = orc.cnn_loss_grad(q, x, t)
        q[i] -= 2 * eps
        lm, _ = orc.cnn_loss_grad(q, x, t)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])
    if bf16:
        # the bf16 mode rounds where a bfloat16 implementation stores values; its loss stays close
        lb, gb = orc.cnn_loss_grad(p, x, t, bf16=True)
        assert abs(lb - loss) < 0.05 * loss
        assert np.linalg.norm(gb - g) < 0.1 * np.linalg.norm(g)


def test_dilation_shifts_by_the_layer_dilation(orc):
    """A single right-hand tap in layer 2 (dilation 8) or layer 3 (dilation 16) moves the signal by 8 or 16
    subcarriers; layers 1 and 4 use dilation 1."""
    o = offsets()
    for layer, d in ((1, 8), (2, 16)):
        p = np.zeros(orc.cnn_param_count())
        for k in range(3):
            W = p[o[k][0]:o[k][1]].reshape(CH[k + 1], CH[k], 3, 3)
            if k == layer:
                W[0, 0, 1, 2] = 1.0            # in[x + d]
            else:
                W[0, 0, 1, 1] = 1.0
        W4 = p[o[3][0]:o[3][1]].reshape(2, 32, 3, 3)
        W4[0, 0, 1, 1] = 1.0
        x = np.abs(RNG.standard_normal((1, 2, 2, 40)))
        y, _ = orc.cnn_forward(p, x)
        want = np.zeros_like(x[0, 0])
        want[:, :40 - d] = x[0, 0][:, d:]
        assert np.allclose(y[0, 0] - x[0, 0], want, atol=1e-14)
