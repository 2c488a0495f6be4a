"""Ill-conditioned Gram matrices: where the FP32 detector (Eq. 2 by Cholesky and two triangular solves, Section
V-C) stays within the 1e-5 parity bar of the FP64 oracle and where it does not.

The channel estimate is square or nearly square (N_B = N_L, N_L + 1), so H^H H is close to singular and only
sigma^2 (+ the extra loading delta) bounds the condition number kappa(G) of G = H^H H + (sigma^2 + delta) I.
Both sides get the same FP32 inputs (the oracle widens them to FP64) and the same sigma^2 + delta. Standard
backward-error analysis of forming G, r = H^H y in FP32 and of the Cholesky solves bounds the relative error of
x per subcarrier by about (N_B + N_L) kappa(G) u, u = 2^-24; the test checks that bound per subcarrier, that the
1e-5 bar holds while kappa(G) stays below 1e2, and that loading lowers both kappa and the error. The printed
table (run with -s) is the record of error against condition number."""
import numpy as np
import pytest
import torch

from paper_2210_09196_gb300 import host, synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
N_SC = 192


def _case(nl, nb, sigma2, seed):
    rng = np.random.default_rng(seed)
    H = ((rng.standard_normal((N_SC, nl, nb)) + 1j * rng.standard_normal((N_SC, nl, nb))) / np.sqrt(2))
    x = (rng.choice([-1.0, 1.0], (nl, 14, N_SC)) + 1j * rng.choice([-1.0, 1.0], (nl, 14, N_SC))) / np.sqrt(2)
    n = np.sqrt(sigma2 / 2) * (rng.standard_normal((14, N_SC, nb)) + 1j * rng.standard_normal((14, N_SC, nb)))
    y = np.einsum("alb,lsa->sab", H, x) + n          # y[s][a][b] = sum_l H[a][l][b] x[l][s][a] + n
    return H.astype(np.complex64), y.astype(np.complex64)


def _kappa(H, load):
    G = np.einsum("alb,amb->alm", H.conj(), H) + load * np.eye(H.shape[1])[None]
    ev = np.linalg.eigvalsh(G)
    return ev[:, -1] / ev[:, 0]


def _run(orc, nl, nb, sigma2, loading, seed):
    H, y = _case(nl, nb, sigma2, seed)
    cell = synth.SMALL_FP32.with_(n_rx=nb, n_beams=nb, n_layers=nl, n_sc=N_SC, qam_bits=2)
    rx = host.Receiver(host.cfg_for(cell, noise_var=sigma2, loading=loading), max_slots=1)
    x, b, st = rx.mmse_detect(torch.from_numpy(H[None]).cuda(), torch.from_numpy(y[None]).cuda())
    torch.cuda.synchronize()
    rx.close()
    xg = x[0].cpu().numpy().astype(np.complex128)
    H64, y64 = H.astype(np.complex128), y.astype(np.complex128)
    xo, fails = orc.mmse(H64, y64, sigma2, loading=loading)
    kap = _kappa(H64, sigma2 + loading)
    err_sc = np.linalg.norm((xg - xo).reshape(-1, N_SC), axis=0) / np.linalg.norm(xo.reshape(-1, N_SC), axis=0)
    err = float(np.linalg.norm(xg - xo) / np.linalg.norm(xo))
    return err, err_sc, kap, int(st.cpu().numpy()[0]), fails


CASES = [(nl, nb) for nl in (4, 16, 32) for nb in (nl, nl + 1)]
SIGMAS = (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6)


@pytest.mark.parametrize("nl,nb", CASES, ids=lambda v: str(v))
def test_fp32_detector_error_against_condition_number(orc, nl, nb):
    rows = []
    for i, s2 in enumerate(SIGMAS):
        err, err_sc, kap, st, fails = _run(orc, nl, nb, s2, 0.0, seed=100 * nl + nb + i)
        assert st == 0 and fails == 0
        # the FP32 error bound per subcarrier, (N_B + N_L) kappa u (with a factor 2 of slack)
        bound = 2.0 * (nb + nl) * kap * U32
        assert np.all(err_sc <= bound + 1e-7), (s2, float(np.max(err_sc / bound)))
        # the parity bar holds while kappa stays below 1e2
        if np.max(kap) < 1e2:
            assert err <= 1e-5, (s2, err, float(np.max(kap)))
        rows.append((s2, float(np.median(kap)), float(np.max(kap)), err, float(np.max(err_sc))))
    print(f"\nN_L={nl} N_B={nb}: sigma2, median kappa, max kappa, norm-rel err, worst subcarrier err")
    for r in rows:
        print("  %.0e  %.3e  %.3e  %.3e  %.3e" % r)
    # smaller sigma^2, larger kappa, larger error (square H): the error follows the conditioning
    assert rows[-1][3] > rows[0][3]


@pytest.mark.parametrize("nl", (16, 32))
def test_loading_bounds_the_condition_number_and_the_error(orc, nl):
    s2, delta = 1e-6, 1e-3
    err0, _, kap0, _, _ = _run(orc, nl, nl, s2, 0.0, seed=7)
    err1, err_sc1, kap1, st, fails = _run(orc, nl, nl, s2, delta, seed=7)
    assert st == 0 and fails == 0
    assert np.max(kap1) < np.max(kap0) and err1 < err0
    assert np.all(err_sc1 <= 2.0 * (2 * nl) * kap1 * U32 + 1e-7)
    print(f"\nN_L=N_B={nl}, sigma2=1e-6: max kappa {np.max(kap0):.3e} -> {np.max(kap1):.3e} with delta=1e-3, "
          f"error {err0:.3e} -> {err1:.3e}")
