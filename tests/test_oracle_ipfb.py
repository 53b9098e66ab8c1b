"""Pins for the oracle's eigenvalues, circulant inverse and Wiener filter."""
import json
import os

import numpy as np
import pytest

from oracle import ipfb, pfb
from paper_2608_23441_b300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def test_eigenvalues_are_fft_of_zero_padded_kernel():
    # Sec. 3.1: each eigen-spectrum is the FFT of the zero-padded sub-filter w_n.
    N, p, J = 16, 4, 40
    w = pfb.sinc_hamming_window(N, p)
    W = ipfb.eigenvalues(w, J)
    pad = np.zeros((J, N))
    pad[:p] = w
    assert np.allclose(W, np.fft.fft(pad, axis=0), atol=1e-13)
    # circulant eigen-relation: C v_k = conj(W_k) v_k for v_k[j] = exp(2 pi i jk/J)
    n, k = 5, 7
    Cm = ipfb.dense_circulant(w[:, n], J)
    v = np.exp(2j * np.pi * np.arange(J) * k / J)
    assert np.allclose(Cm @ v, np.conj(W[k, n]) * v, atol=1e-12)


@pytest.mark.parametrize("p,path", [(4, "half"), (2, "half"), (5, "zero"), (3, "zero")])
def test_symmetric_window_has_zero_nyquist_eigenvalue(p, path):
    # App. A: a symmetric window that vanishes at its edge gives a zero eigenvalue at
    # the Nyquist frequency, for path N/2 (p even) or path 0 (p odd).
    N, J = 32, 64
    w = pfb.symmetric_sinc_hann_window(N, p)
    W = ipfb.eigenvalues(w, J)
    n = N // 2 if path == "half" else 0
    assert abs(W[J // 2, n]) < 1e-14
    # other paths stay away from zero there
    others = np.delete(np.abs(W[J // 2]), n)
    assert others.min() > 1e-4


def test_sinc_hamming_is_only_nearly_singular():
    # App. A: numpy's Hamming is not exactly symmetric, so the worst eigenvalue is small
    # but not zero; it sits at path N/2, Nyquist.
    N, p, J = 256, 4, 512
    W = np.abs(ipfb.eigenvalues(pfb.sinc_hamming_window(N, p), J))
    k, n = np.unravel_index(np.argmin(W), W.shape)
    assert n == N // 2 and k == J // 2
    assert 1e-4 < W.min() < 1e-2


@pytest.mark.parametrize("N,J", [(8, 16), (64, 96), (256, 512)])
def test_exact_recovery_periodic_unquantized(N, J):
    # Eq. decorrelation on circulant data recovers the input to round-off (Fig. kernels
    # caption: approaches floating-point precision).
    p = 4
    x = synth.gaussian_stream(N * J, 21)
    w = pfb.sinc_hamming_window(N, p)
    xh = ipfb.ipfb_from_spectra(pfb.pfb_spectra(x, w), w, 0.0)
    assert np.linalg.norm(xh - x) / np.linalg.norm(x) < 1e-10


def test_exact_inverse_equals_dense_solve():
    # Brute force: the full periodic PFB as a dense real matrix (rows: Re and Im of every
    # channel of every spectrum).  Dropping the identically-zero Im rows of DC and
    # Nyquist leaves a square T x T system; solving it directly must give the circulant
    # inverse (Eq. decorrelation) for any Hermitian-consistent spectra.
    N, p, J = 8, 4, 16
    w = pfb.sinc_hamming_window(N, p)
    P = ipfb.dense_pfb_matrix(w, J)
    C = N // 2 + 1
    keep = np.ones((J, 2 * C), bool)
    keep[:, C] = False          # Im of DC
    keep[:, 2 * C - 1] = False  # Im of Nyquist
    keep = keep.reshape(-1)
    assert np.abs(P[~keep]).max() < 1e-14
    Ps = P[keep]
    assert Ps.shape == (N * J, N * J)
    rng = np.random.default_rng(2)
    y = rng.standard_normal((J, C)) + 1j * rng.standard_normal((J, C))
    y[:, 0] = y[:, 0].real
    y[:, -1] = y[:, -1].real
    rhs = np.concatenate([y.real, y.imag], axis=1).reshape(-1)[keep]
    x_lu = np.linalg.solve(Ps, rhs)
    assert np.allclose(ipfb.ipfb_from_spectra(y, w, 0.0), x_lu, atol=1e-9)
    # and the dense forward matches pfb_spectra on data
    x = synth.gaussian_stream(N * J, 4)
    Y = pfb.pfb_spectra(x, w)
    assert np.allclose((P @ x).reshape(J, -1),
                       np.concatenate([Y.real, Y.imag], axis=1), atol=1e-12)


def test_wiener_equals_scaled_tikhonov():
    # App. C: Wiener-filtered circulant inversion equals (1 + phi^2) times the Tikhonov
    # solution (C^T C + phi^2 I)^{-1} C^T d in the circulant model.
    N, p, J = 8, 4, 24
    w = pfb.sinc_hamming_window(N, p)
    rng = np.random.default_rng(3)
    d = rng.standard_normal((J, N))
    phi2 = 0.02
    X = ipfb.decorrelate(d, w, phi2, normalize=True)
    for n in range(N):
        assert np.allclose(X[:, n], ipfb.tikhonov_column(d[:, n], w[:, n], phi2, True), atol=1e-11)
    X0 = ipfb.decorrelate(d, w, phi2, normalize=False)
    assert np.allclose(X0 * (1 + phi2), X, atol=1e-12)


def test_wiener_tends_to_exact_inverse():
    N, p, J = 32, 4, 64
    w = pfb.sinc_hamming_window(N, p)
    x = synth.gaussian_stream(N * J, 9)
    Y = pfb.pfb_spectra(x, w)
    e1 = np.linalg.norm(ipfb.ipfb_from_spectra(Y, w, 1e-7) - x)
    e2 = np.linalg.norm(ipfb.ipfb_from_spectra(Y, w, 1e-8) - x)
    assert e2 < e1
    assert 5 < e1 / e2 < 15  # error proportional to phi^2


def test_wiener_on_pure_eigenmode():
    # A single real mode k of sub-stream n comes back scaled by H_n(k) (Eq. wiener weights).
    N, p, J = 16, 4, 64
    w = pfb.sinc_hamming_window(N, p)
    n, k, phi2 = 8, 29, 0.01
    xcol = np.cos(2 * np.pi * k * np.arange(J) / J + 0.3)
    X = np.zeros((J, N))
    X[:, n] = xcol
    d = pfb.polyphase_sum(X.reshape(-1), w)
    out = ipfb.decorrelate(d, w, phi2, normalize=True)
    H = ipfb.wiener_filter(ipfb.eigenvalues(w, J), phi2, True)
    assert np.allclose(out[:, n], H[k, n] * xcol, atol=1e-12)
    assert np.abs(np.delete(out, n, axis=1)).max() < 1e-12


def test_sampled_column_matches_full_inverse():
    N, p, J = 32, 4, 48
    w = pfb.sinc_hamming_window(N, p)
    x = synth.stream_config(N, J, 5, channel=3.3)
    codes, scale, _ = pfb.pfb_forward(x, w)
    full = ipfb.ipfb_wiener(codes, scale, w, 0.014).reshape(J, N)
    for n in (0, 1, N // 2, N - 1):
        assert np.allclose(ipfb.ipfb_column(codes, scale, w, n, 0.014), full[:, n], atol=1e-12)
    # the sampled forms evaluate step 1 (the inverse real FFT) at single indices, in
    # chunks of spectra that do not divide J
    cols = [0, 3, N // 2, N - 1]
    d = ipfb.frames_from_spectra(pfb.dequantize(codes, scale), N)
    assert np.allclose(ipfb.data_columns(codes, scale, N, cols, chunk=20), d[:, cols], atol=1e-12)
    assert np.allclose(ipfb.ipfb_columns(codes, scale, w, cols, 0.014, chunk=20), full[:, cols], atol=1e-12)


def _mc_delta(N, J, w, phi2, noise_level, reps, seed):
    rng = np.random.default_rng(seed)
    num = np.zeros(N * J)
    den = np.zeros(N * J)
    for _ in range(reps):
        x = rng.standard_normal(N * J)
        d = pfb.polyphase_sum(x, w) + np.sqrt(phi2) * rng.standard_normal((J, N))
        xh = ipfb.decorrelate(d, w, noise_level, normalize=False).reshape(-1)
        X = np.fft.fft(x)
        num += np.abs(X - np.fft.fft(xh)) ** 2
        den += np.abs(X) ** 2
    # fold the N images of each sub-stream frequency k = F mod J
    return num.reshape(N, J).sum(0) / den.reshape(N, J).sum(0)


def test_analytic_error_spectra_match_monte_carlo():
    # App. B: delta(f) = 1 - mean_n H_n(Nf) (Wiener) and (1/SNR) mean_n 1/|W_n|^2 (naive)
    # for white input and white additive noise; Monte-Carlo must agree.
    N, p, J = 16, 4, 128
    w = pfb.sinc_hamming_window(N, p)
    phi2 = 0.02
    an_w = ipfb.analytic_delta_wiener(w, J, phi2)
    mc_w = _mc_delta(N, J, w, phi2, phi2, 300, 0)
    assert np.all(np.abs(mc_w / an_w - 1) < 0.15)
    an_n = ipfb.analytic_delta_naive(w, J, 1.0 / phi2)
    # the naive decorrelation uses phi^2 -> 0 in the filter
    rng_reps = 300
    num = np.zeros(J)
    den = np.zeros(J)
    rng = np.random.default_rng(1)
    for _ in range(rng_reps):
        x = rng.standard_normal(N * J)
        d = pfb.polyphase_sum(x, w) + np.sqrt(phi2) * rng.standard_normal((J, N))
        xh = ipfb.decorrelate(d, w, 0.0).reshape(-1)
        X = np.fft.fft(x)
        num += (np.abs(X - np.fft.fft(xh)) ** 2).reshape(N, J).sum(0)
        den += (np.abs(X) ** 2).reshape(N, J).sum(0)
    assert np.all(np.abs((num / den) / an_n - 1) < 0.15)


def test_delta_at_channel_centre():
    # App. B: near a channel centre delta = 1/(1 + SNR); Sec. 4.3 reports about 1.1 %.
    N, p, J = 2048, 4, 64
    w = pfb.sinc_hamming_window(N, p)
    snr = GOLD["quantizer_snr_at_optimal_step"]["value"]
    dc = ipfb.analytic_delta_wiener(w, J, 1.0 / snr)[0]
    assert abs(dc - 1.0 / (1.0 + snr)) < 0.1 / (1.0 + snr)
    assert abs(dc - GOLD["delta_channel_centre"]["value"]) < 0.003
    # exactly 1/(1+SNR) when every W_n(0) = 1
    wn = w / w.sum(axis=0, keepdims=True)
    d0 = ipfb.analytic_delta_wiener(wn, J, 1.0 / snr)[0]
    assert abs(d0 - 1.0 / (1.0 + snr)) < 1e-12


# ----------------------------------------------------------------------------- general eigenvalue filters
def test_pinv_threshold_zero_recovers_periodic_input():
    # Sec. 3.2: with no mode dropped the thresholded pseudo-inverse is the exact inverse,
    # which recovers unquantized circulant data to round-off.
    N, J, p = 64, 128, 4
    x = synth.gaussian_stream(N * J, 23)
    w = pfb.sinc_hamming_window(N, p)
    d = pfb.polyphase_sum(x, w)
    D = np.fft.fft(d, axis=0)
    G = ipfb.pinv_gain(ipfb.eigenvalues(w, J), 0.0)
    xh = np.real(np.fft.ifft(G * D, axis=0)).reshape(-1)
    assert np.linalg.norm(xh - x) / np.linalg.norm(x) < 1e-10


def test_pinv_keeps_or_drops_a_pure_eigenmode():
    # one real mode k of sub-stream n: kept exactly when |W_n(k)| >= threshold, removed otherwise
    N, p, J = 16, 4, 64
    w = pfb.sinc_hamming_window(N, p)
    n, k = 8, 29
    xcol = np.cos(2 * np.pi * k * np.arange(J) / J + 0.3)
    X = np.zeros((J, N))
    X[:, n] = xcol
    d = pfb.polyphase_sum(X.reshape(-1), w)
    D = np.fft.fft(d, axis=0)
    Wk = abs(ipfb.eigenvalues(w, J)[k, n])
    for thr, expect in ((0.5 * Wk, xcol), (2.0 * Wk, 0.0 * xcol)):
        out = np.real(np.fft.ifft(ipfb.pinv_gain(ipfb.eigenvalues(w, J), thr) * D, axis=0))
        assert np.allclose(out[:, n], expect, atol=1e-12)
        assert np.abs(np.delete(out, n, axis=1)).max() < 1e-12


def test_caller_gains_identity_and_scaled_inverse():
    # G = 1 leaves the polyphase data d as it is; G = c / conj(W) on a pure mode returns c x
    N, p, J = 32, 4, 64
    codes = synth.random_code_bytes(J, N // 2, 31)
    scale = synth.random_scale(N // 2 + 1, 32)
    w = pfb.sinc_hamming_window(N, p)
    ones = np.ones((N, J // 2 + 1), dtype=np.complex128)
    d = ipfb.frames_from_spectra(pfb.dequantize(codes, scale), N)
    assert np.allclose(ipfb.ipfb_filter(codes, scale, w, gains_half=ones), d.reshape(-1), atol=1e-12)
    n, k, c = 5, 13, 0.7
    xcol = np.cos(2 * np.pi * k * np.arange(J) / J - 1.1)
    X = np.zeros((J, N))
    X[:, n] = xcol
    dm = pfb.polyphase_sum(X.reshape(-1), w)
    W = ipfb.eigenvalues(w, J)
    Gh = (c / np.conj(W[: J // 2 + 1])).T                       # [N, J/2+1]
    out = np.real(np.fft.ifft(ipfb.full_gain_from_half(Gh, J) * np.fft.fft(dm, axis=0), axis=0))
    assert np.allclose(out[:, n], c * xcol, atol=1e-12)


# ----------------------------------------------------------------------------- overlap-save inverse
def test_stream_chunks_cover_the_interior_once():
    for nspec, chunk, margin in ((1000, 256, 32), (256, 256, 0), (300, 128, 16)):
        starts = ipfb.stream_chunks(nspec, chunk, margin)
        covered = np.zeros(nspec, dtype=int)
        S = chunk - 2 * margin
        for k, st in enumerate(starts):
            covered[st + margin:st + chunk - margin] += 1
        assert np.all(covered[margin:nspec - margin] >= 1)
        assert starts[0] == 0 and starts[-1] + chunk == nspec


def test_stream_inverse_converges_to_the_global_inverse():
    # App. C: the Wiener kernels decay within tens of frames, so the overlap-save inverse
    # of a periodic run approaches the run's global circulant inverse as the margin grows;
    # one chunk over the whole run with no margin is the global inverse itself
    N, p, J = 64, 4, 1024
    x = synth.gaussian_stream(N * J, 91)
    w = pfb.sinc_hamming_window(N, p)
    codes, scale, _ = pfb.pfb_forward(x, w)
    phi2 = 0.0141
    ref = ipfb.ipfb_wiener(codes, scale, w, phi2).reshape(J, N)
    assert np.allclose(ipfb.ipfb_wiener_stream(codes, scale, w, phi2, J, 0), ref.reshape(-1))
    errs = []
    for margin in (4, 16, 64, 112):
        got = ipfb.ipfb_wiener_stream(codes, scale, w, phi2, 256, margin).reshape(-1, N)
        want = ref[margin:J - margin]
        errs.append(np.sqrt(np.mean((got - want) ** 2) / np.mean(want ** 2)))
    assert all(b < a for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < 1e-6, errs
