"""Pins for the oracle's up-channelization and ML / conjugate-gradient solve."""
import numpy as np
import pytest

from oracle import ipfb, ml, pfb, upchan
from paper_2608_23441_b300 import synth


def test_upchannelize_brute_dft_and_parseval():
    L = 64
    x = synth.gaussian_stream(5 * L + 17, 1)   # trailing partial block dropped
    X = upchannelize = upchan.upchannelize(x, L)
    assert X.shape == (5, L // 2 + 1)
    for b in range(5):
        seg = x[b * L:(b + 1) * L]
        assert np.allclose(X[b], upchan.brute_rdft(seg), atol=1e-11)
        # Parseval for a real block: sum x^2 = (|X0|^2 + 2 sum |Xc|^2 + |X_{L/2}|^2) / L
        e = (abs(X[b, 0]) ** 2 + 2 * np.sum(abs(X[b, 1:-1]) ** 2) + abs(X[b, -1]) ** 2) / L
        assert e == pytest.approx(np.sum(seg ** 2), rel=1e-12)
    assert upchannelize is X


def test_upchannelize_bin_centred_tone():
    L, c0 = 256, 37
    t = np.arange(3 * L)
    x = np.cos(2 * np.pi * c0 * t / L)
    X = upchan.upchannelize(x, L)
    mag = np.abs(X)
    assert np.allclose(mag[:, c0], L / 2, rtol=1e-12)
    mag[:, c0] = 0
    assert mag.max() < 1e-9


def _problem(N=8, p=4, J=32, seed=0, frac=0.2, noise=1e-2):
    w = pfb.sinc_hamming_window(N, p)
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((J, N))
    d = pfb.polyphase_sum(x.reshape(-1), w) + np.sqrt(noise) * rng.standard_normal((J, N))
    mask = (rng.uniform(size=(J, N)) < frac).astype(np.float64)
    return w, x, d, mask


def test_operator_fft_equals_stencil_and_explicit_CtC():
    w, x, d, mask = _problem(N=16, J=40)
    V = np.random.default_rng(5).standard_normal(d.shape)
    A1 = ml.normal_operator_fft(w, V, 0.3, mask, 1.7)
    A2 = ml.normal_operator_stencil(w, V, 0.3, mask, 1.7)
    assert np.allclose(A1, A2, atol=1e-12)
    A3 = ml.apply_CT(w, ml.apply_C(w, V)) / 0.3 + 1.7 * mask * V
    assert np.allclose(A1, A3, atol=1e-12)
    # C^T is the transpose of C: <C u, v> = <u, C^T v> per column
    U = np.random.default_rng(6).standard_normal(d.shape)
    assert np.allclose(np.sum(ml.apply_C(w, U) * V, 0), np.sum(U * ml.apply_CT(w, V), 0))
    # and C is exactly the periodic polyphase sum
    assert np.allclose(ml.apply_C(w, U), pfb.polyphase_sum(U.reshape(-1), w))


@pytest.mark.parametrize("precond", ["none", "wiener"])
def test_cg_matches_dense_normal_equations(precond):
    # Eq. chi squared: the minimiser solves the dense normal equations column by column.
    w, x, d, mask = _problem()
    sig2 = 1e-2
    X, it, rel = ml.ml_solve_d(d, w, sig2, mask, x, 1.0, precond, 1e-12, 2000)
    assert np.all(rel <= 1e-12)
    for n in range(d.shape[1]):
        ref = ml.dense_ml_column(d[:, n], w[:, n], sig2, mask[:, n], x[:, n], 1.0)
        assert np.allclose(X[:, n], ref, rtol=0, atol=1e-9 * np.abs(ref).max())
    tr = ml.true_relative_residual(d, w, sig2, mask, x, 1.0, X)
    assert np.all(tr < 1e-10)


def test_toy_model_single_saved_sample():
    # Sec. 4.2.2: symmetric window, no quantization: path N/2 loses its Nyquist mode
    # (null vector alternating +-1); one saved sample pins it and the solve is exact.
    N, p, J = 16, 4, 64
    w = pfb.symmetric_sinc_hann_window(N, p)
    x = np.random.default_rng(3).standard_normal((J, N))
    d = pfb.polyphase_sum(x.reshape(-1), w)
    # without a prior the alternating mode is invisible to chi^2
    alt = (-1.0) ** np.arange(J)
    assert np.abs(ml.apply_C(w[:, N // 2:N // 2 + 1], alt[:, None])).max() < 1e-14
    mask = np.zeros((J, N))
    mask[11, N // 2] = 1.0
    X, it, rel = ml.ml_solve_d(d, w, 1.0, mask, x, 1.0, "none", 1e-13, 5000)
    assert np.linalg.norm(X - x) / np.linalg.norm(x) < 1e-8


def test_wiener_pcg_exact_without_mask():
    # With an empty mask the Wiener preconditioner is the exact inverse: one iteration.
    w, x, d, _ = _problem(N=16, J=64)
    mask = np.zeros_like(d)
    X, it, rel = ml.ml_solve_d(d, w, 0.05, mask, x, 1.0, "wiener", 1e-10, 50)
    assert np.all(it == 1)
    # and the answer is the exact circulant inverse of d
    assert np.allclose(X, ipfb.decorrelate(d, w, 0.0), atol=1e-8)


def test_cg_residual_and_error_decrease():
    # CG minimises the A-norm of the error monotonically (Shewchuk 1994).
    w, x, d, mask = _problem(N=8, J=48, seed=4)
    sig2 = 1e-2
    Xs = [ml.ml_solve_d(d, w, sig2, mask, x, 1.0, "none", 0.0, k)[0] for k in range(0, 12)]
    Xstar = ml.ml_solve_d(d, w, sig2, mask, x, 1.0, "none", 1e-13, 3000)[0]
    A = lambda V: ml.normal_operator_fft(w, V, sig2, mask, 1.0)  # noqa: E731
    enorm = [np.sum((X - Xstar) * A(X - Xstar), axis=0) for X in Xs]
    for a, b in zip(enorm[:-1], enorm[1:]):
        assert np.all(b <= a * (1 + 1e-9) + 1e-18)


def test_paper_protocol_wiener_start_improves_chi2():
    # Sec. 4.3: Wiener initial guess, then 25 CG iterations; chi^2 must not increase.
    w, x, d, mask = _problem(N=16, J=64, seed=7)
    sig2 = 1e-2
    x0 = ml.wiener_initial_guess(d, w, 0.01)

    def chi2(X):
        r = d - ml.apply_C(w, X)
        return np.sum(r * r) / sig2 + np.sum(mask * (X - x) ** 2)

    X25 = ml.ml_solve_d(d, w, sig2, mask, x, 1.0, "none", 0.0, 25, x0=x0)[0]
    assert chi2(X25) < chi2(x0)


def test_path_sample_mask_fraction_and_layout():
    # Sec. 4.3: saving every R-th sample of L of N sub-filter paths keeps beta = L / (R N)
    N, J, R = 2048, 64, 4
    for beta, L_expect in ((0.01, 82), (0.10, 820)):     # the paper's 82 ... 820 paths
        L = synth.saved_paths(N, beta, R)
        assert L == L_expect
        m = synth.path_sample_mask(N, J, L, R).reshape(J, N)
        assert abs(m.mean() - L / (R * N)) < 1e-15
        cols = np.nonzero(m.any(axis=0))[0]
        assert cols.size == L and cols[0] == N // 2 - L // 2 and cols[-1] == N // 2 + L // 2 - 1
        assert np.array_equal(np.nonzero(m.any(axis=1))[0], np.arange(0, J, R))


def test_pfb_upchannelize_reduces_to_block_dft_and_matches_pfb():
    # one tap of unit weight is the plain block DFT; p taps are the forward PFB of
    # Eq. pfb with the frame length N replaced by L
    L, nb = 256, 12
    x = synth.gaussian_stream(L * nb + 37, 71)
    assert np.allclose(upchan.pfb_upchannelize(x, np.ones((1, L))), upchan.upchannelize(x, L), atol=1e-10)
    w = pfb.sinc_hamming_window(L, 4)
    ref = pfb.pfb_spectra(x[:L * nb], w, periodic=True)
    assert np.allclose(upchan.pfb_upchannelize(x, w), ref, atol=1e-9)
    # a tone at the centre of fine channel c0 stays in c0 (the flat PFB passband)
    c0 = 40
    t = np.arange(L * nb)
    X = upchan.pfb_upchannelize(np.cos(2 * np.pi * c0 * t / L), w)
    pw = np.mean(np.abs(X) ** 2, axis=0)
    assert pw[c0] > 1e3 * np.delete(pw, c0).max()


def test_ml_stream_single_chunk_is_the_solve_and_chunks_stitch_in_place():
    from oracle import pfb as opfb
    # One chunk covering the run (margin 0) is exactly ml_solve.  With the prior on
    # every sample (a short-ranged inverse operator, decay of a few frames) the chunked
    # solve agrees with the solve of the whole run on every kept frame, which checks
    # the chunk starts, the kept range and the stitching offsets: a one-frame shift
    # anywhere fails.
    from oracle import ml as oml
    N, p, J = 8, 4, 192
    rng = np.random.default_rng(3)
    w = opfb.sinc_hamming_window(N, p)
    x = rng.standard_normal(J * N)
    codes, scale, spec = opfb.pfb_forward(x, w)
    mask = np.ones(J * N, np.uint8)
    sig2, lam = 0.02, 50.0   # |W|^2 / sigma^2 + lam within [50, 100]: decay well under a frame
    xa, ia, ra = oml.ml_solve(codes, scale, w, sig2, mask, x, lam, "wiener", 1e-12, 500)
    xs, is_, rs = oml.ml_solve_stream(codes, scale, w, sig2, mask, x, J, 0, lam, "wiener", 1e-12, 500)
    assert np.array_equal(xs, xa) and np.array_equal(is_, ia)
    chunk, margin = 64, 24
    xs, _, _ = oml.ml_solve_stream(codes, scale, w, sig2, mask, x, chunk, margin, lam, "wiener", 1e-12, 500)
    ref = xa.reshape(J, N)[margin:J - margin].reshape(-1)
    assert np.max(np.abs(xs - ref)) <= 1e-8 * np.max(np.abs(ref))
    # a stitching error shows: the same solve shifted by one frame is far off
    shifted = xa.reshape(J, N)[margin + 1:J - margin + 1].reshape(-1)
    assert np.max(np.abs(xs - shifted)) > 0.1 * np.max(np.abs(ref))
