"""Oracle: circulant inverse PFB with optional Wiener filtering (FP64).

Test infrastructure only (see oracle/__init__.py).

Steps, in the paper's order (Sec. 3.1, Sec. 4.1, App. C):
  1. recorded spectra -> N-point inverse real FFT per spectrum ("undoing F"),
     giving the [J, N] polyphase array d; column n is d_n (Eq. pfbsubsampled);
  2. per column, J-point DFT along the frame axis: F d_n;
  3. divide by the conjugate sub-filter spectrum (F w_n)^* (Eq. decorrelation),
     optionally Wiener-weighted by H_n (Eq. wiener weights);
  4. inverse J-point DFT; x_hat[j*N + n] = x_hat_n[j].

Readings:
  * Sec. 3.1 extends d_n "to b frames" without saying how; here the recorded
    spectra are J periodic spectra of J frames, so the circulant model is exact
    and exactly J frames are reconstructed.
  * Eq. wiener weights is written for the filter H_n applied before the
    decorrelation; the combined per-mode gain is G = H_n / W_n^* =
    W_n (1 + phi^2) / (|W_n|^2 + phi^2), identical to conj(W)/(|W|^2 + N/S)
    under the opposite DFT sign for W.  phi^2 = 0 is the exact inverse
    1 / W_n^*.  The (1 + phi^2) factor is optional (App. B); `normalize`
    switches it.
"""
from __future__ import annotations

import numpy as np

from .pfb import dequantize


def eigenvalues(window: np.ndarray, nframes: int, ks=None) -> np.ndarray:
    """Sec. 3.1: W_n(k) = (F w_n)_k = sum_r w[r, n] exp(-2 pi i r k / J), the
    J-point DFT of the zero-padded sub-filter w_n (the eigenvalues of the circulant
    W_n^circ).  Direct p-term sum; phases from the exactly reduced (r*k mod J)/J.
    Returns complex [len(ks), N] (all k < J when ks is None)."""
    p, N = window.shape
    J = int(nframes)
    k = np.arange(J, dtype=np.int64) if ks is None else np.asarray(ks, dtype=np.int64)
    out = np.zeros((k.shape[0], N), dtype=np.complex128)
    for r in range(p):
        ph = np.exp(-2j * np.pi * ((r * k) % J).astype(np.float64) / J)
        out += ph[:, None] * window[r][None, :]
    return out


def gain(W: np.ndarray, noise_level: float, normalize: bool = True) -> np.ndarray:
    """Per-mode decorrelation gain G = H_n / W_n^* (Eq. decorrelation with
    Eq. wiener weights): W (1 + phi^2) / (|W|^2 + phi^2); phi^2 = 0 gives 1/W^*."""
    phi2 = float(noise_level)
    if phi2 == 0.0:
        # exact inverse; a mode with W == 0 exactly carries no information and is
        # dropped (the truncated pseudo-inverse of Sec. 4.2.2)
        Wc = np.conj(W)
        safe = np.where(Wc == 0, 1.0, Wc)
        return np.where(Wc == 0, 0.0, 1.0 / safe)
    norm = (1.0 + phi2) if normalize else 1.0
    return W * norm / (np.abs(W) ** 2 + phi2)


def wiener_filter(W: np.ndarray, noise_level: float, normalize: bool = True) -> np.ndarray:
    """Eq. wiener weights: H_n = |W_n|^2 / (|W_n|^2 + phi^2) * (1 + phi^2)."""
    phi2 = float(noise_level)
    norm = (1.0 + phi2) if normalize else 1.0
    a2 = np.abs(W) ** 2
    return a2 / (a2 + phi2) * norm


def frames_from_spectra(spectra: np.ndarray, lblock: int) -> np.ndarray:
    """Step 1: N-point inverse real DFT of every spectrum (normalised 1/N)."""
    return np.fft.irfft(spectra, n=lblock, axis=1)


def decorrelate(d: np.ndarray, window: np.ndarray, noise_level: float,
                normalize: bool = True) -> np.ndarray:
    """Steps 2-4 on the [J, N] polyphase array d: per column, F d_n times G, then
    F^dagger (normalised 1/J).  Returns the [J, N] reconstruction."""
    J, N = d.shape
    D = np.fft.fft(d, axis=0)
    G = gain(eigenvalues(window, J), noise_level, normalize)
    return np.real(np.fft.ifft(G * D, axis=0))


def pinv_gain(W: np.ndarray, threshold: float) -> np.ndarray:
    """Thresholded pseudo-inverse, one of the eigenvalue filters Sec. 3.2 allows on the
    circulant eigenmodes: G = 1 / conj(W) where |W| >= threshold, 0 elsewhere."""
    G = np.zeros(W.shape, dtype=np.complex128)
    keep = np.abs(W) >= threshold
    G[keep] = 1.0 / np.conj(W[keep])
    return G


def full_gain_from_half(gains_half: np.ndarray, nframes: int) -> np.ndarray:
    """Caller-supplied gains [N, J/2 + 1] (modes k <= J/2 of every column) extended to
    all J modes by G(J - k) = conj G(k), the symmetry that keeps the columns real.
    Returns [J, N]."""
    N, K = gains_half.shape
    J = nframes
    assert K == J // 2 + 1
    G = np.zeros((J, N), dtype=np.complex128)
    G[:K] = gains_half.T
    k = np.arange(K, J)
    G[k] = np.conj(gains_half.T[J - k])
    return G


def ipfb_filter(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, threshold: float | None = None,
                gains_half: np.ndarray | None = None) -> np.ndarray:
    """Circulant inverse PFB with a general eigenvalue filter (Sec. 3.2): per column,
    F d_n times G_n, then F^dagger (1/J); G is the thresholded pseudo-inverse
    (pinv_gain) or caller-supplied gains (full_gain_from_half).  Returns x_hat [J*N]."""
    p, N = window.shape
    d = frames_from_spectra(dequantize(codes, scale), N)
    J = d.shape[0]
    if threshold is not None:
        G = pinv_gain(eigenvalues(window, J), threshold)
    else:
        G = full_gain_from_half(np.asarray(gains_half, dtype=np.complex128), J)
    D = np.fft.fft(d, axis=0)
    return np.real(np.fft.ifft(G * D, axis=0)).reshape(-1)


def stream_chunks(nspec: int, chunk: int, margin: int):
    """Chunk starts of the overlap-save inverse: chunks of `chunk` spectra stepping by
    S = chunk - 2 margin, the last one aligned to the end of the run; the chunk at
    `start` contributes frames [start + margin, start + margin + S) (the last one its
    frames up to nspec - margin)."""
    S = chunk - 2 * margin
    assert S > 0 and nspec >= chunk
    starts = list(range(0, nspec - chunk + 1, S))
    if starts[-1] + chunk < nspec:
        starts.append(nspec - chunk)
    return starts


def ipfb_wiener_stream(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, noise_level: float,
                       chunk: int, margin: int, normalize: bool = True) -> np.ndarray:
    """Overlap-save circulant inverse of a long run of spectra (App. C: the Wiener
    decorrelation kernels are short, so a chunk inverted as if periodic is exact up to
    the kernel's tail beyond `margin` frames from its edges): every chunk of `chunk`
    spectra is inverted with ipfb_wiener and its frames margin .. chunk - margin kept.
    Returns frames [margin, nspec - margin) in time order, [(nspec - 2 margin) * N]."""
    p, N = window.shape
    nspec = codes.shape[0]
    out = np.zeros((nspec - 2 * margin, N))
    for st in stream_chunks(nspec, chunk, margin):
        xc = ipfb_wiener(codes[st:st + chunk], scale, window, noise_level, normalize).reshape(chunk, N)
        out[st:st + chunk - 2 * margin] = xc[margin:chunk - margin]
    return out.reshape(-1)


def ipfb_from_spectra(spectra: np.ndarray, window: np.ndarray, noise_level: float,
                      normalize: bool = True) -> np.ndarray:
    """Circulant (Wiener) inverse PFB of complex spectra [J, N/2+1]; returns x_hat [J*N]."""
    p, N = window.shape
    d = frames_from_spectra(spectra, N)
    return decorrelate(d, window, noise_level, normalize).reshape(-1)


def ipfb_wiener(codes: np.ndarray, scale: np.ndarray, window: np.ndarray,
                noise_level: float, normalize: bool = True) -> np.ndarray:
    """Inverse PFB of packed 4-bit codes: dequantize, then ipfb_from_spectra."""
    return ipfb_from_spectra(dequantize(codes, scale), window, noise_level, normalize)


def ipfb_column(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, n: int,
                noise_level: float, normalize: bool = True) -> np.ndarray:
    """Column n of the reconstruction only (x_hat[j*N + n] for all j), for checking
    sampled outputs of full-size runs.  Step 1 is evaluated at the single index n
    as d[j, n] = (1/N) sum over the full Hermitian spectrum of Y[j, c] e^{+2 pi i c n/N}."""
    p, N = window.shape
    Y = dequantize(codes, scale)  # [J, C]
    C = Y.shape[1]
    c = np.arange(C, dtype=np.int64)
    ph = np.exp(2j * np.pi * ((c * n) % N).astype(np.float64) / N)
    wt = np.full(C, 2.0)
    wt[0] = 1.0
    wt[C - 1] = 1.0
    # the Nyquist and DC terms enter once, interior channels twice (conjugate pair)
    dn = np.real(Y @ (wt * ph)) / N
    J = Y.shape[0]
    Dn = np.fft.fft(dn)
    Wn = eigenvalues(window[:, n:n + 1], J)[:, 0]
    G = gain(Wn, noise_level, normalize)
    return np.real(np.fft.ifft(G * Dn))


def data_columns(codes: np.ndarray, scale: np.ndarray, lblock: int, ns, chunk: int = 4096) -> np.ndarray:
    """Columns ns of the polyphase data d (step 1: the N-point inverse real FFT of the
    dequantized spectra), [J, len(ns)], evaluated only at the requested indices (in
    chunks of spectra, so full-size inputs stay cheap)."""
    from .pfb import unpack_codes
    N = lblock
    ns = np.asarray(ns, dtype=np.int64)
    J, half = codes.shape
    C = half + 1
    c = np.arange(C, dtype=np.int64)
    wt = np.full(C, 2.0)
    wt[0] = 1.0
    wt[C - 1] = 1.0
    ph = np.exp(2j * np.pi * ((np.outer(c, ns)) % N).astype(np.float64) / N) * wt[:, None]  # [C, k]
    s = np.asarray(scale, dtype=np.float32).astype(np.float64)
    d = np.empty((J, ns.shape[0]))
    for j0 in range(0, J, chunk):
        q_re, q_im = unpack_codes(codes[j0:j0 + chunk])
        Y = (q_re.astype(np.float64) + 1j * q_im.astype(np.float64)) * s[None, :]
        d[j0:j0 + chunk] = np.real(Y @ ph) / N
    return d


def ipfb_columns(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, ns,
                 noise_level: float, normalize: bool = True, chunk: int = 4096) -> np.ndarray:
    """Columns ns of the reconstruction, [J, len(ns)], evaluating step 1 only at the
    requested indices (data_columns)."""
    p, N = window.shape
    ns = np.asarray(ns, dtype=np.int64)
    J = codes.shape[0]
    d = data_columns(codes, scale, N, ns, chunk)
    out = np.empty_like(d)
    for i, n in enumerate(ns):
        Wn = eigenvalues(window[:, n:n + 1], J)[:, 0]
        out[:, i] = np.real(np.fft.ifft(gain(Wn, noise_level, normalize) * np.fft.fft(d[:, i])))
    return out


# --------------------------------------------------------------------------- #
# Dense brute-force references (pins; tiny sizes only)
# --------------------------------------------------------------------------- #

def dense_pfb_matrix(window: np.ndarray, nframes: int) -> np.ndarray:
    """The periodic PFB as one real matrix P of shape [J*(N+2), J*N]: rows are the
    real and imaginary parts of every rfft channel of every spectrum, built column
    by column from Eq. pfboperator (y = F S W x) applied to unit vectors."""
    p, N = window.shape
    J = int(nframes)
    T = J * N
    C = N // 2 + 1
    P = np.zeros((J * 2 * C, T))
    Fm = np.exp(-2j * np.pi * np.outer(np.arange(C), np.arange(N)) / N)  # [C, N]
    for t in range(T):
        j_in, n = divmod(t, N)
        col = np.zeros((J, C), dtype=np.complex128)
        for r in range(p):
            j_out = (j_in - r) % J  # frame j_in feeds spectrum j_out with tap r
            col[j_out] += window[r, n] * Fm[:, n]
        P[:, t] = np.concatenate([col.real, col.imag], axis=1).reshape(-1)
    return P


def dense_circulant(window_col: np.ndarray, nframes: int) -> np.ndarray:
    """W_n^circ of Eq. circ_convolution: (C x)[j] = sum_r w_r x[(j + r) mod J]."""
    J = int(nframes)
    Cm = np.zeros((J, J))
    for j in range(J):
        for r, wr in enumerate(window_col):
            Cm[j, (j + r) % J] += wr
    return Cm


def tikhonov_column(d_col: np.ndarray, window_col: np.ndarray, noise_level: float,
                    normalize: bool = True) -> np.ndarray:
    """App. C: Tikhonov-regularised least squares for one column,
    (1 + phi^2)(C^T C + phi^2 I)^{-1} C^T d, by a dense solve."""
    J = d_col.shape[0]
    Cm = dense_circulant(window_col, J)
    phi2 = float(noise_level)
    A = Cm.T @ Cm + phi2 * np.eye(J)
    x = np.linalg.solve(A, Cm.T @ d_col)
    return x * ((1.0 + phi2) if normalize else 1.0)


# --------------------------------------------------------------------------- #
# Analytic error spectra (App. B)
# --------------------------------------------------------------------------- #

def analytic_delta_naive(window: np.ndarray, nframes: int, snr: float) -> np.ndarray:
    """App. B: delta(f) = (1/SNR)(1/N) sum_n 1/|W_n(Nf)|^2 for unfiltered
    decorrelation of white input, evaluated at the J sub-stream frequencies."""
    W = eigenvalues(window, nframes)
    return np.mean(1.0 / np.abs(W) ** 2, axis=1) / snr


def analytic_delta_wiener(window: np.ndarray, nframes: int, noise_level: float) -> np.ndarray:
    """App. B: delta(f) = 1 - (1/N) sum_n H_n(Nf) with the un-normalised Wiener
    filter H_n = |W_n|^2/(|W_n|^2 + phi^2), phi^2 = 1/SNR."""
    W = eigenvalues(window, nframes)
    H = wiener_filter(W, noise_level, normalize=False)
    return 1.0 - np.mean(H, axis=1)
