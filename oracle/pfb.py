"""Oracle: window, forward critically-sampled PFB, 4-bit quantizer (FP64).

Test infrastructure only (see oracle/__init__.py).

Readings of the paper used here:
  * Eq. chan_dft / Eq. pfb print `sinc[m - M/2]`, `h[rN + M]` and the exponent
    `mk/N`; read as sinc((m - M/2)/N), h[rN + n] and exp(-2 pi i n k / N).
  * Hamming taper with numpy's cos(2 pi m/(M-1)) normalisation (App. A).
  * n_chan = N/2 in Sec. 2.2; the real FFT here keeps N/2 + 1 channels (DC and
    Nyquist have exactly zero imaginary part).
  * Quantizer: 15-level mid-tread, levels -7..7 (Sec. 4.3), with a per-channel
    step Delta_c = RMS_c / 2.5.  The decision is taken in float32:
    code = clamp(rint(v_f32 / Delta_f32), -7, 7), rint rounding half to even,
    a zero step gives code 0.
"""
from __future__ import annotations

import numpy as np


def sinc_hamming_window(lblock: int, ntap: int) -> np.ndarray:
    """Sec. 2.2 (Eq. chan_dft, the text after Eq. pfb) and App. A:
    w[m] = sinc((m - M/2)/N) * (0.54 - 0.46 cos(2 pi m/(M-1))), m < M = ntap*N,
    returned reshaped as the [ntap, N] window array of Sec. 2.3."""
    N, p = int(lblock), int(ntap)
    M = N * p
    m = np.arange(M, dtype=np.float64)
    t = (m - M / 2.0) / N
    sinc = np.ones(M)
    nz = t != 0.0
    sinc[nz] = np.sin(np.pi * t[nz]) / (np.pi * t[nz])
    taper = 0.54 - 0.46 * np.cos(2.0 * np.pi * m / (M - 1))
    return (sinc * taper).reshape(p, N)


def symmetric_sinc_hann_window(lblock: int, ntap: int) -> np.ndarray:
    """An exactly symmetric window with w[0] = 0 and w[m] = w[M - m] (the two
    requirements of App. A): sinc((m - M/2)/N) times a period-M Hann taper."""
    N, p = int(lblock), int(ntap)
    M = N * p
    m = np.arange(M, dtype=np.float64)
    t = (m - M / 2.0) / N
    sinc = np.ones(M)
    nz = t != 0.0
    sinc[nz] = np.sin(np.pi * t[nz]) / (np.pi * t[nz])
    taper = 0.5 - 0.5 * np.cos(2.0 * np.pi * m / M)
    return (sinc * taper).reshape(p, N)


def polyphase_sum(x: np.ndarray, window: np.ndarray, periodic: bool = True) -> np.ndarray:
    """Sec. 2.3: the window array slides down the [frames, N] data array one frame
    at a time; spectrum j is fed by frames j..j+p-1, each multiplied by its window
    row, summed over rows:  d[j, n] = sum_r w[r, n] x[(j + r) N + n].
    periodic=True wraps frame indices mod J (the circulant model of Eq.
    circ_convolution: J spectra from J frames); otherwise J - p + 1 spectra."""
    p, N = window.shape
    X = np.asarray(x, dtype=np.float64).reshape(-1, N)
    J = X.shape[0]
    if periodic:
        d = np.zeros((J, N))
        for r in range(p):
            d += window[r][None, :] * X[(np.arange(J) + r) % J]
    else:
        Jo = J - p + 1
        d = np.zeros((Jo, N))
        for r in range(p):
            d += window[r][None, :] * X[r:r + Jo]
    return d


def pfb_spectra(x: np.ndarray, window: np.ndarray, periodic: bool = True) -> np.ndarray:
    """Eq. pfb: polyphase sum followed by the N-point DFT exp(-2 pi i n k/N) of
    each summed frame, positive-frequency half (N/2 + 1 channels)."""
    d = polyphase_sum(x, window, periodic)
    return np.fft.rfft(d, axis=1)


def channel_rms(spectra: np.ndarray) -> np.ndarray:
    """RMS of the real and imaginary parts of each channel over all spectra, in
    FP64.  Interior channels: sqrt(sum(Re^2 + Im^2) / (2 J)); DC and Nyquist have
    no imaginary part: sqrt(sum(Re^2) / J)."""
    J, C = spectra.shape
    re2 = np.sum(spectra.real ** 2, axis=0)
    im2 = np.sum(spectra.imag ** 2, axis=0)
    rms = np.sqrt((re2 + im2) / (2.0 * J))
    rms[0] = np.sqrt(re2[0] / J)
    rms[C - 1] = np.sqrt(re2[C - 1] / J)
    return rms


def channel_scale(spectra: np.ndarray, divisor: float = 2.5) -> np.ndarray:
    """Per-channel quantizer step Delta_c = RMS_c / 2.5, rounded once to float32."""
    return (channel_rms(spectra) / divisor).astype(np.float32)


def quantize_f32(values: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Sec. 4.3 mid-tread 15-level quantizer on float32 inputs:
    code = clamp(rint(v / Delta), -7, 7) with an IEEE float32 divide and rint
    rounding half to even; Delta == 0 gives code 0.  `values` float32 [..., C],
    `scale` float32 [C].  Returns int8 codes."""
    v = np.asarray(values, dtype=np.float32)
    s = np.broadcast_to(np.asarray(scale, dtype=np.float32), v.shape)
    with np.errstate(divide="ignore", invalid="ignore"):
        q = np.rint(np.divide(v, s, dtype=np.float32))
    q = np.where(s == 0, np.float32(0), q)
    q = np.clip(q, -7, 7)
    return q.astype(np.int8)


def quantize_spectra(spectra: np.ndarray, scale: np.ndarray):
    """Quantize the real and imaginary parts separately after rounding the FP64
    spectra to float32.  Returns (q_re, q_im) int8 [J, C]."""
    re = spectra.real.astype(np.float32)
    im = spectra.imag.astype(np.float32)
    return quantize_f32(re, scale), quantize_f32(im, scale)


def pack_codes(q_re: np.ndarray, q_im: np.ndarray) -> np.ndarray:
    """Folded 4-bit layout, N/2 bytes per spectrum.  Byte c (0 < c < N/2) holds
    Re_c in the low nibble and Im_c in the high nibble, two's complement.  Byte 0
    holds Re_0 (low) and Re_{N/2} (high): DC and Nyquist have zero imaginary
    part, so nothing is lost."""
    J, C = q_re.shape
    half = C - 1
    lo = q_re[:, :half].astype(np.int16) & 0xF
    hi = q_im[:, :half].astype(np.int16) & 0xF
    hi[:, 0] = q_re[:, half].astype(np.int16) & 0xF
    return (lo | (hi << 4)).astype(np.uint8)


def unpack_codes(codes: np.ndarray):
    """Inverse of pack_codes: (q_re, q_im) int8 [J, N/2 + 1]."""
    c = np.asarray(codes, dtype=np.uint8)
    J, half = c.shape
    lo = (c & 0xF).astype(np.int16)
    hi = (c >> 4).astype(np.int16)
    lo = np.where(lo >= 8, lo - 16, lo)
    hi = np.where(hi >= 8, hi - 16, hi)
    q_re = np.zeros((J, half + 1), dtype=np.int8)
    q_im = np.zeros((J, half + 1), dtype=np.int8)
    q_re[:, :half] = lo
    q_im[:, 1:half] = hi[:, 1:]
    q_re[:, half] = hi[:, 0]
    return q_re, q_im


def dequantize(codes: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Recorded spectra q * Delta_c as complex FP64 [J, N/2 + 1]."""
    q_re, q_im = unpack_codes(codes)
    s = np.asarray(scale, dtype=np.float32).astype(np.float64)
    return (q_re.astype(np.float64) + 1j * q_im.astype(np.float64)) * s[None, :]


def pfb_forward(x: np.ndarray, window: np.ndarray, scale: np.ndarray | None = None,
                periodic: bool = True):
    """Forward PFB with 4-bit quantization (the simulation of Sec. 4.3).
    Returns (codes uint8 [J, N/2], scale float32 [N/2+1], spectra complex128)."""
    spec = pfb_spectra(x, window, periodic)
    if scale is None:
        scale = channel_scale(spec)
    q_re, q_im = quantize_spectra(spec, scale)
    return pack_codes(q_re, q_im), np.asarray(scale, dtype=np.float32), spec


def quantization_snr(sigma: float, step: float, nsamples: int, seed: int) -> float:
    """App. B: SNR = Var[s] / Var[s - Q(s)] of the 15-level quantizer on Gaussian
    samples of standard deviation `sigma` with level spacing `step` (FP64)."""
    rng = np.random.default_rng(seed)
    s = rng.standard_normal(nsamples) * sigma
    q = np.clip(np.rint(s / step), -7, 7) * step
    return float(np.var(s) / np.var(s - q))
