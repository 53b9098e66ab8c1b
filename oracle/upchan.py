"""Oracle: up-channelization (re-channelization) of a reconstructed stream (FP64).

Test infrastructure only (see oracle/__init__.py).

Sec. 4.3 re-channelizes the inverted stream with frames 64 times longer than the
original PFB to reach 64x finer channels.  Reading used here: a plain real DFT
(no window) of consecutive, non-overlapping blocks of L samples starting at
t = 0, X_b[c] = sum_{t<L} x[b L + t] exp(-2 pi i t c / L), c <= L/2; a trailing
partial block is dropped.  pfb_upchannelize is the paper's windowed form: a PFB
with frames L samples long and p taps (Sec. 4.3, "channelized again using a PFB
with 64-times longer frame size"), periodic over the stream's blocks.
"""
from __future__ import annotations

import numpy as np


def upchannelize(x: np.ndarray, block: int) -> np.ndarray:
    """Block real DFT: complex128 [floor(T/L), L/2 + 1]."""
    L = int(block)
    nb = x.shape[0] // L
    return np.fft.rfft(np.asarray(x[:nb * L], dtype=np.float64).reshape(nb, L), axis=1)


def pfb_upchannelize(x: np.ndarray, window: np.ndarray) -> np.ndarray:
    """Windowed re-channelization with frames L = window.shape[1] long and p =
    window.shape[0] taps: per block b, s_b[t] = sum_{r<p} w[r, t] x[((b + r) mod nb) L + t]
    (the polyphase sum of Eq. pfb with N -> L, periodic over the nb = floor(T/L)
    blocks), then X_b = rfft(s_b).  complex128 [nb, L/2 + 1]."""
    p, L = window.shape
    nb = x.shape[0] // L
    xb = np.asarray(x[:nb * L], dtype=np.float64).reshape(nb, L)
    s = np.zeros((nb, L))
    for r in range(p):
        s += window[r][None, :] * np.roll(xb, -r, axis=0)
    return np.fft.rfft(s, axis=1)


def upchannelize_block(x: np.ndarray, block: int, b: int) -> np.ndarray:
    """Spectrum of block b only (for sampled checks of full-size runs)."""
    L = int(block)
    return np.fft.rfft(np.asarray(x[b * L:(b + 1) * L], dtype=np.float64))


def brute_rdft(seg: np.ndarray) -> np.ndarray:
    """O(L^2) direct evaluation of the same transform (pin for tiny L)."""
    L = seg.shape[0]
    t = np.arange(L)
    c = np.arange(L // 2 + 1)
    ph = np.exp(-2j * np.pi * ((np.outer(c, t)) % L) / L)
    return ph @ seg
