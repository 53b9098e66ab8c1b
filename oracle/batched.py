"""Oracle: batched inverse PFB of many independent streams (FP64).

Test infrastructure only (see oracle/__init__.py).  Each stream is inverted on its
own by ipfb.ipfb_wiener (Eq. decorrelation, Eq. wiener weights); the frame count J
may be any integer (numpy's FFT handles every length), so the circulant of size J is
never padded.
"""
from __future__ import annotations

from .ipfb import ipfb_wiener


def ipfb_batched(streams, normalize: bool = True):
    """streams: iterable of (codes, scale, window, noise_level).  Returns a list of x_hat."""
    return [ipfb_wiener(c, s, w, nl, normalize) for (c, s, w, nl) in streams]
