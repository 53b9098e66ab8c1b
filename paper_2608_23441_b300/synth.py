"""Seeded synthetic inputs shaped like the paper's simulated workloads.

This module draws random numbers only; it holds none of the method's
arithmetic (no window formula, no PFB, no quantizer, no inversion).  Both the
CUDA path's tests/benchmark and the FP64 oracle take their inputs from here.

The paper's own data are synthetic white noise (Sec. 4.3): a standard-normal
time stream, optionally with weak tones.  All generators use numpy's PCG64
(`numpy.random.default_rng(seed)`) in float64.
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_stream(nsamples: int, seed: int) -> np.ndarray:
    """White standard-normal time stream, float64 (Sec. 4.3 simulation input)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(nsamples)


def tone_params(lblock: int, ntones: int, seed: int, channel: float | None = None):
    """Tone frequencies (in units of PFB channels, i.e. cycles per lblock samples)
    and phases.  With `channel` given, one tone at that fractional channel; else
    `ntones` channels drawn U(1, lblock/2 - 1).  Returns (channels, phases)."""
    rng = np.random.default_rng(seed + 7919)
    if channel is not None:
        chans = np.array([float(channel)])
        phases = rng.uniform(0.0, 2.0 * math.pi, size=1)
    else:
        chans = rng.uniform(1.0, lblock / 2 - 1.0, size=ntones)
        phases = rng.uniform(0.0, 2.0 * math.pi, size=ntones)
    return chans, phases


def add_tones(x: np.ndarray, lblock: int, chans, phases, amplitude: float = 0.1,
              chunk: int = 1 << 22) -> np.ndarray:
    """x[t] += amplitude * sin(2*pi*(chan/lblock)*t + phase) for every tone (in place,
    chunked so that 2^28-sample streams stay within a few hundred MB of temporaries)."""
    T = x.shape[0]
    for t0 in range(0, T, chunk):
        t = np.arange(t0, min(T, t0 + chunk), dtype=np.float64)
        for c, ph in zip(chans, phases):
            # reduce the phase exactly: (c/lblock)*t mod 1 computed in two parts
            x[t0:t0 + t.shape[0]] += amplitude * np.sin(2.0 * math.pi * np.mod(c * t / lblock, 1.0) + ph)
    return x


def stream_config(lblock: int, nframes: int, seed: int, ntones: int = 0,
                  channel: float | None = None, amplitude: float = 0.1) -> np.ndarray:
    """Gaussian noise (sigma = 1) plus weak tones, nframes*lblock samples, float64."""
    x = gaussian_stream(lblock * nframes, seed)
    if channel is not None or ntones > 0:
        chans, phases = tone_params(lblock, ntones, seed, channel)
        add_tones(x, lblock, chans, phases, amplitude)
    return x


def random_taps_window(ntap: int, lblock: int, seed: int, dominant: float = 1.0,
                       spread: float = 0.3) -> np.ndarray:
    """A well-conditioned [ntap, lblock] window for exact-inverse tests: tap 0 of
    every column is `dominant`, the others U(0, spread), so that every column's
    circulant eigenvalues satisfy |W| >= dominant - (ntap-1)*spread > 0."""
    rng = np.random.default_rng(seed + 104729)
    w = rng.uniform(0.0, spread, size=(ntap, lblock))
    w[0, :] = dominant
    return w


def prior_chunks(nsamples: int, nchunks: int, fraction: float, seed: int):
    """Contiguous known-sample chunks: the stream is cut into `nchunks` equal
    segments and one chunk of round(fraction*nsamples/nchunks) samples is placed
    in each segment at a uniform random offset (so chunks never overlap).
    Returns (starts int64[nchunks], length)."""
    seg = nsamples // nchunks
    length = int(round(fraction * nsamples / nchunks))
    length = max(1, min(length, seg))
    rng = np.random.default_rng(seed + 15485863)
    offs = rng.integers(0, seg - length + 1, size=nchunks)
    starts = np.arange(nchunks, dtype=np.int64) * seg + offs
    return starts, length


def mask_from_chunks(nsamples: int, starts, length: int) -> np.ndarray:
    """Byte mask (1 = known sample) from chunk starts and a common length."""
    m = np.zeros(nsamples, dtype=np.uint8)
    for s in starts:
        m[int(s):int(s) + length] = 1
    return m


def batched_geometries(nstreams: int, seed: int, lblocks=(1024, 2048, 4096),
                       jmin: int = 1024, jmax: int = 16384):
    """Uneven stream shapes: lblock uniform over `lblocks`, nframes = round(exp(U(ln jmin,
    ln jmax))) (any integer).  Returns a list of (lblock, nframes)."""
    rng = np.random.default_rng(seed + 32452843)
    lb = rng.choice(np.asarray(lblocks), size=nstreams)
    nf = np.rint(np.exp(rng.uniform(math.log(jmin), math.log(jmax), size=nstreams))).astype(np.int64)
    return [(int(a), int(b)) for a, b in zip(lb, nf)]


def prior_fraction_draw(seed: int, lo: float = 0.02, hi: float = 0.20) -> float:
    """Prior fraction U[lo, hi] for one training instance."""
    return float(np.random.default_rng(seed + 49979687).uniform(lo, hi))
