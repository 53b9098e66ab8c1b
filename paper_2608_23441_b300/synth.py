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
              block: int = 4096) -> np.ndarray:
    """x[t] += amplitude * sum over tones of sin(2 pi (chan/lblock) t + phase), in place.
    Evaluated block-wise as sin(a_k + b_u) = sin a_k cos b_u + cos a_k sin b_u with
    t = k*block + u: one [blocks, 2*ntones] x [2*ntones, block] matrix product adds
    every tone to a 2^28-sample stream in about a second."""
    T = x.shape[0]
    nfull = T // block
    u = np.arange(block, dtype=np.float64)
    k = np.arange(nfull, dtype=np.float64)
    A = np.empty((nfull, 2 * len(chans)))
    B = np.empty((2 * len(chans), block))
    for i, (c, ph) in enumerate(zip(chans, phases)):
        f = float(c) / float(lblock)
        bu = 2.0 * math.pi * np.mod(f * u, 1.0)
        ak = 2.0 * math.pi * np.mod(f * block * k, 1.0) + ph
        A[:, 2 * i], A[:, 2 * i + 1] = np.sin(ak), np.cos(ak)
        B[2 * i], B[2 * i + 1] = np.cos(bu), np.sin(bu)
        if T > nfull * block:
            t = np.arange(nfull * block, T, dtype=np.float64)
            x[nfull * block:] += amplitude * np.sin(2.0 * math.pi * np.mod(f * t, 1.0) + ph)
    if nfull:
        step = 8192
        xv = x[: nfull * block].reshape(nfull, block)
        for r0 in range(0, nfull, step):
            xv[r0:r0 + step] += amplitude * (A[r0:r0 + step] @ B)
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


def saved_paths(lblock: int, fraction: float, every: int = 4) -> int:
    """Number L of sub-filter paths to save every `every`-th sample of for a saved
    fraction beta = L / (every * lblock) of the stream (Sec. 4.3), rounded to an even
    count so that the paths sit symmetrically around lblock / 2."""
    L = int(round(fraction * every * lblock / 2.0)) * 2
    return max(2, min(L, lblock))


def path_sample_mask(lblock: int, nframes: int, npaths: int, every: int = 4, phase: int = 0) -> np.ndarray:
    """Byte mask (1 = saved sample) in time order [nframes * lblock]: every `every`-th
    frame (frames j with j % every == phase) of the `npaths` sub-filter paths
    n in [lblock/2 - npaths/2, lblock/2 + npaths/2), the saving scheme of Sec. 4.3."""
    m = np.zeros((nframes, lblock), dtype=np.uint8)
    n0 = lblock // 2 - npaths // 2
    m[phase::every, n0:n0 + npaths] = 1
    return m.reshape(-1)


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


def random_code_bytes(nspec: int, half: int, seed: int) -> np.ndarray:
    """Random 4-bit code bytes [nspec, half]: both nibbles uniform over the 15
    two's-complement levels -7..7 (nibble value 8, i.e. -8, never appears)."""
    rng = np.random.default_rng(seed + 86028121)
    lv = np.array([0, 1, 2, 3, 4, 5, 6, 7, 9, 10, 11, 12, 13, 14, 15], dtype=np.uint8)
    lo = lv[rng.integers(0, 15, size=(nspec, half))]
    hi = lv[rng.integers(0, 15, size=(nspec, half))]
    return (lo | (hi << 4)).astype(np.uint8)


def random_scale(nchan: int, seed: int) -> np.ndarray:
    """Positive per-channel quantizer steps, float32, log-uniform over [0.5, 2]."""
    rng = np.random.default_rng(seed + 122949823)
    return np.exp(rng.uniform(np.log(0.5), np.log(2.0), size=nchan)).astype(np.float32)


def gaussian_stream_torch(nsamples: int, seed: int, device):
    """White standard-normal stream generated on a torch device (float32) with a
    seeded torch.Generator; for large benchmark batches, where host generation would
    dominate.  Not bit-identical to gaussian_stream."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return torch.randn(int(nsamples), generator=g, device=device, dtype=torch.float32)
