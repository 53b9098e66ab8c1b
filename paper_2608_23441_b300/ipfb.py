"""Thin Python binding of libipfb (include/ipfb.h): argument marshalling only.

Every compute step runs in the library's CUDA kernels; this module checks
dtypes, shapes and devices of torch tensors, allocates outputs and workspaces
with torch (device memory only) and passes raw pointers plus the current torch
CUDA stream.  There is no CPU fallback: without the built library, or with
tensors that are not on a CUDA device, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libipfb.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "ipfb.h")

OK = 0
ERR_INVALID, ERR_UNSUPPORTED, ERR_WORKSPACE, ERR_NOT_CONVERGED, ERR_TIMEOUT, ERR_CUDA = -1, -2, -3, -4, -5, -6
OP_FORWARD, OP_WIENER, OP_WIENER_UPCHAN, OP_ML, OP_ML_LEARNED, OP_ML_PAIRS = 1, 2, 3, 4, 5, 6
OP_WIENER_STREAM = 7
OP_ML_STREAM = 8
NET_FORWARD, NET_GRAD = 1, 2
NET_NPARAMS = 10145


class Geom(ctypes.Structure):
    _fields_ = [("lblock", ctypes.c_int), ("ntap", ctypes.c_int),
                ("nframes", ctypes.c_int), ("periodic", ctypes.c_int)]


class MLParams(ctypes.Structure):
    _fields_ = [("noise_var", ctypes.c_double), ("prior_weight", ctypes.c_double), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("precond", ctypes.c_int), ("net_from", ctypes.c_int)]


PRECOND = {"none": 0, "wiener": 1, "learned": 2}
FILTER_THRESHOLD, FILTER_GAINS = 1, 2


class StreamDesc(ctypes.Structure):
    _fields_ = [("lblock", ctypes.c_int), ("ntap", ctypes.c_int), ("nframes", ctypes.c_int),
                ("codes", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("window", ctypes.c_void_p),
                ("noise_level", ctypes.c_double), ("x_out", ctypes.c_void_p)]


class IpfbError(RuntimeError):
    def __init__(self, fn: str, rc: int):
        self.rc = rc
        msg = f"{fn}: {strerror(rc)} ({rc})"
        if rc == ERR_CUDA:
            msg += f": {last_cuda_error()}"
        super().__init__(msg)


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t
_I64 = ctypes.c_int64

_SIGS = {
    "ipfb_strerror": (ctypes.c_char_p, [_I]),
    "ipfb_last_cuda_error": (ctypes.c_char_p, []),
    "ipfb_version": (_I, []),
    "ipfb_set_max_column_run": (_I, [_I]),
    "ipfb_set_net_wait_limit": (_I, [ctypes.c_longlong]),
    "ipfb_stage_timing": (_I, [_I]),
    "ipfb_stage_times": (_I, [ctypes.c_char_p, _SZ, ctypes.POINTER(_D), ctypes.POINTER(_I), _I]),
    "ipfb_workspace_size": (_I, [ctypes.POINTER(Geom), _I, ctypes.POINTER(_SZ)]),
    "ipfb_sinc_hamming_window": (_I, [_I, _I, _P]),
    "pfb_forward": (_I, [ctypes.POINTER(Geom), _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "pfb_quantize": (_I, [_I, _I, _P, _P, _P, _P]),
    "ipfb_wiener": (_I, [ctypes.POINTER(Geom), _P, _P, _P, _D, _I, _P, _P, _SZ, _P]),
    "ipfb_filter": (_I, [ctypes.POINTER(Geom), _P, _P, _P, _I, _D, _P, _P, _P, _SZ, _P]),
    "ipfb_wiener_stream": (_I, [ctypes.POINTER(Geom), _I64, _P, _P, _P, _D, _I, _I, _P, _P, _SZ, _P]),
    "ipfb_ml_solve_stream": (_I, [ctypes.POINTER(Geom), _I64, _P, _P, _P, ctypes.POINTER(MLParams), _P, _P, _P, _I,
                                  _P, _P, _P, _P, _SZ, _P]),
    "upchannelize": (_I, [_P, _I64, _I64, _P, _P, _SZ, _P]),
    "upchannelize_pfb": (_I, [_P, _I64, _I64, _I, _P, _P, _P, _SZ, _P]),
    "ipfb_wiener_upchannelize": (_I, [ctypes.POINTER(Geom), _P, _P, _P, _D, _I, _I, _P, _P, _P, _SZ, _P]),
    "ipfb_batched_plan": (_I, [ctypes.POINTER(StreamDesc), _I, _I, ctypes.c_char_p, ctypes.POINTER(_P),
                               ctypes.POINTER(_SZ)]),
    "ipfb_batched_prepare": (_I, [_P, _P, _SZ, _P]),
    "ipfb_batched_run": (_I, [_P, _P, _SZ, _P]),
    "ipfb_batched_autotune": (_I, [_P, _P, _SZ, _P, ctypes.c_char_p]),
    "ipfb_batched_variant": (_I, [_P, _I, ctypes.c_char_p, _SZ]),
    "ipfb_batched_free": (_I, [_P]),
    "ipfb_ml_solve": (_I, [ctypes.POINTER(Geom), _P, _P, _P, ctypes.POINTER(MLParams), _P, _P, _P, _P, _I, _P, _P,
                           _P, _SZ, _P]),
    "ipfb_net_nparams": (_I, []),
    "ipfb_net_workspace_size": (_I, [_I, _I, _I, ctypes.POINTER(_SZ)]),
    "ipfb_net_forward": (_I, [_P, _I, _I, _P, _P, _P, _SZ, _P]),
    "ipfb_net_grad": (_I, [_P, _I, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "ipfb_net_adam": (_I, [_P, _P, _P, _P, _I, _I, _D, _D, _D, _D, _P]),
    "ipfb_ml_training_pairs": (_I, [ctypes.POINTER(Geom), _P, ctypes.POINTER(MLParams), _P, _P, _P, _P, _I, _P, _P,
                                    _P, _SZ, _P]),
}


def lib():
    """Load libipfb.so from the package directory (built by `build.py`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2608_23441_b300.build`")
        handle = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            if hasattr(handle, name):
                f = getattr(handle, name)
                f.restype = res
                f.argtypes = args
        _lib = handle
    return _lib


def header_functions() -> list[str]:
    """Names of every function declared in include/ipfb.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([A-Za-z_][A-Za-z0-9_]*)\s*\(",
                      text, flags=re.M)


def strerror(rc: int) -> str:
    return lib().ipfb_strerror(rc).decode()


def last_cuda_error() -> str:
    return lib().ipfb_last_cuda_error().decode()


def _check(fn: str, rc: int):
    if rc != OK:
        raise IpfbError(fn, rc)


def set_max_column_run(frames: int):
    _check("ipfb_set_max_column_run", lib().ipfb_set_max_column_run(int(frames)))


def set_net_wait_limit(cycles: int):
    """Testing knob: bound (SM clocks) on the net forward's accumulator wait; < 0 restores
    the built-in bound of about a second."""
    _check("ipfb_set_net_wait_limit", lib().ipfb_set_net_wait_limit(int(cycles)))


def stage_timing(enable: bool):
    """Start (and clear) or stop per-kernel CUDA-event timing inside the library."""
    _check("ipfb_stage_timing", lib().ipfb_stage_timing(int(bool(enable))))


def stage_times() -> dict:
    """{kernel name: (total ms, launches)} recorded since stage_timing(True)."""
    cap = 4096
    names = ctypes.create_string_buffer(cap)
    ms = (_D * 64)()
    cnt = (_I * 64)()
    n = lib().ipfb_stage_times(names, cap, ms, cnt, 64)
    if n < 0:
        raise IpfbError("ipfb_stage_times", n)
    keys = names.value.decode().split(",") if n else []
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(keys)}


def geom(lblock: int, ntap: int, nframes: int, periodic: int = 1) -> Geom:
    return Geom(int(lblock), int(ntap), int(nframes), int(periodic))


def workspace_size(g: Geom, op: int) -> int:
    n = _SZ(0)
    _check("ipfb_workspace_size", lib().ipfb_workspace_size(ctypes.byref(g), op, ctypes.byref(n)))
    return int(n.value)


def sinc_hamming_window(lblock: int, ntap: int) -> np.ndarray:
    """Host-side window of the library, float32 [ntap, lblock]."""
    out = np.empty(int(lblock) * int(ntap), dtype=np.float32)
    _check("ipfb_sinc_hamming_window",
           lib().ipfb_sinc_hamming_window(int(lblock), int(ntap), out.ctypes.data_as(_P)))
    return out.reshape(int(ntap), int(lblock))


# --------------------------------------------------------------------------- torch side
def _torch():
    import torch
    return torch


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workspace(nbytes: int, device, ws=None):
    torch = _torch()
    if nbytes == 0:
        return None, 0
    if ws is not None:
        return ws, ws.numel() * ws.element_size()
    return torch.empty(nbytes, dtype=torch.uint8, device=device), nbytes


def pfb_forward(x, window, scale=None, return_spectra: bool = False, workspace=None):
    """Forward PFB + 4-bit quantization.  x float32 [J*N] (CUDA); window float32
    [ntap, N].  Returns (codes uint8 [J, N/2], scale float32 [N/2+1], spectra
    complex64 [J, N/2+1] or None)."""
    torch = _torch()
    window = _dev(window, torch.float32, "window")
    p, N = window.shape
    x = _dev(x, torch.float32, "x")
    J = x.numel() // N
    if J * N != x.numel():
        raise ValueError("len(x) must be a multiple of lblock")
    g = geom(N, p, J)
    codes = torch.empty((J, N // 2), dtype=torch.uint8, device=x.device)
    scale_out = torch.empty(N // 2 + 1, dtype=torch.float32, device=x.device)
    spec = torch.empty((J, N // 2 + 1), dtype=torch.complex64, device=x.device) if return_spectra else None
    if scale is not None:
        scale = _dev(scale, torch.float32, "scale")
    ws, wsb = _workspace(workspace_size(g, OP_FORWARD), x.device, workspace)
    _check("pfb_forward", lib().pfb_forward(ctypes.byref(g), _ptr(x), _ptr(window), _ptr(scale), _ptr(codes),
                                            _ptr(scale_out), _ptr(spec), _ptr(ws), wsb, _stream()))
    return codes, scale_out, spec


def pfb_quantize(spectra, scale):
    """Quantize complex64 spectra [nspec, N/2+1] with float32 scale [N/2+1]."""
    torch = _torch()
    spectra = _dev(spectra, torch.complex64, "spectra")
    scale = _dev(scale, torch.float32, "scale")
    nspec, C = spectra.shape
    N = 2 * (C - 1)
    codes = torch.empty((nspec, N // 2), dtype=torch.uint8, device=spectra.device)
    _check("pfb_quantize", lib().pfb_quantize(N, nspec, _ptr(spectra), _ptr(scale), _ptr(codes), _stream()))
    return codes


def ipfb_wiener(codes, scale, window, noise_level: float, normalize: bool = True, out=None, workspace=None):
    """Circulant (Wiener) inverse PFB.  codes uint8 [J, N/2]; scale float32 [N/2+1];
    window float32 [ntap, N].  Returns x float32 [J*N] (time order)."""
    torch = _torch()
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    p, N = window.shape
    J = codes.shape[0]
    g = geom(N, p, J)
    x = out if out is not None else torch.empty(J * N, dtype=torch.float32, device=codes.device)
    ws, wsb = _workspace(workspace_size(g, OP_WIENER), codes.device, workspace)
    _check("ipfb_wiener", lib().ipfb_wiener(ctypes.byref(g), _ptr(codes), _ptr(scale), _ptr(window),
                                            float(noise_level), int(bool(normalize)), _ptr(x), _ptr(ws), wsb,
                                            _stream()))
    return x


def ipfb_filter(codes, scale, window, threshold: float | None = None, gains=None, out=None, workspace=None):
    """Circulant inverse PFB with another eigenvalue filter (ipfb_filter): the
    thresholded pseudo-inverse (threshold >= 0) or caller gains (complex64 [N, J/2+1],
    G_n(k) for k <= J/2).  Exactly one of threshold / gains.  Returns x float32 [J*N]."""
    torch = _torch()
    if (threshold is None) == (gains is None):
        raise ValueError("give exactly one of threshold, gains")
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    p, N = window.shape
    J = codes.shape[0]
    g = geom(N, p, J)
    if gains is not None:
        gains = _dev(gains, torch.complex64, "gains")
        if tuple(gains.shape) != (N, J // 2 + 1):
            raise ValueError("gains must be [N, J/2 + 1]")
    x = out if out is not None else torch.empty(J * N, dtype=torch.float32, device=codes.device)
    ws, wsb = _workspace(workspace_size(g, OP_WIENER), codes.device, workspace)
    mode = FILTER_THRESHOLD if threshold is not None else FILTER_GAINS
    _check("ipfb_filter", lib().ipfb_filter(ctypes.byref(g), _ptr(codes), _ptr(scale), _ptr(window), mode,
                                            float(threshold or 0.0), _ptr(gains), _ptr(x), _ptr(ws), wsb,
                                            _stream()))
    return x


def upchannelize(x, block: int, out=None):
    """Block real DFT of a time-ordered float32 stream: complex64 [len(x)//L, L/2+1]."""
    torch = _torch()
    x = _dev(x, torch.float32, "x")
    L = int(block)
    nb = x.numel() // L
    if out is None:
        out = torch.empty((nb, L // 2 + 1), dtype=torch.complex64, device=x.device)
    _check("upchannelize", lib().upchannelize(_ptr(x), x.numel(), L, _ptr(out), None, 0, _stream()))
    return out


def ipfb_wiener_stream(codes, scale, window, noise_level: float, chunk: int, margin: int, normalize: bool = True,
                       out=None, workspace=None):
    """Overlap-save Wiener inverse of a long run of spectra (ipfb_wiener_stream):
    chunks of `chunk` spectra, `margin` frames dropped at each chunk edge.  codes uint8
    [nspec, N/2]; returns x float32 [(nspec - 2 margin) * N], frames margin ..
    nspec - margin - 1."""
    torch = _torch()
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    p, N = window.shape
    nspec = codes.shape[0]
    g = geom(N, p, int(chunk))
    x = out if out is not None else torch.empty((nspec - 2 * margin) * N, dtype=torch.float32, device=codes.device)
    ws, wsb = _workspace(workspace_size(g, OP_WIENER_STREAM), codes.device, workspace)
    _check("ipfb_wiener_stream", lib().ipfb_wiener_stream(ctypes.byref(g), int(nspec), _ptr(codes), _ptr(scale),
                                                          _ptr(window), float(noise_level), int(bool(normalize)),
                                                          int(margin), _ptr(x), _ptr(ws), wsb, _stream()))
    return x


def ml_solve_stream(codes, scale, window, noise_var: float, mask, prior, chunk: int, margin: int,
                    prior_weight: float = 1.0, precond: str = "none", tol: float = 1e-6, max_iter: int = 1000,
                    x0=None, out=None, workspace=None):
    """Overlap-save ML reconstruction of a long run (ipfb_ml_solve_stream): chunks of
    `chunk` spectra, `margin` frames dropped at each chunk edge.  codes uint8
    [nspec, N/2]; mask uint8 / prior, x0 float32 [nspec * N].  Returns (x float32
    [(nspec - 2 margin) * N] frames margin .. nspec - margin - 1, iters int32 [N],
    resid float32 [2, N], both the largest over the chunks)."""
    torch = _torch()
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    mask = _dev(mask, torch.uint8, "mask")
    prior = _dev(prior, torch.float32, "prior")
    x0 = None if x0 is None else _dev(x0, torch.float32, "x0")
    p, N = window.shape
    nspec = codes.shape[0]
    g = geom(N, p, int(chunk))
    x = out if out is not None else torch.empty((nspec - 2 * margin) * N, dtype=torch.float32, device=codes.device)
    iters = torch.empty(N, dtype=torch.int32, device=codes.device)
    resid = torch.empty((2, N), dtype=torch.float32, device=codes.device)
    prm = MLParams(float(noise_var), float(prior_weight), float(tol), int(max_iter), PRECOND[precond], 0)
    ws, wsb = _workspace(workspace_size(g, OP_ML_STREAM), codes.device, workspace)
    _check("ipfb_ml_solve_stream", lib().ipfb_ml_solve_stream(
        ctypes.byref(g), int(nspec), _ptr(codes), _ptr(scale), _ptr(window), ctypes.byref(prm), _ptr(mask),
        _ptr(prior), _ptr(x0), int(margin), _ptr(x), _ptr(iters), _ptr(resid), _ptr(ws), wsb, _stream()))
    return x, iters, resid


def upchannelize_pfb(x, window, out=None, workspace=None):
    """Windowed re-channelization (upchannelize_pfb): a PFB with frames L =
    window.shape[1] long and window.shape[0] taps over x float32 [T] (CUDA).
    Returns complex64 [T // L, L/2 + 1]."""
    torch = _torch()
    x = _dev(x, torch.float32, "x")
    window = _dev(window, torch.float32, "window")
    p, L = window.shape
    nb = x.numel() // L
    if out is None:
        out = torch.empty((nb, L // 2 + 1), dtype=torch.complex64, device=x.device)
    ws, wsb = _workspace(max(1, nb * L * 4), x.device, workspace)
    _check("upchannelize_pfb", lib().upchannelize_pfb(_ptr(x), x.numel(), L, p, _ptr(window), _ptr(out), _ptr(ws),
                                                      wsb, _stream()))
    return out


def ipfb_wiener_upchannelize(codes, scale, window, noise_level: float, upfactor: int, normalize: bool = True,
                             want_x: bool = False, out=None, x_out=None, workspace=None):
    """Wiener iPFB followed by up-channelization with L = upfactor * lblock.
    Returns (spectra complex64 [J/upfactor, L/2+1], x float32 [J*N] or None)."""
    torch = _torch()
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    p, N = window.shape
    J = codes.shape[0]
    g = geom(N, p, J)
    L = int(upfactor) * N
    if out is None:
        out = torch.empty((J // int(upfactor), L // 2 + 1), dtype=torch.complex64, device=codes.device)
    if want_x and x_out is None:
        x_out = torch.empty(J * N, dtype=torch.float32, device=codes.device)
    ws, wsb = _workspace(workspace_size(g, OP_WIENER_UPCHAN), codes.device, workspace)
    _check("ipfb_wiener_upchannelize",
           lib().ipfb_wiener_upchannelize(ctypes.byref(g), _ptr(codes), _ptr(scale), _ptr(window),
                                          float(noise_level), int(bool(normalize)), int(upfactor), _ptr(out),
                                          _ptr(x_out), _ptr(ws), wsb, _stream()))
    return out, x_out


def ml_solve(codes, scale, window, noise_var: float, mask, prior, prior_weight: float = 1.0,
             precond: str = "none", tol: float = 1e-6, max_iter: int = 1000, x0=None, net=None,
             workspace=None, net_from: int = 0):
    """ML inverse PFB with a time-domain prior by conjugate gradient.
    codes uint8 [J, N/2]; scale float32 [N/2+1]; window float32 [ntap, N];
    mask uint8 [J*N] (nonzero = saved); prior float32 [J*N]; x0 float32 [J*N] or None.
    Returns (x float32 [J*N], iters int32 [N], resid float32 [2, N])."""
    torch = _torch()
    codes = _dev(codes, torch.uint8, "codes")
    scale = _dev(scale, torch.float32, "scale")
    window = _dev(window, torch.float32, "window")
    mask = _dev(mask, torch.uint8, "mask")
    prior = _dev(prior, torch.float32, "prior")
    p, N = window.shape
    J = codes.shape[0]
    g = geom(N, p, J)
    if x0 is not None:
        x = _dev(x0, torch.float32, "x0").clone()
    else:
        x = torch.empty(J * N, dtype=torch.float32, device=codes.device)
    iters = torch.empty(N, dtype=torch.int32, device=codes.device)
    resid = torch.empty((2, N), dtype=torch.float32, device=codes.device)
    prm = MLParams(float(noise_var), float(prior_weight), float(tol), int(max_iter), PRECOND[precond], int(net_from))
    if precond == "learned":
        if net is None:
            raise ValueError("precond='learned' needs net (float32 CUDA tensor of NET_NPARAMS parameters)")
        net = _dev(net, torch.float32, "net")
        if net.numel() != NET_NPARAMS:
            raise ValueError(f"net has {net.numel()} parameters, expected {NET_NPARAMS}")
    ws, wsb = _workspace(workspace_size(g, OP_ML_LEARNED if precond == "learned" else OP_ML), codes.device,
                         workspace)
    _check("ipfb_ml_solve", lib().ipfb_ml_solve(ctypes.byref(g), _ptr(codes), _ptr(scale), _ptr(window),
                                                ctypes.byref(prm), _ptr(mask), _ptr(prior), _ptr(net), _ptr(x),
                                                int(x0 is not None), _ptr(iters), _ptr(resid), _ptr(ws), wsb,
                                                _stream()))
    return x, iters, resid


def net_workspace_size(op: int, nslots: int, nframes: int) -> int:
    n = _SZ(0)
    _check("ipfb_net_workspace_size", lib().ipfb_net_workspace_size(int(op), int(nslots), int(nframes),
                                                                    ctypes.byref(n)))
    return n.value


def _net_args(theta, xin):
    torch = _torch()
    theta = _dev(theta, torch.float32, "theta")
    if theta.numel() != NET_NPARAMS:
        raise ValueError(f"theta has {theta.numel()} values, expected {NET_NPARAMS}")
    xin = _dev(xin, torch.float32, "xin")
    if xin.dim() != 3 or xin.shape[1] != 2:
        raise ValueError("xin must be [nslots, 2, J]")
    return theta, xin


def net_forward(theta, xin, workspace=None):
    """Net output y [nslots, J] for inputs xin [nslots, 2, J] (ipfb_net_forward)."""
    torch = _torch()
    theta, xin = _net_args(theta, xin)
    ns, _, J = xin.shape
    y = torch.empty((ns, J), dtype=torch.float32, device=xin.device)
    ws, wsb = _workspace(net_workspace_size(NET_FORWARD, ns, J), xin.device, workspace)
    _check("ipfb_net_forward", lib().ipfb_net_forward(_ptr(theta), ns, J, _ptr(xin), _ptr(y), _ptr(ws), wsb,
                                                      _stream()))
    return y


def net_grad(theta, xin, target, workspace=None):
    """(loss [1], grad [NET_NPARAMS]) of the mean squared error of net(xin) against
    target [nslots, J] (ipfb_net_grad)."""
    torch = _torch()
    theta, xin = _net_args(theta, xin)
    target = _dev(target, torch.float32, "target")
    ns, _, J = xin.shape
    if tuple(target.shape) != (ns, J):
        raise ValueError("target must be [nslots, J]")
    loss = torch.empty(1, dtype=torch.float32, device=xin.device)
    grad = torch.empty(NET_NPARAMS, dtype=torch.float32, device=xin.device)
    ws, wsb = _workspace(net_workspace_size(NET_GRAD, ns, J), xin.device, workspace)
    _check("ipfb_net_grad", lib().ipfb_net_grad(_ptr(theta), ns, J, _ptr(xin), _ptr(target), _ptr(loss),
                                                _ptr(grad), _ptr(ws), wsb, _stream()))
    return loss, grad


def net_adam(theta, m, v, grad, step: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
             eps: float = 1e-8):
    """One Adam step in place on theta, m, v (ipfb_net_adam)."""
    torch = _torch()
    theta = _dev(theta, torch.float32, "theta")
    m = _dev(m, torch.float32, "m")
    v = _dev(v, torch.float32, "v")
    grad = _dev(grad, torch.float32, "grad")
    n = theta.numel()
    if not (m.numel() == v.numel() == grad.numel() == n):
        raise ValueError("theta, m, v, grad must have the same size")
    _check("ipfb_net_adam", lib().ipfb_net_adam(_ptr(theta), _ptr(m), _ptr(v), _ptr(grad), n, int(step),
                                                float(lr), float(beta1), float(beta2), float(eps), _stream()))


def ml_training_pairs(window, noise_var: float, mask, x_star, x_k, pair_index, prior_weight: float = 1.0,
                      workspace=None):
    """Net training examples (xin [2 npairs, 2, J], target [2 npairs, J]) from two
    iterates x_star, x_k [J*N] of the ML solve (ipfb_ml_training_pairs); pair_index
    is a host sequence of column-pair indices."""
    torch = _torch()
    window = _dev(window, torch.float32, "window")
    mask = _dev(mask, torch.uint8, "mask")
    x_star = _dev(x_star, torch.float32, "x_star")
    x_k = _dev(x_k, torch.float32, "x_k")
    pair_index = np.ascontiguousarray(np.asarray(pair_index, dtype=np.int32))
    p, N = window.shape
    J = x_star.numel() // N
    g = geom(N, p, J)
    npairs = pair_index.size
    xin = torch.empty((2 * npairs, 2, J), dtype=torch.float32, device=window.device)
    target = torch.empty((2 * npairs, J), dtype=torch.float32, device=window.device)
    prm = MLParams(float(noise_var), float(prior_weight), 0.0, 0, 0)
    ws, wsb = _workspace(workspace_size(g, OP_ML_PAIRS), window.device, workspace)
    _check("ipfb_ml_training_pairs", lib().ipfb_ml_training_pairs(
        ctypes.byref(g), _ptr(window), ctypes.byref(prm), _ptr(mask), _ptr(x_star), _ptr(x_k),
        pair_index.ctypes.data_as(ctypes.c_void_p),
        npairs, _ptr(xin), _ptr(target), _ptr(ws), wsb, _stream()))
    return xin, target


class BatchedPlan:
    """Many independent streams inverted together (ipfb_batched_*).  Each stream is
    a dict with CUDA tensors codes uint8 [J, N/2], scale float32 [N/2+1], window
    float32 [4, N] and a float noise_level; outputs are allocated here (x[i],
    float32 [J*N]).  run() is capturable in a CUDA graph after prepare()."""

    def __init__(self, streams, normalize: bool = True, tune_cache: str | None = None):
        torch = _torch()
        self._keep = []
        self.x = []
        descs = (StreamDesc * len(streams))()
        for i, st in enumerate(streams):
            codes = _dev(st["codes"], torch.uint8, "codes")
            scale = _dev(st["scale"], torch.float32, "scale")
            window = _dev(st["window"], torch.float32, "window")
            p, N = window.shape
            J = codes.shape[0]
            x = torch.empty(J * N, dtype=torch.float32, device=codes.device)
            self.x.append(x)
            self._keep += [codes, scale, window]
            descs[i] = StreamDesc(N, p, J, codes.data_ptr(), scale.data_ptr(), window.data_ptr(),
                                  float(st["noise_level"]), x.data_ptr())
        self._descs = descs
        plan = _P()
        nbytes = _SZ(0)
        cache = tune_cache.encode() if tune_cache else None
        _check("ipfb_batched_plan", lib().ipfb_batched_plan(descs, len(streams), int(bool(normalize)), cache,
                                                            ctypes.byref(plan), ctypes.byref(nbytes)))
        self.plan = plan
        self.ws = torch.empty(max(1, nbytes.value), dtype=torch.uint8, device=streams[0]["codes"].device)
        self.ws_bytes = nbytes.value

    def prepare(self):
        _check("ipfb_batched_prepare", lib().ipfb_batched_prepare(self.plan, _ptr(self.ws), self.ws_bytes,
                                                                  _stream()))

    def run(self):
        _check("ipfb_batched_run", lib().ipfb_batched_run(self.plan, _ptr(self.ws), self.ws_bytes, _stream()))
        return self.x

    def autotune(self, cache_path: str | None = None):
        c = cache_path.encode() if cache_path else None
        _check("ipfb_batched_autotune", lib().ipfb_batched_autotune(self.plan, _ptr(self.ws), self.ws_bytes,
                                                                    _stream(), c))

    def variant(self, M: int) -> str:
        buf = ctypes.create_string_buffer(64)
        _check("ipfb_batched_variant", lib().ipfb_batched_variant(self.plan, int(M), buf, 64))
        return buf.value.decode()

    def close(self):
        if getattr(self, "plan", None):
            lib().ipfb_batched_free(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
