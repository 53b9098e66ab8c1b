"""pfb_forward_noalloc: the forward PFB for callers that cannot pass a workspace
(for example streaming ingest code that reserves all device memory up front and may
not allocate per call).  Called through the raw C ABI, twice in a row, and checked
against pfb_forward (which takes a caller-provided workspace): both run the same
kernels, so the FP32 spectra must agree bit for bit, the steps (FP64 sums formed
with atomics in a different order) to one float32 ulp, and every code must be the
bit-exact float32 decision clamp(rint(v / Delta), -7, 7) on the call's own
spectrum and step, with codes equal to pfb_forward's wherever the two steps are
equal.  The second call must first clear what the first left in the shared array."""
import ctypes

import numpy as np
import pytest

from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402


def _noalloc(g, x, w, codes, scale, spec):
    L = ipfb.lib()
    f = L.pfb_forward_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ipfb.Geom)] + [ctypes.c_void_p] * 6
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(ctypes.byref(g), ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(w.data_ptr()),
             ctypes.c_void_p(codes.data_ptr()), ctypes.c_void_p(scale.data_ptr()),
             ctypes.c_void_p(spec.data_ptr()), stream)


def test_noalloc_matches_workspace_entry_twice():
    N, p, J = 1024, 4, 256
    x = synth.stream_config(N, J, 21, ntones=3).astype(np.float32)
    w = opfb.sinc_hamming_window(N, p).astype(np.float32)
    xg = torch.from_numpy(x).cuda()
    wg = torch.from_numpy(w).cuda()
    ref_codes, ref_scale, ref_spec = ipfb.pfb_forward(xg, wg, return_spectra=True)
    ref_codes, ref_scale, ref_spec = ref_codes.cpu().numpy(), ref_scale.cpu().numpy(), ref_spec.cpu().numpy()
    g = ipfb.geom(N, p, J)
    for call in range(2):
        codes = torch.empty((J, N // 2), dtype=torch.uint8, device="cuda")
        scale = torch.empty(N // 2 + 1, dtype=torch.float32, device="cuda")
        spec = torch.empty((J, N // 2 + 1), dtype=torch.complex64, device="cuda")
        rc = _noalloc(g, xg, wg, codes, scale, spec)
        assert rc == 0, (call, rc, ipfb.strerror(rc))
        torch.cuda.synchronize()
        s = scale.cpu().numpy()
        assert np.all(np.abs(s.view(np.int32) - ref_scale.view(np.int32)) <= 1), call
        sp = spec.cpu().numpy()
        assert np.array_equal(sp.view(np.float32), ref_spec.view(np.float32)), call
        got = codes.cpu().numpy()
        want = opfb.pack_codes(*opfb.quantize_spectra(sp.astype(np.complex128), s))
        assert np.array_equal(got, want), call
        same = s == ref_scale                      # channels whose steps agree exactly
        colmask = same[: N // 2] & np.r_[same[0] and same[N // 2], np.ones(N // 2 - 1, bool)]
        assert np.array_equal(got[:, colmask], ref_codes[:, colmask]), call


def test_noalloc_rejects_oversized_lblock():
    g = ipfb.geom(32768, 4, 16)
    fake = torch.empty(1, device="cuda")
    L = ipfb.lib()
    f = L.pfb_forward_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ipfb.Geom)] + [ctypes.c_void_p] * 6
    p = ctypes.c_void_p(fake.data_ptr())
    assert f(ctypes.byref(g), p, p, p, p, None, None) == ipfb.ERR_UNSUPPORTED
