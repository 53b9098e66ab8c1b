"""pfb_forward_noalloc: the forward PFB for callers that cannot pass a workspace
(for example streaming ingest code that reserves all device memory up front and may
not allocate per call).  Called through the raw C ABI, twice in a row, and checked
against pfb_forward (which takes a caller-provided workspace) with the tolerances
of the other forward-PFB tests: spectra and scales to 1e-5 relative, codes equal
except where the FP64 sums' rounding moves a value across a decision boundary.
The second call must first clear what the first left in the shared array."""
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
        assert np.max(np.abs(s / ref_scale - 1)) < 1e-5, call
        sp = spec.cpu().numpy()
        assert np.sqrt(np.mean(np.abs(sp - ref_spec) ** 2) / np.mean(np.abs(ref_spec) ** 2)) < 1e-5
        assert np.mean(codes.cpu().numpy() != ref_codes) < 2e-3, call


def test_noalloc_rejects_oversized_lblock():
    g = ipfb.geom(32768, 4, 16)
    fake = torch.empty(1, device="cuda")
    L = ipfb.lib()
    f = L.pfb_forward_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.POINTER(ipfb.Geom)] + [ctypes.c_void_p] * 6
    p = ctypes.c_void_p(fake.data_ptr())
    assert f(ctypes.byref(g), p, p, p, p, None, None) == ipfb.ERR_UNSUPPORTED
