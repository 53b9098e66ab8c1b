"""Guard zones around every caller-owned buffer (a substitute for a memory checker
on this pool): each workspace and output buffer sits between 64 KB guards filled with
a byte pattern; after every entry point has run, the guards must be untouched, so a
write past the end (or before the start) of any buffer fails the test.  Sizes are
small but span several tiles, both column-transform forms (one CTA and clusters,
through the on-chip column run), both ML forms (on chip and HBM-resident) and the
learned solve."""
import ctypes

import numpy as np
import pytest

from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402

G = 1 << 16
PAT = 0xA5


class Guarded:
    """A device buffer of nbytes between two guard zones."""

    def __init__(self, nbytes, dtype=torch.uint8, fill=None):
        self.nbytes = int(nbytes)
        self.buf = torch.full((self.nbytes + 2 * G,), PAT, dtype=torch.uint8, device="cuda")
        inner = self.buf[G:G + self.nbytes]
        self.t = inner.view(dtype) if self.nbytes else inner
        if fill is not None:
            self.t.copy_(fill.reshape(-1).view(dtype) if fill.dtype != dtype else fill.reshape(-1))

    def ptr(self):
        return ctypes.c_void_p(self.buf.data_ptr() + G)

    def intact(self):
        head, tail = self.buf[:G], self.buf[G + self.nbytes:]
        return bool((head == PAT).all()) and bool((tail == PAT).all())


def guarded_like(t):
    return Guarded(t.numel() * t.element_size(), t.dtype, fill=t)


def _inputs(N, J, seed):
    x = synth.stream_config(N, J, seed).astype(np.float32)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    xt = torch.from_numpy(x).cuda()
    wt = torch.from_numpy(w).cuda()
    codes, scale, _ = ipfb.pfb_forward(xt, wt)
    return xt, wt, codes, scale


def _check_all(bufs):
    torch.cuda.synchronize()
    bad = [name for name, b in bufs.items() if not b.intact()]
    assert not bad, bad


@pytest.mark.parametrize("run", [8192, 512])
def test_guards_forward_inverse_upchannelize(run):
    N, J = 256, 1024
    ipfb.set_max_column_run(run)
    try:
        xt, wt, codes, scale = _inputs(N, J, 61)
        L = ipfb.lib()
        g = ipfb.geom(N, 4, J)
        # forward
        b = {"codes": Guarded(J * N // 2), "scale": Guarded((N // 2 + 1) * 4, torch.float32),
             "spec": Guarded(J * (N // 2 + 1) * 8, torch.complex64),
             "ws": Guarded(ipfb.workspace_size(g, ipfb.OP_FORWARD))}
        assert L.pfb_forward(ctypes.byref(g), ipfb._ptr(xt), ipfb._ptr(wt), None, b["codes"].ptr(), b["scale"].ptr(),
                             b["spec"].ptr(), b["ws"].ptr(), b["ws"].nbytes, ipfb._stream()) == 0
        _check_all(b)
        assert torch.equal(b["codes"].t.view(J, N // 2), codes)
        # Wiener inverse, thresholded pseudo-inverse
        for name in ("wiener", "filter"):
            b = {"x": Guarded(J * N * 4, torch.float32), "ws": Guarded(ipfb.workspace_size(g, ipfb.OP_WIENER))}
            if name == "wiener":
                rc = L.ipfb_wiener(ctypes.byref(g), ipfb._ptr(codes), ipfb._ptr(scale), ipfb._ptr(wt), 0.0141, 1,
                                   b["x"].ptr(), b["ws"].ptr(), b["ws"].nbytes, ipfb._stream())
            else:
                rc = L.ipfb_filter(ctypes.byref(g), ipfb._ptr(codes), ipfb._ptr(scale), ipfb._ptr(wt),
                                   ipfb.FILTER_THRESHOLD, 0.05, None, b["x"].ptr(), b["ws"].ptr(), b["ws"].nbytes,
                                   ipfb._stream())
            assert rc == 0
            _check_all(b)
        # fused inverse + up-channelization (x_out too)
        U = 64
        b = {"out": Guarded((J // U) * (U * N // 2 + 1) * 8, torch.complex64), "x": Guarded(J * N * 4, torch.float32),
             "ws": Guarded(ipfb.workspace_size(g, ipfb.OP_WIENER_UPCHAN))}
        assert L.ipfb_wiener_upchannelize(ctypes.byref(g), ipfb._ptr(codes), ipfb._ptr(scale), ipfb._ptr(wt), 0.0141,
                                          1, U, b["out"].ptr(), b["x"].ptr(), b["ws"].ptr(), b["ws"].nbytes,
                                          ipfb._stream()) == 0
        _check_all(b)
        # streaming inverse and windowed re-channelization through the wrappers
        chunk, margin = 512, 64
        gs = ipfb.geom(N, 4, chunk)
        out = Guarded((J - 2 * margin) * N * 4, torch.float32)
        ws = Guarded(ipfb.workspace_size(gs, ipfb.OP_WIENER_STREAM))
        ipfb.ipfb_wiener_stream(codes, scale, wt, 0.0141, chunk, margin, out=out.t, workspace=ws.t)
        _check_all({"out": out, "ws": ws})
        wup = torch.from_numpy(ipfb.sinc_hamming_window(16 * N, 4)).cuda()
        nb = J // 16
        out = Guarded(nb * (16 * N // 2 + 1) * 8, torch.complex64)
        ws = Guarded(max(1, nb * 16 * N * 4))
        ipfb.upchannelize_pfb(xt, wup, out=out.t.view(nb, 16 * N // 2 + 1), workspace=ws.t)
        _check_all({"out": out, "ws": ws})
    finally:
        ipfb.set_max_column_run(8192)


def _ml_call(g, codes, scale, wt, prm, mask, prior, net, x0, ws_op):
    N, J = g.lblock, g.nframes
    b = {"x": guarded_like(x0), "iters": Guarded(N * 4, torch.int32), "resid": Guarded(2 * N * 4, torch.float32),
         "ws": Guarded(ipfb.workspace_size(g, ws_op))}
    rc = ipfb.lib().ipfb_ml_solve(ctypes.byref(g), ipfb._ptr(codes), ipfb._ptr(scale), ipfb._ptr(wt),
                                  ctypes.byref(prm), ipfb._ptr(mask), ipfb._ptr(prior), ipfb._ptr(net), b["x"].ptr(),
                                  1, b["iters"].ptr(), b["resid"].ptr(), b["ws"].ptr(), b["ws"].nbytes,
                                  ipfb._stream())
    assert rc == 0, ipfb.strerror(rc)
    _check_all(b)
    return b


@pytest.mark.parametrize("run,J", [(8192, 1024), (512, 1024), (512, 4096)])
@pytest.mark.parametrize("precond", [0, 1])
def test_guards_ml(run, J, precond):
    # (8192, 1024): the on-chip solve; (512, *): the HBM-resident one, 2- and 8-CTA clusters
    N = 128
    ipfb.set_max_column_run(run)
    try:
        xt, wt, codes, scale = _inputs(N, J, 62)
        starts, Lc = synth.prior_chunks(N * J, 8, 0.1, 62)
        mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, Lc)).cuda()
        g = ipfb.geom(N, 4, J)
        prm = ipfb.MLParams(2e-4, 1.0, 1e-6, 300, precond, 0)
        b = _ml_call(g, codes, scale, wt, prm, mask, xt, None, xt * 0.9, ipfb.OP_ML)
        assert int(b["iters"].t.max()) >= 1
    finally:
        ipfb.set_max_column_run(8192)


def test_guards_ml_learned_and_stream():
    N, J = 128, 1024
    xt, wt, codes, scale = _inputs(N, J, 63)
    starts, Lc = synth.prior_chunks(N * J, 8, 0.1, 63)
    mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, Lc)).cuda()
    from paper_2608_23441_b300 import precond_train as pt
    net = torch.from_numpy(pt.init_theta(1)).cuda()
    g = ipfb.geom(N, 4, J)
    prm = ipfb.MLParams(2e-4, 1.0, 1e-6, 60, 2, 1)
    _ml_call(g, codes, scale, wt, prm, mask, xt, net, xt * 0.9, ipfb.OP_ML_LEARNED)
    # overlap-save ML through the wrapper
    chunk, margin = 512, 64
    out = Guarded((J - 2 * margin) * N * 4, torch.float32)
    ws = Guarded(ipfb.workspace_size(ipfb.geom(N, 4, chunk), ipfb.OP_ML_STREAM))
    ipfb.ml_solve_stream(codes, scale, wt, 2e-4, mask, xt, chunk, margin, precond="wiener", tol=1e-6, max_iter=100,
                         out=out.t, workspace=ws.t)
    _check_all({"out": out, "ws": ws})


def test_guards_net_kernels():
    from paper_2608_23441_b300 import precond_train as pt
    theta = torch.from_numpy(pt.init_theta(2)).cuda()
    ns, J = 6, 1000
    xin = torch.randn((ns, 2, J), device="cuda")
    tgt = torch.randn((ns, J), device="cuda")
    for op in (ipfb.NET_FORWARD, ipfb.NET_GRAD):
        ws = Guarded(ipfb.net_workspace_size(op, ns, J))
        if op == ipfb.NET_FORWARD:
            ipfb.net_forward(theta, xin, workspace=ws.t)
        else:
            ipfb.net_grad(theta, xin, tgt, workspace=ws.t)
        _check_all({"ws": ws})
