"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/ipfb.h declares, and rejects bad arguments on the host (no GPU needed:
every call here fails validation before anything is enqueued)."""
import ctypes

import numpy as np
import pytest

from oracle import pfb as opfb
from paper_2608_23441_b300 import ipfb


def test_library_exports_every_header_symbol():
    names = ipfb.header_functions()
    assert len(names) >= 10
    handle = ipfb.lib()
    missing = [n for n in names if not hasattr(handle, n)]
    assert not missing, missing
    assert ipfb.lib().ipfb_version() >= 100


def test_strerror_codes():
    for rc in (0, -1, -2, -3, -4, -5, -6):
        assert ipfb.strerror(rc)
    assert ipfb.strerror(12345) == "unknown status"


def test_workspace_sizes():
    g = ipfb.geom(4096, 4, 65536)
    assert ipfb.workspace_size(g, ipfb.OP_WIENER) == 65536 * 4096 * 4
    assert ipfb.workspace_size(g, ipfb.OP_WIENER_UPCHAN) == 2 * 65536 * 4096 * 4
    assert ipfb.workspace_size(g, ipfb.OP_FORWARD) == 2 * 2049 * 8
    assert ipfb.workspace_size(ipfb.geom(2048, 4, 8192), ipfb.OP_WIENER_STREAM) == 2 * 8192 * 2048 * 4
    with pytest.raises(ipfb.IpfbError) as e:
        ipfb.workspace_size(ipfb.geom(4096, 4, 65537), ipfb.OP_WIENER)
    assert e.value.rc == ipfb.ERR_UNSUPPORTED
    with pytest.raises(ipfb.IpfbError) as e:
        ipfb.workspace_size(ipfb.geom(4096, 4, 1024), 99)
    assert e.value.rc == ipfb.ERR_INVALID
    with pytest.raises(ipfb.IpfbError) as e:
        ipfb.workspace_size(ipfb.geom(4096, 4, 1024, periodic=0), ipfb.OP_WIENER)
    assert e.value.rc == ipfb.ERR_UNSUPPORTED


def test_learned_workspace_sizes():
    g = ipfb.geom(4096, 4, 8192)
    ml = ipfb.workspace_size(g, ipfb.OP_ML)
    learned = ipfb.workspace_size(g, ipfb.OP_ML_LEARNED)
    vec = 4096 * 8192 * 4
    # d, five FCG vectors, net outputs (one vector) and inputs (two), the prior-mask
    # bits of every thread (one 32-bit word per 16 frames of a column pair), small state
    mbits = 2048 * (8192 // 16) * 4
    assert 9 * vec + mbits <= learned <= 9 * vec + mbits + (1 << 20)
    assert ml == 2 * vec
    assert ipfb.workspace_size(g, ipfb.OP_ML_PAIRS) == 2 * vec + 2048 * 4
    with pytest.raises(ipfb.IpfbError):
        ipfb.workspace_size(ipfb.geom(4096, 8, 8192), ipfb.OP_ML_LEARNED)
    fwd = ipfb.net_workspace_size(ipfb.NET_FORWARD, 16, 8192)
    grad = ipfb.net_workspace_size(ipfb.NET_GRAD, 16, 8192)
    assert fwd >= 2 * 22592
    # one partial gradient (+ loss) per 224-frame tile of every slot
    assert grad - fwd == 16 * ((8192 + 223) // 224) * (ipfb.NET_NPARAMS + 1) * 4


def test_ml_workspace_beyond_the_on_chip_run():
    g = ipfb.geom(2048, 4, 65536)
    ml = ipfb.workspace_size(g, ipfb.OP_ML)
    vec = 1024 * 65536 * 8  # one pair-packed vector
    # seven vectors, the mask bits, per-tile partial sums and small state
    assert 7 * vec + 1024 * 65536 <= ml <= 7 * vec + 1024 * 65536 + (8 << 20)
    assert ipfb.workspace_size(g, ipfb.OP_ML_STREAM) >= ml + 2048 * 65536 * 4
    with pytest.raises(ipfb.IpfbError):
        ipfb.workspace_size(g, ipfb.OP_ML_LEARNED)
    # the on-chip column run decides the form
    g2 = ipfb.geom(64, 4, 2048)
    assert ipfb.workspace_size(g2, ipfb.OP_ML) == 2 * 64 * 2048 * 4
    assert ipfb.lib().ipfb_set_max_column_run(512) == 0
    try:
        assert ipfb.workspace_size(g2, ipfb.OP_ML) >= 7 * 32 * 2048 * 8
        # 8192 frames would split into 8 runs of 1024: no cluster transform of that length
        with pytest.raises(ipfb.IpfbError) as e:
            ipfb.workspace_size(ipfb.geom(64, 4, 8192), ipfb.OP_ML)
        assert e.value.rc == ipfb.ERR_UNSUPPORTED
    finally:
        ipfb.lib().ipfb_set_max_column_run(8192)


def test_library_window_matches_oracle_window():
    for N, p in ((64, 4), (256, 4), (4096, 4), (128, 3)):
        w = ipfb.sinc_hamming_window(N, p)
        ref = opfb.sinc_hamming_window(N, p)
        assert w.dtype == np.float32 and w.shape == (p, N)
        assert np.array_equal(w, ref.astype(np.float32))


def test_host_validation_rejects_before_launch():
    L = ipfb.lib()
    g = ipfb.geom(256, 4, 64)
    G = ctypes.byref(g)
    # null pointers
    assert L.ipfb_wiener(G, None, None, None, 0.01, 1, None, None, 0, None) == ipfb.ERR_INVALID
    assert L.pfb_forward(G, None, None, None, None, None, None, None, 0, None) == ipfb.ERR_INVALID
    assert L.upchannelize(None, 0, 1024, None, None, 0, None) == ipfb.ERR_INVALID
    # bogus (never dereferenced) pointers with bad sizes or flags
    fake = ctypes.c_void_p(0x1000)
    assert L.ipfb_wiener(G, fake, fake, fake, -1.0, 1, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    assert L.ipfb_wiener(G, fake, fake, fake, float("nan"), 1, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    assert L.ipfb_wiener(G, fake, fake, fake, 0.01, 1, fake, fake, 16, None) == ipfb.ERR_WORKSPACE
    assert L.upchannelize(fake, 4096, 1000, fake, None, 0, None) == ipfb.ERR_UNSUPPORTED
    g_bad = ipfb.geom(100, 4, 64)
    assert L.ipfb_wiener(ctypes.byref(g_bad), fake, fake, fake, 0.01, 1, fake, fake, 1 << 30, None) \
        == ipfb.ERR_UNSUPPORTED
    g_taps = ipfb.geom(256, 17, 64)
    assert L.ipfb_wiener(ctypes.byref(g_taps), fake, fake, fake, 0.01, 1, fake, fake, 1 << 30, None) \
        == ipfb.ERR_UNSUPPORTED
    # forward without a scale needs its FP64 reduction workspace
    assert L.pfb_forward(G, fake, fake, None, fake, fake, None, None, 0, None) == ipfb.ERR_WORKSPACE
    g_up = ipfb.geom(256, 4, 64)
    assert L.ipfb_wiener_upchannelize(ctypes.byref(g_up), fake, fake, fake, 0.01, 1, 3, fake, None, fake,
                                      1 << 30, None) == ipfb.ERR_UNSUPPORTED
    assert ipfb.lib().ipfb_set_max_column_run(1000) == ipfb.ERR_INVALID
    # learned-preconditioner entry points
    assert L.ipfb_net_nparams() == ipfb.NET_NPARAMS == 10145
    assert L.ipfb_net_forward(None, 1, 16, fake, fake, fake, 1 << 20, None) == ipfb.ERR_INVALID
    assert L.ipfb_net_forward(fake, 0, 16, fake, fake, fake, 1 << 20, None) == ipfb.ERR_INVALID
    assert L.ipfb_net_forward(fake, 1, 16, fake, fake, fake, 16, None) == ipfb.ERR_WORKSPACE
    assert L.ipfb_net_grad(fake, 1, 16, fake, fake, None, None, fake, 1 << 20, None) == ipfb.ERR_INVALID
    assert L.ipfb_net_adam(fake, fake, fake, fake, 10, 0, 1e-3, 0.9, 0.999, 1e-8, None) == ipfb.ERR_INVALID
    assert L.ipfb_net_adam(fake, fake, fake, fake, 10, 1, 1e-3, 1.0, 0.999, 1e-8, None) == ipfb.ERR_INVALID
    prm = ipfb.MLParams(0.1, 1.0, 1e-6, 10, 2)
    g_ml = ipfb.geom(256, 4, 512)
    assert L.ipfb_ml_solve(ctypes.byref(g_ml), fake, fake, fake, ctypes.byref(prm), fake, fake, None, fake, 0,
                           fake, fake, fake, 1 << 40, None) == ipfb.ERR_INVALID      # learned needs the net
    assert L.ipfb_ml_solve(ctypes.byref(g_ml), fake, fake, fake, ctypes.byref(prm), fake, fake, fake, fake, 0,
                           fake, fake, fake, 16, None) == ipfb.ERR_WORKSPACE
    assert L.ipfb_ml_training_pairs(ctypes.byref(g_ml), fake, ctypes.byref(prm), fake, fake, fake, fake, -1,
                                    fake, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    bad = (ctypes.c_int * 2)(3, 128)    # pair 128 does not exist for lblock 256
    assert L.ipfb_ml_training_pairs(ctypes.byref(g_ml), fake, ctypes.byref(prm), fake, fake, fake, bad, 2,
                                    fake, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    # code arrays are read with 16-byte loads: an unaligned start is refused
    odd = ctypes.c_void_p(0x1008)
    assert L.ipfb_wiener(G, odd, fake, fake, 0.01, 1, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    # the overlap-save inverse: margin, run length and workspace are checked on the host
    g_s = ipfb.geom(256, 4, 64)
    assert L.ipfb_wiener_stream(ctypes.byref(g_s), 1000, fake, fake, fake, 0.01, 1, 32, fake, fake, 1 << 30,
                                None) == ipfb.ERR_INVALID          # 64 - 2 * 32 < 1
    assert L.ipfb_wiener_stream(ctypes.byref(g_s), 32, fake, fake, fake, 0.01, 1, 8, fake, fake, 1 << 30,
                                None) == ipfb.ERR_INVALID          # run shorter than one chunk
    assert L.ipfb_wiener_stream(ctypes.byref(g_s), 1000, fake, fake, fake, 0.01, 1, 8, fake, fake, 16,
                                None) == ipfb.ERR_WORKSPACE
    # the windowed re-channelizer: taps, block size and workspace are checked on the host
    assert L.upchannelize_pfb(fake, 1 << 20, 4096, 0, fake, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    assert L.upchannelize_pfb(fake, 1 << 20, 3000, 4, fake, fake, fake, 1 << 30, None) == ipfb.ERR_UNSUPPORTED
    assert L.upchannelize_pfb(fake, 1 << 20, 4096, 4, fake, fake, fake, 16, None) == ipfb.ERR_WORKSPACE
    # general eigenvalue filters: mode, threshold and gains are checked on the host
    assert L.ipfb_filter(G, fake, fake, fake, 7, 0.1, None, fake, fake, 1 << 30, None) == ipfb.ERR_INVALID
    assert L.ipfb_filter(G, fake, fake, fake, ipfb.FILTER_THRESHOLD, -1.0, None, fake, fake, 1 << 30, None) \
        == ipfb.ERR_INVALID
    assert L.ipfb_filter(G, fake, fake, fake, ipfb.FILTER_GAINS, 0.0, None, fake, fake, 1 << 30, None) \
        == ipfb.ERR_INVALID
    assert L.ipfb_filter(G, fake, fake, fake, ipfb.FILTER_THRESHOLD, 0.1, None, fake, fake, 16, None) \
        == ipfb.ERR_WORKSPACE
    # the up-channelizer's workspace is moved with 16-byte copies: 16-byte aligned
    assert L.ipfb_wiener_upchannelize(ctypes.byref(g_up), fake, fake, fake, 0.01, 1, 64, fake, None, odd,
                                      1 << 30, None) == ipfb.ERR_INVALID


def test_binding_refuses_cpu_tensors():
    torch = pytest.importorskip("torch")
    x = torch.zeros(1024, dtype=torch.float32)
    w = torch.zeros(4, 256, dtype=torch.float32)
    with pytest.raises(TypeError):
        ipfb.pfb_forward(x, w)
    with pytest.raises(TypeError):
        ipfb.upchannelize(x, 1024)



def test_batched_plan_lengths_and_default_variants():
    """The batched plan is built on the host alone (descriptor pointers are checked, never
    dereferenced): the Bluestein length classes report their kernels -- the tuned
    defaults for the powers of two, the fixed 5- and 6-CTA kernels for 20480 and
    24576 -- and a length that is neither is refused."""
    L = ipfb.lib()
    fake = 0x10000
    shapes = [(1024, 1024), (2048, 1500), (4096, 3000), (1024, 5000), (1024, 9000), (2048, 11000), (1024, 16384)]
    descs = (ipfb.StreamDesc * len(shapes))()
    for i, (N, J) in enumerate(shapes):
        descs[i] = ipfb.StreamDesc(N, 4, J, fake, fake, fake, 0.0141, fake)
    plan = ctypes.c_void_p()
    nbytes = ctypes.c_size_t(0)
    assert L.ipfb_batched_plan(descs, len(shapes), 1, None, ctypes.byref(plan), ctypes.byref(nbytes)) == 0
    assert nbytes.value > 0
    buf = ctypes.create_string_buffer(64)

    def variant(M):
        rc = L.ipfb_batched_variant(plan, M, buf, 64)
        return buf.value.decode() if rc == 0 else rc

    assert variant(2048) == "c1_ts16_r32" and variant(4096) == "c1_ts16_r32"
    assert variant(8192) == "c1_t256_r32"
    assert variant(16384) == "c1_t1024_r32" and variant(32768) == "c2_t1024_r32"
    assert variant(20480) == "c5_t256_r32" and variant(24576) == "c6_t256_r32"
    assert variant(28672) == ipfb.ERR_INVALID and variant(65536) == ipfb.ERR_INVALID
    assert L.ipfb_batched_free(plan) == 0
    # frame counts outside 1024 .. 16384 and unaligned code arrays are refused
    for N, J, codes in ((1024, 16385, fake), (1024, 1023, fake), (1024, 4000, fake + 8)):
        one = (ipfb.StreamDesc * 1)(ipfb.StreamDesc(N, 4, J, codes, fake, fake, 0.0141, fake))
        p = ctypes.c_void_p()
        assert L.ipfb_batched_plan(one, 1, 1, None, ctypes.byref(p), ctypes.byref(nbytes)) != 0
