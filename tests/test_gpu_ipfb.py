"""GPU parity: forward PFB, quantizer, Wiener/exact inverse PFB and
up-channelization through the C ABI, against the FP64 oracle on the same seeded
inputs.

Tolerances (relative RMS over the whole output, the FP32 kernels against FP64):
  exact inverse on well-conditioned windows    1e-5
  Wiener-filtered inverse                      1e-4
  up-channelization, forward spectra           1e-5
  4-bit codes                                  bit-exact on identical float32
                                               (value, step) pairs
The FP32 FFTs have round-off near 1e-7 * sqrt(log2 n) relative; these bounds
leave two orders of magnitude for the conditioning of the per-mode gain
(|G| <= (1 + phi^2) / (2 phi) ~ 4.3 for phi^2 = 0.014).
"""
import numpy as np
import pytest

from oracle import ipfb as oipfb
from oracle import pfb as opfb
from oracle import upchan as oup
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402


def relrms(a, b):
    a = np.asarray(a).astype(np.complex128)
    b = np.asarray(b).astype(np.complex128)
    return float(np.sqrt(np.mean(np.abs(a - b) ** 2)) / np.sqrt(np.mean(np.abs(b) ** 2)))


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(autouse=True)
def _reset_run():
    ipfb.set_max_column_run(8192)
    yield
    ipfb.set_max_column_run(8192)


# ----------------------------------------------------------------------------- quantizer
def test_quantize_bit_exact_on_identical_inputs():
    N, J = 256, 300
    rng = np.random.default_rng(0)
    C = N // 2 + 1
    spec = (rng.standard_normal((J, C)) * 3 + 1j * rng.standard_normal((J, C)) * 3).astype(np.complex64)
    spec[:, 0] = spec[:, 0].real
    spec[:, -1] = spec[:, -1].real
    scale = synth.random_scale(C, 1)
    scale[5] = 0.0  # zero step -> code 0
    # exact decision boundaries: v = (k + 1/2) * s for a power-of-two step
    scale[7] = 0.5
    spec[:10, 7] = (np.arange(10) - 4.5).astype(np.float32) * 0.5 + 1j * 0.25
    q_re, q_im = opfb.quantize_f32(spec.real, scale), opfb.quantize_f32(spec.imag, scale)
    want = opfb.pack_codes(q_re, q_im)
    got = ipfb.pfb_quantize(cuda(spec), cuda(scale)).cpu().numpy()
    assert np.array_equal(got, want)


# ----------------------------------------------------------------------------- forward
@pytest.mark.parametrize("N,J", [(64, 16), (256, 512), (1024, 64), (4096, 40)])
def test_pfb_forward_parity(N, J):
    x = synth.stream_config(N, J, 1, channel=N / 6.3)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    xf = x.astype(np.float32)
    spec_or = opfb.pfb_spectra(xf.astype(np.float64), w.astype(np.float64))
    scale_or = opfb.channel_scale(spec_or)
    codes, scale, spec = ipfb.pfb_forward(cuda(xf), cuda(w), return_spectra=True)
    spec = spec.cpu().numpy()
    scale = scale.cpu().numpy()
    assert relrms(spec, spec_or) < 1e-5
    assert np.max(np.abs(scale / scale_or - 1)) < 1e-5
    # codes with the oracle's step: mismatches only where FP32 spectrum error can
    # move v/Delta across a decision boundary
    codes2, _, _ = ipfb.pfb_forward(cuda(xf), cuda(w), scale=cuda(scale_or))
    q_re, q_im = opfb.quantize_spectra(spec_or, scale_or)
    want = opfb.pack_codes(q_re, q_im)
    got = codes2.cpu().numpy()
    bad = got != want
    # Sec. 4.3 quantizer read as a float32 decision (the oracle's channel step, the
    # GPU's FP32 spectrum): a code may differ from the FP64 oracle's only where the
    # FP32 spectrum's own error moves v / Delta across a decision boundary, i.e. the
    # oracle's v / Delta lies within 1e-5 steps of a half-integer.  The flips are
    # counted and reported.
    t_re = spec_or.real[:, : N // 2] / scale_or[None, : N // 2]
    t_im = spec_or.imag[:, : N // 2] / scale_or[None, : N // 2]
    dist = np.minimum(np.abs(np.abs(t_re) % 1 - 0.5), np.abs(np.abs(t_im) % 1 - 0.5))
    t_ny = spec_or.real[:, N // 2] / scale_or[N // 2]
    dist[:, 0] = np.minimum(np.abs(np.abs(t_re[:, 0]) % 1 - 0.5), np.abs(np.abs(t_ny) % 1 - 0.5))
    # the FP32 spectrum's error in steps, largest over all values
    e_re = np.abs(spec.real - spec_or.real) / scale_or[None, :]
    e_im = np.abs(spec.imag - spec_or.imag) / scale_or[None, :]
    err_steps = float(max(e_re.max(), e_im.max()))
    nflip = int(bad.sum())
    print(f"pfb_forward N={N} J={J}: {nflip} of {bad.size} code bytes differ from the FP64 oracle; "
          f"FP32 spectrum error up to {err_steps:.2e} steps")
    assert err_steps < 1e-5
    if nflip:
        assert np.all(dist[bad] <= err_steps)
    # the same codes again from the GPU's own FP32 spectrum with the same step: the
    # decision itself is bit-exact
    want32 = opfb.pack_codes(*opfb.quantize_spectra(spec.astype(np.complex128), scale_or))
    assert np.array_equal(got, want32)


# ----------------------------------------------------------------------------- inverse
CASES = [
    # N, J, noise_level, normalize, column run
    (64, 16, 0.014, True, 8192),
    (256, 512, 0.014, True, 8192),
    (256, 512, 0.014, False, 8192),
    (128, 2048, 0.02, True, 8192),
    (512, 8192, 0.014, True, 8192),
    (64, 1024, 0.014, True, 512),   # cluster of 2
    (64, 2048, 0.014, True, 512),   # cluster of 4
    (128, 4096, 0.014, True, 512),  # cluster of 8
]


@pytest.mark.parametrize("N,J,phi2,norm,run", CASES)
def test_ipfb_wiener_parity(N, J, phi2, norm, run):
    ipfb.set_max_column_run(run)
    x = synth.stream_config(N, J, 3, channel=N / 7.1)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    ref = oipfb.ipfb_wiener(codes, scale, w, phi2, norm)
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), phi2, norm).cpu().numpy()
    assert relrms(got, ref) < 1e-4


@pytest.mark.parametrize("N,J,run", [(64, 64, 8192), (256, 512, 8192), (128, 8192, 8192), (64, 2048, 512),
                                     (128, 4096, 512)])
def test_exact_inverse_well_conditioned(N, J, run):
    # random-tap window with |W| >= 0.1: the exact inverse recovers the input
    ipfb.set_max_column_run(run)
    w = synth.random_taps_window(4, N, 5).astype(np.float32).astype(np.float64)
    x = synth.gaussian_stream(N * J, 6)
    spec = opfb.pfb_spectra(x, w)
    scale = np.full(N // 2 + 1, 0.02, np.float32)
    q_re, q_im = opfb.quantize_spectra(spec, scale)
    codes = opfb.pack_codes(q_re, q_im)
    ref = oipfb.ipfb_wiener(codes, scale, w, 0.0)
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.0).cpu().numpy()
    assert relrms(got, ref) < 1e-5


def test_exact_inverse_recovers_unquantized_input():
    # fine quantizer (no clipping) on a well-conditioned window: x_hat ~ x
    N, J = 256, 256
    w = synth.random_taps_window(4, N, 7).astype(np.float32).astype(np.float64)
    x = synth.gaussian_stream(N * J, 8)
    spec = opfb.pfb_spectra(x, w)
    scale = (np.abs(spec).max(axis=0) / 7.0 * 1.0001).astype(np.float32)
    codes = opfb.pack_codes(*opfb.quantize_spectra(spec, scale))
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.0).cpu().numpy()
    ref = oipfb.ipfb_wiener(codes, scale, w, 0.0)
    assert relrms(got, ref) < 1e-5
    assert relrms(got, x) < 0.2  # only 4-bit quantization noise remains


def test_ipfb_random_codes_edge_columns():
    N, J = 128, 256
    codes = synth.random_code_bytes(J, N // 2, 11)
    scale = synth.random_scale(N // 2 + 1, 12)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.01).cpu().numpy()
    ref = oipfb.ipfb_wiener(codes, scale, w, 0.01)
    assert relrms(got, ref) < 1e-4
    cols = [0, 1, N // 2 - 1, N // 2, N - 1]
    refc = oipfb.ipfb_columns(codes, scale, w, cols, 0.01)
    gotc = got.reshape(J, N)[:, cols]
    assert relrms(gotc, refc) < 1e-4


def test_ipfb_zero_input():
    N, J = 64, 32
    codes = np.zeros((J, N // 2), np.uint8)
    scale = np.ones(N // 2 + 1, np.float32)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w), 0.014).cpu().numpy()
    assert np.all(got == 0)


def test_ipfb_ntap_variants():
    for p in (1, 2, 3, 8):
        N, J = 128, 128
        w = synth.random_taps_window(p, N, 20 + p, spread=0.6 / max(1, p - 1) if p > 1 else 0.3)
        w = w.astype(np.float32).astype(np.float64)
        codes = synth.random_code_bytes(J, N // 2, 30 + p)
        scale = synth.random_scale(N // 2 + 1, 40 + p)
        got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.005).cpu().numpy()
        ref = oipfb.ipfb_wiener(codes, scale, w, 0.005)
        assert relrms(got, ref) < 1e-4, p


# ----------------------------------------------------------------------------- up-channelization
@pytest.mark.parametrize("L,nb", [(1024, 3), (2048, 2), (16384, 2), (65536, 2), (262144, 2)])
def test_upchannelize_parity(L, nb):
    x = synth.gaussian_stream(L * nb + 100, 9).astype(np.float32)
    got = ipfb.upchannelize(cuda(x), L).cpu().numpy()
    ref = oup.upchannelize(x.astype(np.float64), L)
    assert got.shape == ref.shape
    assert relrms(got, ref) < 1e-5


def test_upchannelize_tone_and_nyquist():
    L = 8192
    t = np.arange(2 * L)
    x = (np.cos(2 * np.pi * 1234 * t / L) + 0.5 * (-1.0) ** t + 0.25).astype(np.float32)
    got = ipfb.upchannelize(cuda(x), L).cpu().numpy()
    ref = oup.upchannelize(x.astype(np.float64), L)
    assert relrms(got, ref) < 1e-5
    assert abs(got[0, 1234]) == pytest.approx(L / 2, rel=1e-5)
    assert got[0, L // 2].real == pytest.approx(0.5 * L, rel=1e-5)
    assert got[0, 0].real == pytest.approx(0.25 * L, rel=1e-4)


# ----------------------------------------------------------------------------- pipeline
@pytest.mark.parametrize("N,J,U,run", [(256, 512, 64, 8192), (512, 256, 64, 8192), (64, 1024, 64, 512),
                                       (2048, 128, 64, 8192), (1024, 256, 64, 8192), (1024, 1024, 64, 512),
                                       (4096, 128, 64, 8192),
                                       # columns longer than the run: clusters of C = 4 and 8 CTAs
                                       # of S = 512 frames, lblock 1024 / 2048 / 4096
                                       (1024, 2048, 64, 512), (2048, 4096, 64, 512), (4096, 4096, 64, 512)])
def test_ipfb_wiener_upchannelize(N, J, U, run):
    ipfb.set_max_column_run(run)
    x = synth.stream_config(N, J, 13, ntones=4)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    xr = oipfb.ipfb_wiener(codes, scale, w, 0.014)
    ref = oup.upchannelize(xr, U * N)
    out, xo = ipfb.ipfb_wiener_upchannelize(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.014, U,
                                            want_x=True)
    assert relrms(out.cpu().numpy(), ref) < 1e-4
    assert relrms(xo.cpu().numpy(), xr) < 1e-4


# ----------------------------------------------------------------------------- config 1 end to end
def test_config1_small_wiener():
    # lblock 256, ntap 4, sinc x Hamming 1024, 512 frames, tone at fractional channel 40.3
    N, p, J = 256, 4, 512
    x = synth.stream_config(N, J, 1, channel=40.3)
    w = opfb.sinc_hamming_window(N, p).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    phi2 = float(np.var(opfb.dequantize(codes, scale) - spec) / np.var(spec))
    ref = oipfb.ipfb_wiener(codes, scale, w, phi2)
    got = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), phi2).cpu().numpy()
    assert relrms(got, ref) < 1e-4
    # GPU forward on the same stream gives the same codes except at boundaries
    gc, gs, _ = ipfb.pfb_forward(cuda(x.astype(np.float32)), cuda(w.astype(np.float32)))
    assert np.mean(gc.cpu().numpy() != opfb.pfb_forward(x.astype(np.float32).astype(np.float64), w)[0]) < 2e-3


# ----------------------------------------------------------------------------- general eigenvalue filters
def _threshold_in_gap(absW, q):
    """A threshold between two consecutive |W| values near quantile q, at least 2e-5
    relative away from both: FP32 |W| is within ~1e-6 relative of FP64, so both sides
    keep the same modes."""
    v = np.unique(np.sort(absW.reshape(-1)))
    i0 = int(q * (v.size - 1))
    for i in range(i0, v.size - 1):
        lo, hi = v[i], v[i + 1]
        if hi - lo > 4e-5 * hi:
            return 0.5 * (lo + hi)
    raise AssertionError("no gap")


@pytest.mark.parametrize("N,J,run", [(256, 512, 8192), (64, 2048, 512)])
def test_filter_threshold_pinv_matches_oracle(N, J, run):
    ipfb.set_max_column_run(run)
    x = synth.stream_config(N, J, 61, ntones=3)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    absW = np.abs(oipfb.eigenvalues(w, J))
    for q in (0.02, 0.2):
        thr = _threshold_in_gap(absW, q)
        got = ipfb.ipfb_filter(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), threshold=thr)
        ref = oipfb.ipfb_filter(codes, scale, w, threshold=thr)
        assert relrms(got.cpu().numpy(), ref) < 1e-4, (q, thr)
    # threshold 0 is the exact inverse
    g0 = ipfb.ipfb_filter(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), threshold=0.0)
    e0 = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.0)
    assert relrms(g0.cpu().numpy(), e0.cpu().numpy().astype(np.float64)) < 1e-6
    ipfb.set_max_column_run(8192)


@pytest.mark.parametrize("N,J,run", [(256, 512, 8192), (64, 2048, 512)])
def test_filter_caller_gains_matches_oracle(N, J, run):
    ipfb.set_max_column_run(run)
    x = synth.stream_config(N, J, 62, ntones=3)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    rng = np.random.default_rng(63)
    G = (rng.uniform(0.2, 1.5, size=(N, J // 2 + 1)) * np.exp(1j * rng.uniform(-np.pi, np.pi, size=(N, J // 2 + 1))))
    G[:, 0] = G[:, 0].real                    # DC and Nyquist gains real, as for a real filter
    G[:, -1] = G[:, -1].real
    Gd = torch.from_numpy(G.astype(np.complex64)).cuda()
    got = ipfb.ipfb_filter(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), gains=Gd)
    ref = oipfb.ipfb_filter(codes, scale, w, gains_half=G.astype(np.complex64).astype(np.complex128))
    assert relrms(got.cpu().numpy(), ref) < 1e-4
    # the Wiener gains given as caller gains reproduce ipfb_wiener
    phi2 = 0.014
    Gw = oipfb.gain(oipfb.eigenvalues(w, J), phi2, True)[: J // 2 + 1].T
    gw = ipfb.ipfb_filter(cuda(codes), cuda(scale), cuda(w.astype(np.float32)),
                          gains=torch.from_numpy(np.ascontiguousarray(Gw).astype(np.complex64)).cuda())
    ew = ipfb.ipfb_wiener(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), phi2)
    assert relrms(gw.cpu().numpy(), ew.cpu().numpy().astype(np.float64)) < 1e-5
    ipfb.set_max_column_run(8192)


@pytest.mark.parametrize("L,nb,p", [(4096, 9, 4), (1024, 5, 1), (131072, 3, 4)])
def test_upchannelize_pfb_matches_oracle(L, nb, p):
    # the windowed re-channelizer (a PFB with frames L long, p taps, periodic over blocks)
    x = synth.gaussian_stream(L * nb + 123, 81).astype(np.float32)
    w = opfb.sinc_hamming_window(L, p).astype(np.float32) if p > 1 else np.ones((1, L), np.float32)
    got = ipfb.upchannelize_pfb(cuda(x), cuda(w))
    ref = oup.pfb_upchannelize(x.astype(np.float64), w.astype(np.float64))
    assert got.shape == ref.shape
    assert relrms(got.cpu().numpy(), ref) < 1e-5


# ----------------------------------------------------------------------------- overlap-save inverse
@pytest.mark.parametrize("N,nspec,chunk,margin", [(256, 2000, 512, 64), (64, 4096, 1024, 112), (128, 1024, 1024, 0)])
def test_wiener_stream_matches_oracle(N, nspec, chunk, margin):
    x = synth.stream_config(N, nspec, 95, ntones=3)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    got = ipfb.ipfb_wiener_stream(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), 0.014, chunk, margin)
    ref = oipfb.ipfb_wiener_stream(codes, scale, w, 0.014, chunk, margin)
    assert got.shape[0] == ref.shape[0] == (nspec - 2 * margin) * N
    assert relrms(got.cpu().numpy(), ref) < 1e-4


def test_wiener_stream_approaches_the_global_inverse():
    # a periodic run of 4096 spectra: chunks of 1024 with a 112-frame margin agree with
    # the run's global circulant inverse to the round-off of the FP32 path
    N, J = 64, 4096
    x = synth.stream_config(N, J, 96)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    codes, scale, _ = opfb.pfb_forward(x, w.astype(np.float64))
    wg = cuda(w)
    full = ipfb.ipfb_wiener(cuda(codes), cuda(scale), wg, 0.014).cpu().numpy().reshape(J, N)
    m = 112
    got = ipfb.ipfb_wiener_stream(cuda(codes), cuda(scale), wg, 0.014, 1024, m).cpu().numpy().reshape(-1, N)
    assert relrms(got, full[m:J - m].astype(np.float64)) < 1e-5
