"""Pins for the oracle's window, forward PFB, quantizer and byte packing.

Each check is tied to something the paper or the mathematics fixes, reached by
a different route than the oracle function it checks."""
import json
import os

import numpy as np
import pytest

from oracle import pfb
from paper_2608_23441_b300 import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_numbers.json")))


def brute_dft(v):
    n = v.shape[0]
    k = np.arange(n)
    return np.exp(-2j * np.pi * np.outer(k, k) / n) @ v


@pytest.mark.parametrize("n", [1, 2, 3, 8, 15, 64])
def test_fft_convention_matches_operator_F(n):
    # Sec. 2.3: F_{n,k} = exp(-2 pi i n k / N); the oracle uses numpy's FFT as a primitive.
    v = np.random.default_rng(n).standard_normal(n)
    assert np.allclose(np.fft.fft(v), brute_dft(v), atol=1e-12)
    assert np.allclose(np.fft.rfft(v), brute_dft(v)[: n // 2 + 1], atol=1e-12)


def test_window_values():
    N, p = 64, 4
    w = pfb.sinc_hamming_window(N, p).reshape(-1)
    M = N * p
    # centre: sinc(0) = 1 times the taper
    assert w[M // 2] == pytest.approx(0.54 - 0.46 * np.cos(2 * np.pi * (M // 2) / (M - 1)), abs=1e-15)
    # sinc zeros every N samples away from the centre
    for k in (-2, -1, 1):
        assert abs(w[M // 2 + k * N]) < 1e-15
    # sub-filters have DC response near 1 (App. B assumes W_n ~ 1)
    dc = w.reshape(p, N).sum(axis=0)
    assert 0.98 < dc.mean() < 1.03


def test_pfb_equals_every_pth_bin_of_long_dft():
    # Eq. chan_dft_osamp: a PFB spectrum equals bins k' = p k of the M-point DFT of
    # the windowed segment.
    N, p, J = 16, 4, 10
    x = synth.gaussian_stream(N * J, 3)
    win = pfb.sinc_hamming_window(N, p)
    Y = pfb.pfb_spectra(x, win, periodic=True)
    h = win.reshape(-1)
    M = N * p
    for j in range(J):
        seg = np.array([x[(j * N + m) % (N * J)] for m in range(M)])
        long = brute_dft(seg * h)
        assert np.allclose(Y[j], long[::p][: N // 2 + 1], atol=1e-12)


def test_pfb_nonperiodic_frame_count():
    N, p, J = 8, 4, 12
    x = synth.gaussian_stream(N * J, 5)
    win = pfb.sinc_hamming_window(N, p)
    Yp = pfb.pfb_spectra(x, win, periodic=True)
    Yn = pfb.pfb_spectra(x, win, periodic=False)
    assert Yn.shape == (J - p + 1, N // 2 + 1)
    assert np.allclose(Yp[: J - p + 1], Yn, atol=1e-13)


def test_quantizer_hand_cases():
    s = np.float32(1.0)
    v = np.array([0.5, 1.5, 2.5, -0.5, -1.5, -2.5, 7.49, 7.5, 8.0, -100.0, 3.4999998, 0.0],
                 dtype=np.float32)
    want = [0, 2, 2, 0, -2, -2, 7, 7, 7, -7, 3, 0]
    assert pfb.quantize_f32(v, np.full(v.shape, s, dtype=np.float32)).tolist() == want
    # a zero step gives code 0
    assert pfb.quantize_f32(np.array([3.0], np.float32), np.array([0.0], np.float32)).tolist() == [0]
    # step 0.25: 0.375/0.25 = 1.5 -> 2, 0.625/0.25 = 2.5 -> 2 (exact in float32)
    q = pfb.quantize_f32(np.array([0.375, 0.625], np.float32), np.full(2, 0.25, np.float32))
    assert q.tolist() == [2, 2]


def test_quantizer_error_bound():
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(20000) * 2).astype(np.float32)
    s = np.float32(0.4)
    q = pfb.quantize_f32(v, np.full(v.shape, s, np.float32)).astype(np.float64)
    inside = np.abs(v / s) <= 7.0
    assert np.all(np.abs(v[inside] / float(s) - q[inside]) <= 0.5 + 1e-6)
    assert np.all(np.abs(q) <= 7)


def test_pack_unpack_roundtrip_and_layout():
    J, N = 3, 8
    C = N // 2 + 1
    rng = np.random.default_rng(1)
    q_re = rng.integers(-7, 8, size=(J, C)).astype(np.int8)
    q_im = rng.integers(-7, 8, size=(J, C)).astype(np.int8)
    q_im[:, 0] = 0
    q_im[:, C - 1] = 0
    codes = pfb.pack_codes(q_re, q_im)
    assert codes.shape == (J, N // 2) and codes.dtype == np.uint8
    r2, i2 = pfb.unpack_codes(codes)
    assert np.array_equal(r2, q_re) and np.array_equal(i2, q_im)
    # explicit nibble layout: Re -7 -> 0x9 low, Im 3 -> 0x3 high
    a = np.zeros((1, C), np.int8)
    b = np.zeros((1, C), np.int8)
    a[0, 1], b[0, 1] = -7, 3
    a[0, 0], a[0, C - 1] = 5, -1
    c = pfb.pack_codes(a, b)
    assert c[0, 1] == 0x39
    assert c[0, 0] == 0xF5


def test_quantizer_snr_matches_paper():
    # App. B: step 0.353 sigma gives SNR about 80 (19 dB).
    step = GOLD["quantizer_optimal_step_over_sigma"]["value"]
    snr = pfb.quantization_snr(1.0, step, 2_000_000, 11)
    snr_db = 10 * np.log10(snr)
    assert abs(snr_db - GOLD["quantizer_snr_db_at_optimal_step"]["value"]) < 0.5
    assert 70 < snr < 90
    # Eq. snr_enob with R = 4 bits gives the same 19 dB
    e = GOLD["enob_fit"]
    assert abs(e["slope_db_per_bit"] * e["bits"] + e["offset_db"] - 19.0) < 0.01
    # the step is near-optimal: 0.30 and 0.45 sigma are both worse
    assert pfb.quantization_snr(1.0, 0.30, 500_000, 12) < snr
    assert pfb.quantization_snr(1.0, 0.45, 500_000, 12) < snr


def test_forward_quantized_dc_nyquist_folding():
    N, p, J = 32, 4, 64
    x = synth.stream_config(N, J, 2, channel=5.3)
    win = pfb.sinc_hamming_window(N, p)
    codes, scale, spec = pfb.pfb_forward(x, win)
    assert np.all(spec[:, 0].imag == 0) and np.all(spec[:, -1].imag == 0)
    q_re, q_im = pfb.quantize_spectra(spec, scale)
    r2, i2 = pfb.unpack_codes(codes)
    assert np.array_equal(r2, q_re) and np.array_equal(i2, q_im)
    # per-channel RMS / 2.5 -> about 2.5 steps per RMS, 4-bit codes well exercised
    y = pfb.dequantize(codes, scale)
    err = np.var(y - spec) / np.var(spec)
    assert 0.005 < err < 0.03


def test_channel_rms_hand_cases():
    # Sec. 4.3 quantizer step, read per channel (workload spec): RMS_c over the real
    # and imaginary parts of channel c, i.e. sqrt(sum_j (Re^2 + Im^2) / (2 J)) for
    # interior channels and sqrt(sum_j Re^2 / J) at DC and Nyquist (no imaginary
    # part).  Values worked out by hand: a /J-for-/(2J) slip (a factor sqrt 2), a
    # dropped Im term, or treating DC / Nyquist like interior channels all fail.
    J, C = 4, 5
    spec = np.zeros((J, C), np.complex128)
    spec[:, 1] = 3 + 4j                      # every interior sample 3 + 4i
    spec[:, 2] = [1, 1j, 3 + 4j, 0]          # 1 + 1 + 25 + 0 = 27 over 2J = 8 values
    spec[:, 3] = [2j, -2j, 2j, -2j]          # imaginary only: 16 / 8 = 2
    spec[:, 0] = [2, -2, 2, -2]              # DC, real only: 16 / 4
    spec[:, 4] = [1, -1, 3, 0]               # Nyquist: 1 + 1 + 9 + 0 = 11 over J = 4
    rms = pfb.channel_rms(spec)
    want = np.array([2.0, np.sqrt(12.5), np.sqrt(27 / 8), np.sqrt(2.0), np.sqrt(11 / 4)])
    assert np.allclose(rms, want, rtol=0, atol=1e-15)
    # Delta_c = RMS_c / 2.5, formed in FP64 and rounded once to float32
    sc = pfb.channel_scale(spec)
    assert sc.dtype == np.float32
    assert np.array_equal(sc, (want / 2.5).astype(np.float32))
    assert sc[0] == np.float32(0.8) and sc[1] == np.float32(np.sqrt(12.5) / 2.5)


def test_channel_rms_of_gaussian_spectra_is_sigma():
    # A real-input spectrum of white noise of variance s^2 has E|Y_c|^2 = N s^2 for
    # every channel; the interior channels split it equally between Re and Im
    # (N s^2 / 2 each), DC and Nyquist are real with variance N s^2.  So the
    # per-part RMS is sqrt(N/2) s inside and sqrt(N) s at the two real channels --
    # a ratio of sqrt 2 that the special case must reproduce.
    N, J, s = 64, 4000, 1.7
    x = np.random.default_rng(3).standard_normal((J, N)) * s
    rms = pfb.channel_rms(np.fft.rfft(x, axis=1))
    assert np.allclose(rms[1:-1], np.sqrt(N / 2) * s, rtol=0.03)
    assert np.allclose(rms[[0, -1]], np.sqrt(N) * s, rtol=0.04)
