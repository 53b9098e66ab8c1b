"""The GELU constants the net kernels evaluate (csrc/gelu_poly.cuh), checked on the host
against scipy's erf: GELU(x) = x Phi(x) and GELU'(x) = Phi(x) + x phi(x), evaluated as
the device does (max(x, 0) - |x| exp(-x^2/2) R(|x|), R a polynomial, FP32 steps)."""
import numpy as np
import pytest
from scipy.special import erf, erfc

from paper_2608_23441_b300 import gelu_fit


def _exact(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _exact_grad(x):
    x = np.asarray(x, dtype=np.float64)
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


@pytest.fixture(scope="module")
def coef():
    return gelu_fit.read_header()


def test_header_shape(coef):
    assert len(coef) == gelu_fit.DEG + 1
    assert coef[0] == np.float32(0.5)  # R(0) = Q(0) = 1/2


def test_fp32_gelu_within_bound(coef):
    x = np.linspace(-12.0, 12.0, 400001).astype(np.float32)
    g = gelu_fit.gelu_fp32(x, coef).astype(np.float64)
    assert np.max(np.abs(g - _exact(x))) <= 3e-7
    # relative accuracy near zero, where GELU(x) ~ x / 2
    xs = np.concatenate([np.geomspace(1e-6, 0.5, 2000), -np.geomspace(1e-6, 0.5, 2000)]).astype(np.float32)
    gs = gelu_fit.gelu_fp32(xs, coef).astype(np.float64)
    assert np.max(np.abs(gs - _exact(xs)) / np.abs(_exact(xs))) <= 2e-6
    # exact zero and the saturated ends
    assert gelu_fit.gelu_fp32(np.array([0.0]), coef)[0] == 0.0
    assert gelu_fit.gelu_fp32(np.array([30.0]), coef)[0] == np.float32(30.0)
    assert gelu_fit.gelu_fp32(np.array([-30.0]), coef)[0] == 0.0


def test_fp32_gelu_derivative_within_bound(coef):
    f = np.float32
    x = np.linspace(-12.0, 12.0, 200001).astype(f)
    a = np.abs(x)
    t = np.minimum(a, f(gelu_fit.CLAMP))
    r = np.full_like(t, coef[-1])
    for k in range(len(coef) - 2, -1, -1):
        r = (r * t + coef[k]).astype(f)
    e = np.exp(-0.5 * a.astype(np.float64) ** 2).astype(f)
    q = (e * r).astype(f)
    d = (np.where(x >= 0, f(1) - q, q) + (x * f(1.0 / np.sqrt(2.0 * np.pi))) * e).astype(np.float64)
    assert np.max(np.abs(d - _exact_grad(x))) <= 5e-7


def test_fit_reproduces_the_header(coef):
    c = gelu_fit.fit()
    assert np.allclose(c.astype(np.float32), coef, rtol=1e-4, atol=1e-9)


def test_tail_function_is_the_scaled_complement():
    # R(a) = Q(a) exp(a^2 / 2): Q from the normal CDF at a few points
    a = np.array([0.0, 0.5, 1.7, 3.2, 5.9])
    q = 0.5 * erfc(a / np.sqrt(2.0))
    assert np.allclose(gelu_fit.scaled_tail(a), q * np.exp(0.5 * a * a), rtol=1e-12)
