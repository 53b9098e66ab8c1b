"""Pins for the oracle's learned-preconditioner pieces: conv layer against a direct
sum and against FFT circular correlation, analytic gradients against central
finite differences, BF16 rounding against hand-made bit patterns, flexible CG
against plain PCG for a linear preconditioner, and the zero-output net giving the
Wiener preconditioner exactly."""
import numpy as np
import pytest

from oracle import ml as oml
from oracle import net
from oracle import pfb as opfb


def test_param_count():
    assert net.n_params() == 10145


def test_conv_matches_direct_sum_and_fft():
    rng = np.random.default_rng(0)
    J = 37
    x = rng.standard_normal((3, J))
    w = rng.standard_normal((2, 3, 9))
    b = rng.standard_normal(2)
    y = net.conv(x, w, b)
    for co in range(2):
        for j in range(J):
            s = b[co] + sum(w[co, ci, t] * x[ci, (j + t - 4) % J] for ci in range(3) for t in range(9))
            assert abs(y[co, j] - s) < 1e-12
    # circular cross-correlation through the FFT
    for co in range(2):
        acc = np.zeros(J, dtype=complex)
        for ci in range(3):
            h = np.zeros(J)
            for t in range(9):
                h[(t - 4) % J] += w[co, ci, t]
            acc += np.fft.ifft(np.fft.fft(x[ci]) * np.conj(np.fft.fft(h)))
        assert np.allclose(y[co], acc.real + b[co], atol=1e-12)


def test_gelu_and_its_derivative():
    x = np.linspace(-5, 5, 101)
    h = 1e-6
    assert np.allclose(net.gelu_grad(x), (net.gelu(x + h) - net.gelu(x - h)) / (2 * h), atol=1e-8)
    assert net.gelu(np.array([0.0]))[0] == 0.0
    assert abs(net.gelu(np.array([10.0]))[0] - 10.0) < 1e-12
    # x Phi(x) against the normal CDF integrated by quadrature (no erf involved)
    from scipy.integrate import quad
    for v in (-2.3, -0.7, 0.4, 1.9):
        phi_int, _ = quad(lambda t: np.exp(-0.5 * t * t) / np.sqrt(2 * np.pi), -np.inf, v)
        assert abs(net.gelu(np.array([v]))[0] - v * phi_int) < 1e-12
    # odd part: gelu(x) - gelu(-x) = x
    assert np.allclose(net.gelu(x) - net.gelu(-x), x, atol=1e-14)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = net.init_params(3, scale3=1.0)
    for k in p:
        p[k] = p[k] + 0.05 * rng.standard_normal(p[k].shape)
    xin = rng.standard_normal((2, 2, 24))
    xin[:, 1] = (rng.uniform(size=(2, 24)) < 0.3)
    tgt = rng.standard_normal((2, 24))
    L, g = net.loss_and_grad(p, xin, tgt)
    theta = net.flatten(p)
    grad = net.flatten(g)
    idx = rng.choice(theta.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        Lp, _ = net.loss_and_grad(net.unflatten(tp), xin, tgt)
        Lm, _ = net.loss_and_grad(net.unflatten(tm), xin, tgt)
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, grad[i])


def test_bf16_rounding():
    vals = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 2 ** -7, 1.0 + 3 * 2 ** -8, -2.5, 3.0e-5], dtype=np.float32)
    r = net.bf16(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0                # exactly halfway: round to even (mantissa ...0)
    assert r[2] == 1.0 + 2 ** -7      # representable
    assert r[3] == 1.0 + 2 ** -6      # halfway between ...01 and ...10: to even
    assert r[4] == -2.5
    assert abs(r[5] / 3.0e-5 - 1) < 2 ** -8


def test_fcg_equals_pcg_for_linear_preconditioner():
    N, p, J = 8, 4, 48
    w = opfb.sinc_hamming_window(N, p)
    rng = np.random.default_rng(4)
    d = rng.standard_normal((J, N))
    mask = (rng.uniform(size=(J, N)) < 0.15).astype(float)
    prior = rng.standard_normal((J, N))
    sig2 = 0.02
    A = lambda V: oml.normal_operator_fft(w, V, sig2, mask, 1.0)  # noqa: E731
    M = lambda R: oml.wiener_precond(w, R, sig2, mask, 1.0)       # noqa: E731
    B = oml.rhs(w, d, sig2, mask, prior, 1.0)
    X1, it1, _ = oml.cg(A, B, np.zeros_like(B), 1e-10, 500, M)
    X2, it2, _ = net.fcg(A, B, np.zeros_like(B), M, 1e-10, 500)
    assert np.allclose(X1, X2, atol=1e-8 * np.abs(X1).max())
    assert np.all(np.abs(it1 - it2) <= 1)


def test_zero_net_is_wiener_preconditioner():
    N, p, J = 8, 4, 32
    w = opfb.sinc_hamming_window(N, p)
    rng = np.random.default_rng(5)
    R = rng.standard_normal((J, N))
    mask = (rng.uniform(size=(J, N)) < 0.2).astype(float)
    Mw = lambda V: oml.wiener_precond(w, V, 0.05, mask, 1.0)  # noqa: E731
    u = Mw(R)
    p0 = net.init_params(0, scale3=0.0)
    z = net.apply_precond(p0, u, mask, Mw, mask.mean(axis=0))
    assert np.allclose(z, u, atol=1e-14)


def test_constant_net_output_enters_scaled_by_the_prior_share_at_dc():
    # A net whose output is the constant c (all weights zero, output bias c) adds
    # c s times the Wiener filter's response to a constant, weighted by lam mbar: a
    # constant is the k = 0 mode, so the correction is c s rho(0) with
    # rho(0) = lam mbar / (W_n(0)^2 / sigma^2 + lam mbar), W_n(0) = sum_r w[r, n]
    # (Sec. 3.1 eigenvalue at k = 0) -- the prior's share of the Wiener denominator.
    N, p, J, sig2, lam = 8, 4, 32, 0.05, 0.7
    w = opfb.sinc_hamming_window(N, p)
    rng = np.random.default_rng(6)
    R = rng.standard_normal((J, N))
    mask = (rng.uniform(size=(J, N)) < 0.3).astype(float)
    mbar = mask.mean(axis=0)
    Mw = lambda V: oml.wiener_precond(w, V, sig2, mask, lam)  # noqa: E731
    u = Mw(R)
    prm = net.init_params(0, scale3=0.0)
    for k in prm:
        prm[k] = np.zeros_like(prm[k])
    c = 0.37
    prm["b3"] = np.array([c])
    z = net.apply_precond(prm, u, mask, Mw, lam * mbar)
    s = np.sqrt(np.mean(u * u, axis=0))
    W0 = w.sum(axis=0)
    rho0 = lam * mbar / (W0 ** 2 / sig2 + lam * mbar)
    assert np.allclose(z - u, (c * s * rho0)[None, :], rtol=1e-12, atol=1e-14)


def test_adam_minimises_a_quadratic():
    a = net.Adam(3, lr=0.05)
    th = np.array([3.0, -2.0, 1.0])
    for _ in range(2000):
        th = a.step(th, 2 * th)
    assert np.abs(th).max() < 1e-3


def test_adam_first_steps_closed_form():
    # Kingma and Ba (2015), Algorithm 1, worked by hand.  Step 1 from zero moments:
    # m = (1 - b1) g, v = (1 - b2) g^2, so the bias-corrected mh = g and vh = g^2 and
    # every parameter moves by exactly lr g / (|g| + eps).
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-8
    g = np.array([2.0, -0.5, 1e-3, 0.0, -40.0])
    th0 = np.array([1.0, 2.0, -3.0, 0.5, 0.0])
    a = net.Adam(5, lr=lr, b1=b1, b2=b2, eps=eps)
    th1 = a.step(th0, g)
    assert np.allclose(th1, th0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # Step 2 with the same gradient: mh = g (1 - b1)(1 + b1) / (1 - b1^2) = g and
    # vh = g^2 again, so the same move; a missing bias correction would shrink it
    # by (1 - b1^2) / sqrt(1 - b2^2) ~ 4.25.
    b = net.Adam(5, lr=lr, b1=b1, b2=b2, eps=eps)
    t = b.step(th0, g)
    t = b.step(t, g)
    assert np.allclose(t, th0 - 2 * lr * g / (np.abs(g) + eps), rtol=0, atol=1e-14)
    # Step 2 with the gradient reversed: m = -(1 - b1)^2 g, mh = -g (1 - b1)/(1 + b1),
    # v = (1 - b2)(1 + b2) g^2 -> vh = g^2; the second move is
    # +lr (1 - b1)/(1 + b1) g / (|g| + eps).
    c = net.Adam(5, lr=lr, b1=b1, b2=b2, eps=eps)
    t = c.step(th0, g)
    t = c.step(t, -g)
    want = th0 - lr * g / (np.abs(g) + eps) + lr * (1 - b1) / (1 + b1) * g / (np.abs(g) + eps)
    assert np.allclose(t, want, rtol=0, atol=1e-14)
