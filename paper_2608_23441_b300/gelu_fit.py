"""Coefficients of the GELU evaluation in the net kernels (writes csrc/gelu_poly.cuh).

    python -m paper_2608_23441_b300.gelu_fit [--check]

GELU(x) = x Phi(x) with Phi the standard normal CDF.  With a = |x| and the upper
tail Q(a) = 1 - Phi(a),

    GELU(x) = max(x, 0) - a Q(a),      Q(a) = exp(-a^2 / 2) R(a),
    R(a) = erfcx(a / sqrt 2) / 2       (erfcx(z) = exp(z^2) erfc(z), the scaled complement),

so the only transcendental left is the Gaussian factor (one hardware exp2), and R is
smooth and slowly varying (R(0) = 1/2, R(a) ~ 1 / (a sqrt(2 pi)) for large a).  R is
replaced by a polynomial of degree DEG on [0, CLAMP] with R(0) = 1/2 fixed, chosen to
minimise the largest weighted error a exp(-a^2 / 2) |p(a) - R(a)|, which is the error it
leaves in GELU(x).  The minimax fit is reached by Lawson's iteratively reweighted
least squares (Lawson 1961) on Chebyshev-distributed points.  Beyond CLAMP the
polynomial is held at its value at CLAMP; there a exp(-a^2 / 2) < 1e-7, so the GELU
error stays below the FP32 rounding of the result.

The same R gives the derivative GELU'(x) = Phi(x) + x phi(x), phi(x) = exp(-x^2 / 2) /
sqrt(2 pi), Phi(x) = 1 - Q(a) for x >= 0 and Q(a) for x < 0.  The generated constants
are checked against scipy's erf by the host tests (FP32 evaluation within 3e-7
absolute of x Phi(x) for |x| <= 12).
"""
from __future__ import annotations

import argparse
import os

import numpy as np

DEG = 11
CLAMP = 6.0
HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "csrc", "gelu_poly.cuh")


def scaled_tail(a: np.ndarray) -> np.ndarray:
    """R(a) = Q(a) exp(a^2 / 2) = erfcx(a / sqrt 2) / 2."""
    from scipy.special import erfcx
    return 0.5 * erfcx(np.asarray(a, dtype=np.float64) / np.sqrt(2.0))


def fit(deg: int = DEG, clamp: float = CLAMP, npts: int = 4000, iters: int = 100) -> np.ndarray:
    """Coefficients c[0..deg] (c[0] = 1/2) of p(a) = sum_k c[k] a^k ~= R(a) on [0, clamp]."""
    a = 0.5 * clamp * (1.0 - np.cos(np.linspace(0.0, np.pi, npts)))[1:]
    basis = a[:, None] * np.vander(a, deg, increasing=True)  # a^1 .. a^deg
    y = scaled_tail(a) - 0.5
    weight = a * np.exp(-0.5 * a * a)
    lawson = np.ones_like(a)
    for _ in range(iters):
        w = weight * lawson
        s, *_ = np.linalg.lstsq(basis * w[:, None], y * w, rcond=None)
        err = np.abs(basis @ s - y) * weight
        lawson = lawson * (err / err.max()) ** 0.3 + 1e-12
        lawson /= lawson.max()
    return np.concatenate([[0.5], s])


def gelu_fp32(x: np.ndarray, coef: np.ndarray, clamp: float = CLAMP) -> np.ndarray:
    """The device evaluation in FP32, operation by operation (exp in FP64 rounded to
    FP32 stands for the hardware exp2, whose relative error is ~2^-22)."""
    f = np.float32
    x = np.asarray(x, dtype=f)
    a = np.abs(x)
    t = np.minimum(a, f(clamp))
    c = np.asarray(coef, dtype=f)
    r = np.full_like(t, c[-1])
    for k in range(len(c) - 2, -1, -1):
        r = (r * t + c[k]).astype(f)
    e = np.exp(-0.5 * a.astype(np.float64) ** 2).astype(f)
    return (np.maximum(x, f(0)) - a * (e * r).astype(f)).astype(f)


def header_text(coef: np.ndarray) -> str:
    c32 = np.asarray(coef, dtype=np.float32)
    body = "".join(f"  k == {k} ? {float(v)!r}f :\n" for k, v in enumerate(c32))
    return (
        "// Generated by paper_2608_23441_b300/gelu_fit.py; do not edit.\n"
        "// R(a) = erfcx(a / sqrt 2) / 2 ~= sum_k gelu_r(k) a^k on [0, kGeluClamp] (R(0) = 1/2\n"
        "// exact), the weighted minimax fit that bounds the error of\n"
        "// GELU(x) = max(x, 0) - |x| exp(-x^2 / 2) R(|x|).\n"
        "#pragma once\n\n"
        "namespace ipfb {\n\n"
        f"constexpr int kGeluDeg = {len(c32) - 1};\n"
        f"constexpr float kGeluClamp = {CLAMP!r}f;\n"
        "// coefficient k of R (a function, so that unrolled device loops fold it to an immediate)\n"
        f"constexpr float gelu_r(int k) {{\n  return\n{body}  0.0f;\n}}\n\n"
        "}  // namespace ipfb\n")


def read_header(path: str = HEADER) -> np.ndarray:
    """The coefficients as committed in the generated header."""
    txt = open(path).read()
    import re
    body = txt.split("constexpr float gelu_r(int k)")[1]
    vals = dict((int(k), float(v)) for k, v in re.findall(r"k == (\d+) \? ([-+0-9.e]+)f", body))
    return np.array([vals[k] for k in range(len(vals))], dtype=np.float32)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--check", action="store_true", help="print the FP32 error of the committed header")
    args = ap.parse_args(argv)
    if args.check:
        from scipy.special import erf
        x = np.linspace(-12.0, 12.0, 800001).astype(np.float32)
        g = gelu_fp32(x, read_header()).astype(np.float64)
        x64 = x.astype(np.float64)
        print("max |err|", float(np.max(np.abs(g - 0.5 * x64 * (1.0 + erf(x64 / np.sqrt(2.0)))))))
        return 0
    with open(HEADER, "w") as fh:
        fh.write(header_text(fit()))
    print(HEADER)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
