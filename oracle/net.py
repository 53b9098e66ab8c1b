"""Oracle: learned preconditioner for the ML conjugate-gradient solve (FP64).

Test infrastructure only (see oracle/__init__.py).

The paper has no learned component; this follows the workload's specification:
a per-column 1-D convolutional net of three layers (2 -> 32 -> 32 -> 1 channels,
kernel 9, GELU between layers), circular padding along the frame axis, weights
shared by all columns, BF16 operands with FP32 accumulation on the GPU.

Readings:
  * input of column n: the Wiener-preconditioned residual u = M_W r (Eq. wiener
    weights applied as the ML preconditioner) scaled by its RMS s, and the prior
    mask m; output z = u + lam mbar M_W(s g(u / s, m)) = M_W(r + lam mbar s g), a
    learned correction of the Wiener preconditioner passed through it: mode k of the
    correction is scaled by the prior's share of the Wiener denominator,
    rho(k) = lam mbar / (|W(k)|^2 / sigma^2 + lam mbar) (lam mbar = prior weight x
    the column's mask mean), so it acts where the prior term dominates (the
    near-null eigenvalues of App. A) and leaves the modes the Wiener step already
    resolves nearly untouched;
  * GELU in its exact form x Phi(x) = 0.5 x (1 + erf(x / sqrt 2)) (Hendrycks and
    Gimpel 2016), the standard normal CDF Phi written through erf;
  * training target: the CG error e = x* - x_k of the residual r_k = A e; loss
    mean over positions of (g - (e - u)/s)^2;
  * the preconditioner is nonlinear, so the outer iteration is flexible CG with
    the Polak-Ribiere beta = r_{k+1}.(z_{k+1} - z_k) / (r_k.z_k) (Notay 2000).
BF16 emulation: round-to-nearest-even of the float32 bit pattern to 16 bits.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erf

K = 9
HALF = K // 2
C0, C1, C2, C3 = 2, 32, 32, 1
INV_SQRT2 = 1.0 / math.sqrt(2.0)
INV_SQRT2PI = 1.0 / math.sqrt(2.0 * math.pi)


def n_params() -> int:
    return C1 * C0 * K + C1 + C2 * C1 * K + C2 + C3 * C2 * K + C3


def init_params(seed: int, scale3: float = 0.0) -> dict:
    """He-style uniform init for layers 1-2; layer 3 starts at `scale3` (0 gives the
    Wiener preconditioner exactly)."""
    rng = np.random.default_rng(seed)
    def u(shape, fan_in):
        b = math.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, size=shape)
    return {
        "w1": u((C1, C0, K), C0 * K), "b1": np.zeros(C1),
        "w2": u((C2, C1, K), C1 * K), "b2": np.zeros(C2),
        "w3": u((C3, C2, K), C2 * K) * scale3, "b3": np.zeros(C3),
    }


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([p[k].reshape(-1) for k in ("w1", "b1", "w2", "b2", "w3", "b3")])


def unflatten(v: np.ndarray) -> dict:
    shapes = [("w1", (C1, C0, K)), ("b1", (C1,)), ("w2", (C2, C1, K)), ("b2", (C2,)),
              ("w3", (C3, C2, K)), ("b3", (C3,))]
    out, o = {}, 0
    for name, sh in shapes:
        n = int(np.prod(sh))
        out[name] = np.asarray(v[o:o + n], dtype=np.float64).reshape(sh)
        o += n
    return out


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round half to even on the float32 bits)."""
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> 16) & 1
    r = ((b + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(x):
    """x Phi(x), Phi the standard normal CDF."""
    return 0.5 * x * (1.0 + erf(x * INV_SQRT2))


def gelu_grad(x):
    """d/dx [x Phi(x)] = Phi(x) + x phi(x), phi the standard normal density."""
    return 0.5 * (1.0 + erf(x * INV_SQRT2)) + x * INV_SQRT2PI * np.exp(-0.5 * x * x)


def conv(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Circular 1-D convolution (cross-correlation, as in deep-learning conv layers):
    y[co, j] = b[co] + sum_{ci, t} w[co, ci, t] x[ci, (j + t - 4) mod J].
    x: [ci, J] (or [batch, ci, J]); returns [co, J] (or [batch, co, J])."""
    y = np.zeros(x.shape[:-2] + (w.shape[0], x.shape[-1]))
    for t in range(K):
        xs = np.roll(x, -(t - HALF), axis=-1)          # xs[.., j] = x[.., j + t - 4]
        y += np.einsum("oc,...cj->...oj", w[:, :, t], xs)
    return y + b[:, None]


def conv_backward(x, w, dy):
    """Gradients of conv(x, w, b) given dy: (dx, dw, db).  x: [B, ci, J], dy: [B, co, J]."""
    x3 = x.reshape((-1,) + x.shape[-2:])
    dy3 = dy.reshape((-1,) + dy.shape[-2:])
    dw = np.zeros_like(w)
    dx = np.zeros_like(x3)
    for t in range(K):
        xs = np.roll(x3, -(t - HALF), axis=-1)
        dw[:, :, t] = np.einsum("boj,bcj->oc", dy3, xs)
        dxs = np.einsum("oc,boj->bcj", w[:, :, t], dy3)   # gradient w.r.t. xs
        dx += np.roll(dxs, (t - HALF), axis=-1)
    db = dy3.sum(axis=(0, 2))
    return dx.reshape(x.shape), dw, db


def forward(p: dict, xin: np.ndarray, emulate_bf16: bool = False, cache: bool = False):
    """xin: [..., 2, J] (channels u/s, mask).  Returns g [..., J] (and the cache)."""
    q = (lambda a: bf16(a)) if emulate_bf16 else (lambda a: a)
    x0 = q(xin)
    z1 = conv(x0, q(p["w1"]), p["b1"])
    a1 = q(gelu(z1))
    z2 = conv(a1, q(p["w2"]), p["b2"])
    a2 = q(gelu(z2))
    y = conv(a2, q(p["w3"]), p["b3"])[..., 0, :]
    if cache:
        return y, (x0, z1, a1, z2, a2)
    return y


def loss_and_grad(p: dict, xin: np.ndarray, target: np.ndarray, emulate_bf16: bool = False):
    """Mean squared error over all positions and batch items, and its gradient."""
    y, (x0, z1, a1, z2, a2) = forward(p, xin, emulate_bf16, cache=True)
    q = (lambda a: bf16(a)) if emulate_bf16 else (lambda a: a)
    n = y.size
    diff = y - target
    L = float(np.sum(diff * diff) / n)
    dy = (2.0 / n) * diff[..., None, :]
    da2, dw3, db3 = conv_backward(a2, q(p["w3"]), dy)
    dz2 = da2 * gelu_grad(z2)
    da1, dw2, db2 = conv_backward(a1, q(p["w2"]), dz2)
    dz1 = da1 * gelu_grad(z1)
    _, dw1, db1 = conv_backward(x0, q(p["w1"]), dz1)
    return L, {"w1": dw1, "b1": db1, "w2": dw2, "b2": db2, "w3": dw3, "b3": db3}


def net_input(u: np.ndarray, m: np.ndarray):
    """Channels (u/s, m) per column and the scale s = RMS(u).  u, m: [J, ncols]."""
    s = np.sqrt(np.mean(u * u, axis=0))
    s = np.where(s == 0, 1.0, s)
    return np.stack([(u / s).T, m.T.astype(np.float64)], axis=1), s   # [ncols, 2, J]


def apply_precond(p: dict, u: np.ndarray, m: np.ndarray, wiener, lam_mbar, emulate_bf16: bool = False) -> np.ndarray:
    """z = u + lam mbar M_W(s g(u/s, m)), column by column.  u, m: [J, ncols];
    wiener(V) applies M_W to the columns of V; lam_mbar: [ncols] (or a scalar)."""
    xin, s = net_input(u, m)
    g = forward(p, xin, emulate_bf16)          # [ncols, J]
    return u + np.asarray(lam_mbar, dtype=np.float64) * wiener((g * s[:, None]).T)


class Adam:
    """Adam (Kingma and Ba 2015) on a flat parameter vector."""

    def __init__(self, n, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, grad):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * grad
        self.v = self.b2 * self.v + (1 - self.b2) * grad * grad
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def fcg(apply_A, B, X0, precond, tol, max_iter):
    """Flexible CG (Notay 2000) with the Polak-Ribiere beta, every column on its own.
    precond(R) -> Z may be nonlinear.  Returns (X, iterations, relative residual)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    bnorm = np.sqrt(np.sum(B * B, axis=0))
    bnorm = np.where(bnorm == 0, 1.0, bnorm)
    R = B - apply_A(X)
    Z = precond(R)
    P = Z.copy()
    rz = np.sum(R * Z, axis=0)
    it = np.zeros(B.shape[1], dtype=np.int64)
    rel = np.sqrt(np.sum(R * R, axis=0)) / bnorm
    active = rel > tol
    for _ in range(int(max_iter)):
        if not active.any():
            break
        AP = apply_A(P)
        pAp = np.sum(P * AP, axis=0)
        alpha = np.where(active, rz / np.where(pAp == 0, 1.0, pAp), 0.0)
        X += alpha * P
        R_new = R - alpha * AP
        it += active
        rel = np.sqrt(np.sum(R_new * R_new, axis=0)) / bnorm
        active = active & (rel > tol)
        Z_new = precond(R_new)
        beta = np.where(active, np.sum(R_new * (Z_new - Z), axis=0) / np.where(rz == 0, 1.0, rz), 0.0)
        P = np.where(active[None, :], Z_new + beta * P, P)
        rz = np.where(active, np.sum(R_new * Z_new, axis=0), rz)
        R, Z = R_new, Z_new
    return X, it, rel
