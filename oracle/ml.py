"""Oracle: maximum-likelihood inverse PFB with a time-domain prior (FP64).

Test infrastructure only (see oracle/__init__.py).

Sec. 4.2 (Eq. chi squared):
    chi^2 = (d - A x)^T N^{-1} (d - A x) + (x - p)^T Q^{-1} (x - p),
with A = S W after the N-point inverse FFT has undone F, N = sigma^2 I
(quantization noise white and uniform), Q^{-1} = 1 on saved samples and 0
elsewhere.  A decomposes into the N independent sub-filter correlations of
Sec. 2.3; in the circulant model (Eq. circ_convolution) column n obeys
d_n = C_n x_n with (C_n x)[j] = sum_r w[r, n] x[(j + r) mod J].  Setting the
gradient of chi^2 to zero gives, per column, the normal equations
    (C_n^T C_n / sigma^2 + lam M_n) x_n = C_n^T d_n / sigma^2 + lam M_n p_n,
M_n = diag(mask of column n), lam = prior weight (1 in the paper).  They are
solved by conjugate gradient (Sec. 4.2, citing Shewchuk 1994).

Operator forms: F^dagger(|W_n|^2 F v) / sigma^2 (C^T C is circulant with
eigenvalues |W_n(k)|^2), or the equivalent circular stencil with taps
a[s] = sum_r w_r w_{r+s}, |s| < p.

Readings:
  * A is circulant (exact for the periodic simulation used here), N = sigma^2 I
    with sigma^2 = `noise_var` in d units, Q^{-1} = `prior_weight` * mask.
  * Stopping rule: each column stops when ||r||_2 / ||b||_2 <= tol (so the
    global ratio is below tol too); x0 = 0 unless given.  The paper's own
    protocol (Wiener initial guess, 25 iterations; Sec. 4.3) is also reachable
    through x0 and max_iter.
  * Wiener preconditioner: z = F^dagger[F r / (|W_n|^2/sigma^2 + lam mbar_n)],
    mbar_n the mask fraction of column n (the exact inverse of the operator with
    the mask replaced by its mean).
"""
from __future__ import annotations

import numpy as np

from .ipfb import eigenvalues, frames_from_spectra, gain
from .pfb import dequantize


def columns(x_flat: np.ndarray, lblock: int) -> np.ndarray:
    """[J*N] time order -> [J, N]; column n is the sub-stream x_n (Sec. 2.3)."""
    return np.asarray(x_flat).reshape(-1, lblock)


def apply_C(window: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Circular correlation of every column: (C_n x)[j] = sum_r w[r,n] x[(j+r) mod J]."""
    p, N = window.shape
    out = np.zeros_like(X, dtype=np.float64)
    for r in range(p):
        out += window[r][None, :] * np.roll(X, -r, axis=0)
    return out


def apply_CT(window: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Transpose: (C_n^T y)[i] = sum_r w[r,n] y[(i - r) mod J]."""
    p, N = window.shape
    out = np.zeros_like(Y, dtype=np.float64)
    for r in range(p):
        out += window[r][None, :] * np.roll(Y, r, axis=0)
    return out


def normal_operator_fft(window: np.ndarray, V: np.ndarray, noise_var: float,
                        mask: np.ndarray, prior_weight: float) -> np.ndarray:
    """A v = F^dagger(|W_n|^2 F v)/sigma^2 + lam M v, column by column."""
    J = V.shape[0]
    W2 = np.abs(eigenvalues(window, J)) ** 2
    return np.real(np.fft.ifft(W2 * np.fft.fft(V, axis=0), axis=0)) / noise_var + prior_weight * mask * V


def stencil_taps(window: np.ndarray) -> np.ndarray:
    """a[s, n] = sum_r w[r, n] w[r + s, n] for s = -(p-1) .. p-1 (row s + p - 1)."""
    p, N = window.shape
    a = np.zeros((2 * p - 1, N))
    for s in range(-(p - 1), p):
        for r in range(p):
            if 0 <= r + s < p:
                a[s + p - 1] += window[r] * window[r + s]
    return a


def normal_operator_stencil(window: np.ndarray, V: np.ndarray, noise_var: float,
                            mask: np.ndarray, prior_weight: float) -> np.ndarray:
    """Same operator as a circular (2p-1)-tap stencil:
    (C^T C v)[i] = sum_s a[s] v[(i + s) mod J]."""
    p, N = window.shape
    a = stencil_taps(window)
    out = np.zeros_like(V, dtype=np.float64)
    for s in range(-(p - 1), p):
        out += a[s + p - 1][None, :] * np.roll(V, -s, axis=0)
    return out / noise_var + prior_weight * mask * V


def rhs(window: np.ndarray, d: np.ndarray, noise_var: float, mask: np.ndarray,
        prior: np.ndarray, prior_weight: float) -> np.ndarray:
    """b_n = C_n^T d_n / sigma^2 + lam M_n p_n."""
    return apply_CT(window, d) / noise_var + prior_weight * mask * prior


def wiener_precond(window: np.ndarray, R: np.ndarray, noise_var: float, mask: np.ndarray,
                   prior_weight: float) -> np.ndarray:
    """z_n = F^dagger[F r_n / (|W_n|^2/sigma^2 + lam mbar_n)]."""
    J = R.shape[0]
    W2 = np.abs(eigenvalues(window, J)) ** 2
    mbar = prior_weight * np.mean(mask, axis=0)
    P = W2 / noise_var + mbar[None, :]
    return np.real(np.fft.ifft(np.fft.fft(R, axis=0) / P, axis=0))


def cg(apply_A, B: np.ndarray, X0: np.ndarray, tol: float, max_iter: int,
       precond=None):
    """Preconditioned conjugate gradient (Shewchuk 1994, Sec. B2) on every column
    independently, in FP64.  A column stops updating once ||r|| <= tol ||b||.
    Returns (X, iterations per column, recursive relative residual per column)."""
    X = np.array(X0, dtype=np.float64, copy=True)
    bnorm = np.sqrt(np.sum(B * B, axis=0))
    bnorm = np.where(bnorm == 0, 1.0, bnorm)
    R = B - apply_A(X)
    Z = precond(R) if precond is not None else R
    P = Z.copy()
    rz = np.sum(R * Z, axis=0)
    iters = np.zeros(B.shape[1], dtype=np.int64)
    rel = np.sqrt(np.sum(R * R, axis=0)) / bnorm
    active = rel > tol
    for _ in range(int(max_iter)):
        if not active.any():
            break
        AP = apply_A(P)
        pAp = np.sum(P * AP, axis=0)
        alpha = np.where(active, rz / np.where(pAp == 0, 1.0, pAp), 0.0)
        X += alpha[None, :] * P
        R -= alpha[None, :] * AP
        iters += active
        rel = np.sqrt(np.sum(R * R, axis=0)) / bnorm
        active = active & (rel > tol)
        Z = precond(R) if precond is not None else R
        rz_new = np.sum(R * Z, axis=0)
        beta = np.where(active, rz_new / np.where(rz == 0, 1.0, rz), 0.0)
        P = np.where(active[None, :], Z + beta[None, :] * P, P)
        rz = np.where(active, rz_new, rz)
    return X, iters, rel


def polyphase_data(codes: np.ndarray, scale: np.ndarray, lblock: int) -> np.ndarray:
    """d = N-point inverse real FFT of the dequantized spectra ("undoing F", Sec. 4.2)."""
    return frames_from_spectra(dequantize(codes, scale), lblock)


def ml_solve_d(d: np.ndarray, window: np.ndarray, noise_var: float, mask: np.ndarray,
               prior: np.ndarray, prior_weight: float = 1.0, precond: str = "none",
               tol: float = 1e-6, max_iter: int = 1000, x0: np.ndarray | None = None,
               operator: str = "fft"):
    """ML reconstruction from polyphase data d [J, N] with mask/prior [J, N].
    precond: "none" or "wiener".  Returns (X [J, N], iters [N], rel [N])."""
    op = normal_operator_fft if operator == "fft" else normal_operator_stencil
    A = lambda V: op(window, V, noise_var, mask, prior_weight)  # noqa: E731
    B = rhs(window, d, noise_var, mask, prior, prior_weight)
    M = None
    if precond == "wiener":
        M = lambda R: wiener_precond(window, R, noise_var, mask, prior_weight)  # noqa: E731
    X0 = np.zeros_like(B) if x0 is None else np.asarray(x0, dtype=np.float64).reshape(B.shape)
    return cg(A, B, X0, tol, max_iter, M)


def ml_solve(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, noise_var: float,
             mask_flat: np.ndarray, prior_flat: np.ndarray, prior_weight: float = 1.0,
             precond: str = "none", tol: float = 1e-6, max_iter: int = 1000,
             x0_flat: np.ndarray | None = None, operator: str = "fft"):
    """ML inverse PFB of packed codes; mask/prior in time order [J*N].
    Returns (x_hat [J*N], iters [N], rel [N])."""
    p, N = window.shape
    d = polyphase_data(codes, scale, N)
    mask = columns(mask_flat, N).astype(np.float64)
    prior = columns(prior_flat, N).astype(np.float64)
    x0 = None if x0_flat is None else columns(x0_flat, N)
    X, it, rel = ml_solve_d(d, window, noise_var, mask, prior, prior_weight, precond,
                            tol, max_iter, x0, operator)
    return X.reshape(-1), it, rel


def true_relative_residual(d: np.ndarray, window: np.ndarray, noise_var: float,
                           mask: np.ndarray, prior: np.ndarray, prior_weight: float,
                           X: np.ndarray) -> np.ndarray:
    """||b - A x|| / ||b|| per column, evaluated from scratch in FP64."""
    B = rhs(window, d, noise_var, mask, prior, prior_weight)
    R = B - normal_operator_fft(window, X, noise_var, mask, prior_weight)
    bn = np.sqrt(np.sum(B * B, axis=0))
    return np.sqrt(np.sum(R * R, axis=0)) / np.where(bn == 0, 1.0, bn)


def wiener_initial_guess(d: np.ndarray, window: np.ndarray, noise_level: float) -> np.ndarray:
    """The paper's CG starting point (Sec. 4.3): the Wiener-filtered circulant inverse."""
    J = d.shape[0]
    G = gain(eigenvalues(window, J), noise_level, True)
    return np.real(np.fft.ifft(G * np.fft.fft(d, axis=0), axis=0))


def dense_ml_column(d_col, window_col, noise_var, mask_col, prior_col, prior_weight=1.0):
    """Dense normal-equation solve for one column (pin at tiny J)."""
    from .ipfb import dense_circulant
    J = d_col.shape[0]
    Cm = dense_circulant(window_col, J)
    A = Cm.T @ Cm / noise_var + prior_weight * np.diag(mask_col.astype(np.float64))
    b = Cm.T @ d_col / noise_var + prior_weight * mask_col * prior_col
    return np.linalg.solve(A, b)


def ml_solve_stream(codes: np.ndarray, scale: np.ndarray, window: np.ndarray, noise_var: float,
                    mask_flat: np.ndarray, prior_flat: np.ndarray, chunk: int, margin: int,
                    prior_weight: float = 1.0, precond: str = "none", tol: float = 1e-6,
                    max_iter: int = 1000, x0_flat: np.ndarray | None = None):
    """Overlap-save ML reconstruction of a run of spectra longer than one solve (the
    Sec. 4.2 system solved chunk by chunk, as the Wiener inverse is in
    ipfb.ipfb_wiener_stream): every chunk of `chunk` spectra, with its mask, prior
    values and initial guess, is solved by ml_solve as a periodic system, and its frames
    margin .. chunk - margin are kept (chunk starts from ipfb.stream_chunks).  The
    solution's dependence on data far away decays along the frame axis, so away from a
    chunk's edges it agrees with the solve of the whole run.
    Returns (frames [margin, nspec - margin) in time order [(nspec - 2 margin) * N],
    per-column maxima over the chunks of the iteration counts and of the residuals)."""
    from .ipfb import stream_chunks
    p, N = window.shape
    nspec = codes.shape[0]
    out = np.zeros((nspec - 2 * margin, N))
    it_max = np.zeros(N, dtype=np.int64)
    rel_max = np.zeros(N)
    for st in stream_chunks(nspec, chunk, margin):
        sl = slice(st * N, (st + chunk) * N)
        x0 = None if x0_flat is None else np.asarray(x0_flat)[sl]
        xc, it, rel = ml_solve(codes[st:st + chunk], scale, window, noise_var, np.asarray(mask_flat)[sl],
                               np.asarray(prior_flat)[sl], prior_weight, precond, tol, max_iter, x0)
        out[st:st + chunk - 2 * margin] = xc.reshape(chunk, N)[margin:chunk - margin]
        it_max = np.maximum(it_max, it)
        rel_max = np.maximum(rel_max, rel)
    return out.reshape(-1), it_max, rel_max
