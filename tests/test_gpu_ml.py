"""GPU parity of the ML conjugate-gradient solve (Sec. 4.2, Eq. chi squared)
against the FP64 oracle, through the C ABI.

Both sides solve the same SPD system A x = b per column.  The GPU (FP32 vectors,
FP64 reductions) stops at a relative residual `tol`; the test recomputes the
residual of the GPU answer in FP64 and bounds its distance to the oracle's
dense-accurate solution by ||r|| / lambda_min(A) (A symmetric positive definite),
with lambda_min from a dense eigen-solve at these small sizes."""
import numpy as np
import pytest

from oracle import ipfb as oipfb
from oracle import ml as oml
from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402


def cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _instance(N, J, seed, frac=0.1, nchunks=8):
    x = synth.stream_config(N, J, seed)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    d = oml.polyphase_data(codes, scale, N)
    sig2 = float(np.var(d - opfb.polyphase_sum(x, w)))
    starts, L = synth.prior_chunks(N * J, nchunks, frac, seed)
    mask = synth.mask_from_chunks(N * J, starts, L)
    prior = x.astype(np.float32)
    return x, w, codes, scale, d, sig2, mask, prior


def _dense_A(wcol, sig2, mcol, J):
    Cm = oipfb.dense_circulant(wcol, J)
    return Cm.T @ Cm / sig2 + np.diag(mcol)


@pytest.mark.parametrize("precond", ["none", "wiener"])
@pytest.mark.parametrize("N,J", [(64, 256), (128, 512)])
def test_ml_cg_parity_small(N, J, precond):
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 7)
    tol = 1e-6
    xg, it, res = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                cuda(prior), precond=precond, tol=tol, max_iter=5000)
    xg = xg.cpu().numpy().reshape(J, N).astype(np.float64)
    it = it.cpu().numpy()
    res = res.cpu().numpy()
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)
    X, oit, orel = oml.ml_solve_d(d, w, sig2, M, P, 1.0, "none", 1e-12, 20000)
    tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, xg)
    assert np.all(res[0] <= tol)               # the GPU's own stopping test
    assert np.all(tr <= 5 * tol), tr.max()     # true residual in FP64
    assert np.allclose(res[1], tr, rtol=0.2, atol=2e-7)
    B = oml.rhs(w, d, sig2, M, P, 1.0)
    for n in range(N):
        A = _dense_A(w[:, n], sig2, M[:, n], J)
        lmin = np.linalg.eigvalsh(A)[0]
        rn = np.linalg.norm(B[:, n] - A @ xg[:, n])
        err = np.linalg.norm(xg[:, n] - X[:, n])
        assert err <= rn / lmin * 1.01 + 1e-9 * np.linalg.norm(X[:, n]), (n, err, rn / lmin)
    if precond == "none":
        # FP32 and FP64 CG take about the same number of steps to reach 1e-6
        _, oit6, _ = oml.ml_solve_d(d, w, sig2, M, P, 1.0, "none", tol, 20000)
        assert np.all(np.abs(it - oit6) <= np.maximum(3, 0.15 * oit6))


def test_ml_wiener_pcg_no_mask_one_step():
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 8)
    mask[:] = 0
    xg, it, res = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                cuda(prior), precond="wiener", tol=1e-5, max_iter=50)
    it = it.cpu().numpy()
    assert np.all(it <= 2)
    ref = oipfb.ipfb_wiener(codes, scale, w, 0.0)
    got = xg.cpu().numpy()
    # without a prior the ML solution is the exact circulant inverse
    assert np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref ** 2)) < 1e-3


def test_ml_initial_guess_and_iteration_cap():
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 9)
    wg = cuda(w.astype(np.float32))
    xs, it_full, _ = ipfb.ml_solve(cuda(codes), cuda(scale), wg, sig2, cuda(mask), cuda(prior), tol=1e-6,
                                   max_iter=5000)
    # restarting from the converged answer needs (almost) nothing
    _, it2, res2 = ipfb.ml_solve(cuda(codes), cuda(scale), wg, sig2, cuda(mask), cuda(prior), tol=1e-5,
                                 max_iter=5000, x0=xs)
    assert it2.cpu().numpy().max() <= 2
    # a hard cap stops early and reports a residual above tol
    _, it3, res3 = ipfb.ml_solve(cuda(codes), cuda(scale), wg, sig2, cuda(mask), cuda(prior), tol=1e-6,
                                 max_iter=3)
    assert it3.cpu().numpy().max() <= 3
    assert res3.cpu().numpy()[0].max() > 1e-6


def test_ml_config4_sampled_columns():
    # lblock 4096, ntap 4, 8192 spectra, 10 % of samples saved as 64 chunks
    N, J = 4096, 8192
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 4, frac=0.1, nchunks=64)
    for precond in ("none", "wiener"):
        xg, it, res = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                    cuda(prior), precond=precond, tol=1e-6, max_iter=4000)
        res = res.cpu().numpy()
        assert np.all(res[0] <= 1e-6)
        assert np.all(res[1] <= 1e-5)
        cols = np.array([0, 1, 1500, N // 2 - 2, N // 2, N // 2 + 1, N - 1])
        M = mask.reshape(J, N)[:, cols].astype(np.float64)
        P = prior.reshape(J, N)[:, cols].astype(np.float64)
        X, _, _ = oml.ml_solve_d(d[:, cols], w[:, cols], sig2, M, P, 1.0, "wiener", 1e-11, 5000)
        G = xg.cpu().numpy().reshape(J, N)[:, cols].astype(np.float64)
        rel = np.linalg.norm(G - X, axis=0) / np.linalg.norm(X, axis=0)
        assert np.all(rel < 1e-3), rel
        # reconstruction error against the truth agrees to 1e-3 relative
        T = x.reshape(J, N)[:, cols]
        eg = np.linalg.norm(G - T, axis=0) / np.linalg.norm(T, axis=0)
        eo = np.linalg.norm(X - T, axis=0) / np.linalg.norm(T, axis=0)
        assert np.all(np.abs(eg / eo - 1) < 1e-3)


@pytest.mark.parametrize("beta", [0.01, 0.03, 0.10])
def test_ml_paper_protocol_matches_oracle(beta):
    # Sec. 4.3 protocol: every 4th sample of the L central sub-filter paths saved
    # (beta = L / (4 N)), the Wiener-filtered inverse as the initial guess, then a
    # fixed 25 plain-CG iterations.  Both sides take the same 25 steps of the same
    # Krylov recursion from starting points that agree to ~1e-7 (the Wiener parity),
    # so the iterates agree to FP32 round-off amplified by 25 steps.
    N, J = 256, 512
    x = synth.stream_config(N, J, 41)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    d = oml.polyphase_data(codes, scale, N)
    sig2 = float(np.var(d - opfb.polyphase_sum(x, w)))
    phi2 = 0.0141
    L = synth.saved_paths(N, beta)
    mask = synth.path_sample_mask(N, J, L)
    assert abs(mask.mean() - L / (4 * N)) < 1e-12
    prior = x.astype(np.float32)
    wg = cuda(w.astype(np.float32))
    x0 = ipfb.ipfb_wiener(cuda(codes), cuda(scale), wg, phi2)
    lam = 1.0 / sig2   # unit weights on the data and prior terms of Eq. chi squared
    xg, it, _ = ipfb.ml_solve(cuda(codes), cuda(scale), wg, sig2, cuda(mask), cuda(prior), prior_weight=lam,
                              tol=0.0, max_iter=25, x0=x0)
    torch.cuda.synchronize()
    # columns with saved samples take all 25 steps; a column whose FP32 residual reaches
    # exactly zero (no saved samples: the Wiener start is nearly the solution) stops there
    assert int(it.max()) == 25 and int(it.min()) >= 1
    X0 = oml.wiener_initial_guess(d, w, phi2)
    Xo = oml.ml_solve_d(d, w, sig2, mask.reshape(J, N).astype(np.float64), prior.reshape(J, N).astype(np.float64),
                        lam, "none", 0.0, 25, x0=X0)[0]
    got = xg.cpu().numpy().reshape(J, N).astype(np.float64)
    rel = np.sqrt(np.mean((got - Xo) ** 2) / np.mean(Xo ** 2))
    assert rel < 1e-4, rel
    # the 25 steps lower the objective (Eq. chi squared) below that of the Wiener start
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)

    def chi2(X):
        r = d - oml.apply_C(w, X)
        return np.sum(r * r) / sig2 + lam * np.sum(M * (X - P) ** 2)

    assert chi2(got) < chi2(X0), (chi2(got), chi2(X0))


def test_accuracy_simulation_runs_and_orders_the_methods():
    # the Sec. 4.3 simulation at a small size (2^21 samples, 16 re-channelized blocks):
    # every figure finite; the Wiener filter removes the no-filter blow-up near the
    # channel edges and lowers the timestream error
    from paper_2608_23441_b300 import accuracy
    out = accuracy.run(torch, torch.device("cuda", 0), nframes=1024, seed=3, betas=(0.10,), prior_weights=("1",))
    m = out["methods"]
    assert set(m) == {"no_filter", "wiener", "ml_beta_0.10_prior_1"}
    for st in m.values():
        assert all(np.isfinite(v) for v in st.values())
    assert m["wiener"]["max"] < m["no_filter"]["max"]
    assert m["wiener"]["timestream_error"] < m["no_filter"]["timestream_error"]
    assert m["no_filter"]["median_at_channel_centres"] < 0.05


def test_ml_stream_matches_oracle_overlap_save():
    """ipfb_ml_solve_stream (overlap-save ML over a run longer than one solve) against
    the oracle's chunk-by-chunk solve with the same chunks: lblock 256, a run of 1280
    spectra in chunks of 512 with 64-frame margins (three chunks, the last aligned to
    the run's end), the Sec. 4.3 protocol per chunk (a fixed 25 plain-CG steps from a
    given initial guess, unit weights), so both sides take the same Krylov steps and
    agree to FP32 round-off amplified by 25 steps; iterations and residuals are the
    largest over the chunks."""
    N, chunk, margin, nspec = 256, 512, 64, 1280
    x = synth.stream_config(N, nspec, 43)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    d = oml.polyphase_data(codes, scale, N)
    sig2 = float(np.var(d - opfb.polyphase_sum(x, w)))
    L = synth.saved_paths(N, 0.03)
    mask = synth.path_sample_mask(N, nspec, L)
    prior = x.astype(np.float32)
    rng = np.random.default_rng(44)
    x0 = (x + 0.3 * rng.standard_normal(x.shape)).astype(np.float32)
    lam = 1.0 / sig2
    xg, it, res = ipfb.ml_solve_stream(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                       cuda(prior), chunk, margin, prior_weight=lam, tol=0.0, max_iter=25,
                                       x0=cuda(x0))
    got = xg.cpu().numpy().astype(np.float64)
    assert got.shape == ((nspec - 2 * margin) * N,)
    ref, oit, _ = oml.ml_solve_stream(codes, scale, w, sig2, mask, prior.astype(np.float64), chunk, margin, lam,
                                      "none", 0.0, 25, x0.astype(np.float64))
    rel = np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref ** 2))
    assert rel < 1e-4, rel
    assert int(it.max()) == 25 and np.all(it.cpu().numpy() <= 25)
    # the interior of every chunk is written once: no frame left at the initial guess
    x0k = x0.reshape(nspec, N)[margin:nspec - margin].reshape(-1).astype(np.float64)
    assert np.min(np.abs(got - x0k).reshape(-1, N).max(axis=1)) > 0


def test_ml_stream_argument_checks():
    N, chunk = 256, 512
    g = ipfb.geom(N, 4, chunk)
    f = ipfb.lib().ipfb_ml_solve_stream
    fake = torch.empty(1 << 16, device="cuda")
    p = ipfb.ctypes.c_void_p(fake.data_ptr())
    prm = ipfb.MLParams(0.1, 1.0, 1e-6, 10, 2, 0)
    # the learned preconditioner is not offered chunk by chunk
    assert f(ipfb.ctypes.byref(g), 1024, p, p, p, ipfb.ctypes.byref(prm), p, p, None, 64, p, p, p, p, 1 << 30,
             None) == ipfb.ERR_UNSUPPORTED
    prm = ipfb.MLParams(0.1, 1.0, 1e-6, 10, 0, 0)
    for nspec, margin in ((500, 64), (1024, 256), (1024, -1)):
        assert f(ipfb.ctypes.byref(g), nspec, p, p, p, ipfb.ctypes.byref(prm), p, p, None, margin, p, p, p, p,
                 1 << 30, None) == ipfb.ERR_INVALID
