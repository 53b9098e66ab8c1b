"""GPU parity of the ML solve with its CG vectors in HBM (columns longer than the
on-chip run; Sec. 4.2, Eq. chi squared) against the FP64 oracle, through the C ABI.

Small cases reach the path by lowering the on-chip column run to 512 frames
(ipfb_set_max_column_run): 1024-, 2048- and 4096-frame columns then run with the
residue split C = 2, 4, 8 (S = 512; the Wiener preconditioner is the 2-, 4- and 8-CTA
cluster transform) and 1, 1 and 2 tiles of 2048 frames per pair.  The full-size case
is the paper's 2^27 samples (lblock 2048, 65536 frames: C = 8, S = 8192, 32 tiles per
pair) on sampled columns.

Both sides solve the same SPD system per column.  The GPU (FP32 vectors, FP64
reductions) stops at a relative residual `tol`; the tests recompute the residual of
the GPU answer in FP64, bound its distance to the oracle's dense-accurate solution by
||r|| / lambda_min(A) where a dense eigen-solve is affordable, and compare iteration
counts with the oracle's FP64 (P)CG."""
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


@pytest.fixture
def short_run():
    ipfb.set_max_column_run(512)
    yield
    ipfb.set_max_column_run(8192)


def _instance(N, J, seed, frac=0.1, nchunks=8, ntap=4):
    x = synth.stream_config(N, J, seed)
    w = opfb.sinc_hamming_window(N, ntap).astype(np.float32).astype(np.float64)
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


def _solve(codes, scale, w, sig2, mask, prior, **kw):
    xg, it, res = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior),
                                **kw)
    return xg.cpu().numpy().astype(np.float64), it.cpu().numpy(), res.cpu().numpy()


@pytest.mark.parametrize("precond", ["none", "wiener"])
@pytest.mark.parametrize("N,J", [(64, 1024), (64, 2048), (64, 4096)])
def test_mlbig_parity(short_run, N, J, precond):
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 21)
    # the HBM-resident path's workspace: seven pair-packed vectors and the mask bits at least
    assert ipfb.workspace_size(ipfb.geom(N, 4, J), ipfb.OP_ML) >= 7 * (N // 2) * J * 8 + (N // 2) * J
    tol = 1e-6
    xg, it, res = _solve(codes, scale, w, sig2, mask, prior, precond=precond, tol=tol, max_iter=5000)
    xg = xg.reshape(J, N)
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)
    tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, xg)
    assert np.all(res[0] <= tol)               # the GPU's own stopping test
    assert np.all(tr <= 5 * tol), tr.max()     # true residual in FP64
    assert np.allclose(res[1], tr, rtol=0.2, atol=2e-7)
    # FP32 and FP64 (P)CG take about the same number of steps to reach tol
    _, oit, _ = oml.ml_solve_d(d, w, sig2, M, P, 1.0, precond, tol, 20000)
    assert np.all(np.abs(it - oit) <= np.maximum(3, 0.15 * oit)), (it, oit)
    X, _, _ = oml.ml_solve_d(d, w, sig2, M, P, 1.0, "wiener", 1e-12, 20000)
    rel = np.linalg.norm(xg - X, axis=0) / np.linalg.norm(X, axis=0)
    assert np.all(rel < 1e-3), rel.max()
    if J <= 2048:
        B = oml.rhs(w, d, sig2, M, P, 1.0)
        for n in (0, N // 4, N // 2 - 1, N // 2, N - 1):
            A = _dense_A(w[:, n], sig2, M[:, n], J)
            lmin = np.linalg.eigvalsh(A)[0]
            rn = np.linalg.norm(B[:, n] - A @ xg[:, n])
            err = np.linalg.norm(xg[:, n] - X[:, n])
            assert err <= rn / lmin * 1.01 + 1e-9 * np.linalg.norm(X[:, n]), (n, err, rn / lmin)


@pytest.mark.parametrize("precond,steps", [("none", 25), ("wiener", 8)])
@pytest.mark.parametrize("N,J", [(256, 1024), (64, 4096)])
def test_mlbig_fixed_steps_match_oracle(short_run, N, J, precond, steps):
    # the Sec. 4.3 protocol: a Wiener-filtered start and a fixed number of steps with
    # unit weights on both terms; both sides run the same Krylov recursion, so the
    # iterates agree to FP32 round-off amplified by the steps
    x = synth.stream_config(N, J, 31)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    d = oml.polyphase_data(codes, scale, N)
    sig2 = float(np.var(d - opfb.polyphase_sum(x, w)))
    phi2 = 0.0141
    mask = synth.path_sample_mask(N, J, synth.saved_paths(N, 0.03))
    prior = x.astype(np.float32)
    wg = cuda(w.astype(np.float32))
    x0 = ipfb.ipfb_wiener(cuda(codes), cuda(scale), wg, phi2)
    lam = 1.0 / sig2
    xg, it, _ = ipfb.ml_solve(cuda(codes), cuda(scale), wg, sig2, cuda(mask), cuda(prior), prior_weight=lam,
                              precond=precond, tol=0.0, max_iter=steps, x0=x0)
    torch.cuda.synchronize()
    assert int(it.max()) == steps and int(it.min()) >= 1
    X0 = oml.wiener_initial_guess(d, w, phi2)
    Xo = oml.ml_solve_d(d, w, sig2, mask.reshape(J, N).astype(np.float64), prior.reshape(J, N).astype(np.float64),
                        lam, precond, 0.0, steps, x0=X0)[0]
    got = xg.cpu().numpy().reshape(J, N).astype(np.float64)
    rel = np.sqrt(np.mean((got - Xo) ** 2) / np.mean(Xo ** 2))
    assert rel < 1e-4, rel


def test_mlbig_cap_zero_steps_and_restart(short_run):
    N, J = 64, 1024
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 22)
    rng = np.random.default_rng(5)
    x0 = (x + 0.1 * rng.standard_normal(x.shape)).astype(np.float32)
    # no step: the initial guess comes back unchanged, the residuals are those of x0
    xg, it, res = _solve(codes, scale, w, sig2, mask, prior, tol=1e-6, max_iter=0, x0=cuda(x0))
    assert np.all(it == 0)
    assert np.array_equal(xg.astype(np.float32), x0)
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)
    tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, x0.reshape(J, N).astype(np.float64))
    assert np.allclose(res[0], tr, rtol=1e-3) and np.allclose(res[1], tr, rtol=1e-3)
    # a hard cap stops early and reports a residual above tol
    _, it3, res3 = _solve(codes, scale, w, sig2, mask, prior, tol=1e-6, max_iter=3)
    assert it3.max() == 3 and res3[0].max() > 1e-6
    # restarting from a converged answer needs (almost) nothing
    xs, _, _ = _solve(codes, scale, w, sig2, mask, prior, tol=1e-6, max_iter=5000)
    _, it2, _ = _solve(codes, scale, w, sig2, mask, prior, tol=1e-5, max_iter=5000, x0=cuda(xs.astype(np.float32)))
    assert it2.max() <= 2


def test_mlbig_no_mask_is_the_exact_inverse(short_run):
    N, J = 64, 2048
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 23)
    mask[:] = 0
    xg, it, res = _solve(codes, scale, w, sig2, mask, prior, precond="wiener", tol=1e-5, max_iter=50)
    # without a prior the Wiener preconditioner is the exact inverse of the operator
    assert np.all(it <= 2)
    ref = oipfb.ipfb_wiener(codes, scale, w, 0.0)
    assert np.sqrt(np.mean((xg - ref) ** 2) / np.mean(ref ** 2)) < 1e-3


def test_mlbig_generic_taps(short_run):
    # an 8-tap window takes the 15-tap stencil (taps past the window are zero)
    N, J = 64, 2048
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 24, ntap=8)
    for precond in ("none", "wiener"):
        xg, it, res = _solve(codes, scale, w, sig2, mask, prior, precond=precond, tol=1e-6, max_iter=5000)
        M = mask.reshape(J, N).astype(np.float64)
        P = prior.reshape(J, N).astype(np.float64)
        tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, xg.reshape(J, N))
        assert np.all(res[0] <= 1e-6) and np.all(tr <= 5e-6), tr.max()
        _, oit, _ = oml.ml_solve_d(d, w, sig2, M, P, 1.0, precond, 1e-6, 20000)
        assert np.all(np.abs(it - oit) <= np.maximum(3, 0.15 * oit))


def test_mlbig_agrees_with_the_on_chip_solve():
    N, J = 64, 2048
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 25)
    out = {}
    for run in (8192, 512):
        ipfb.set_max_column_run(run)
        try:
            out[run] = _solve(codes, scale, w, sig2, mask, prior, precond="wiener", tol=1e-6, max_iter=500)
        finally:
            ipfb.set_max_column_run(8192)
    (xa, ia, _), (xb, ib, _) = out[8192], out[512]
    assert np.all(np.abs(ia - ib) <= 1)
    assert np.sqrt(np.mean((xa - xb) ** 2) / np.mean(xa ** 2)) < 1e-4


def test_mlbig_stream_chunks_beyond_the_on_chip_run(short_run):
    # overlap-save with chunks solved by the HBM-resident path: 2 chunks of 1024 frames
    N, chunk, margin, nspec = 64, 1024, 128, 1792
    x = synth.stream_config(N, nspec, 45)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, spec = opfb.pfb_forward(x, w)
    d = oml.polyphase_data(codes, scale, N)
    sig2 = float(np.var(d - opfb.polyphase_sum(x, w)))
    mask = synth.path_sample_mask(N, nspec, synth.saved_paths(N, 0.03))
    prior = x.astype(np.float32)
    rng = np.random.default_rng(46)
    x0 = (x + 0.3 * rng.standard_normal(x.shape)).astype(np.float32)
    lam = 1.0 / sig2
    xg, it, res = ipfb.ml_solve_stream(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                       cuda(prior), chunk, margin, prior_weight=lam, tol=0.0, max_iter=25,
                                       x0=cuda(x0))
    got = xg.cpu().numpy().astype(np.float64)
    ref, oit, _ = oml.ml_solve_stream(codes, scale, w, sig2, mask, prior.astype(np.float64), chunk, margin, lam,
                                      "none", 0.0, 25, x0.astype(np.float64))
    assert np.sqrt(np.mean((got - ref) ** 2) / np.mean(ref ** 2)) < 1e-4
    assert int(it.max()) == 25


@pytest.mark.parametrize("run,J", [(512, 2048), (8192, 16384)])
def test_mlbig_recorded_inside_a_callers_graph(run, J):
    """The solve neither synchronises nor reads anything back: recorded inside the
    caller's torch.cuda.graph (its WHILE node and kernels join the capture) and
    replayed, it gives the eager answer bit for bit (the sums are fixed-order)."""
    N = 64
    ipfb.set_max_column_run(run)
    try:
        x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 27)
        args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
        ws = torch.empty(ipfb.workspace_size(ipfb.geom(N, 4, J), ipfb.OP_ML), dtype=torch.uint8, device="cuda")
        for precond in ("wiener", "none"):
            xe, ite, re = ipfb.ml_solve(*args, precond=precond, tol=1e-6, max_iter=3000, workspace=ws)
            xe, ite, re = xe.clone(), ite.clone(), re.clone()
            torch.cuda.synchronize()
            graph = torch.cuda.CUDAGraph()
            side = torch.cuda.Stream()
            side.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(side):
                with torch.cuda.graph(graph, stream=side):
                    xg, itg, rg = ipfb.ml_solve(*args, precond=precond, tol=1e-6, max_iter=3000, workspace=ws)
            torch.cuda.current_stream().wait_stream(side)
            for _ in range(2):
                xg.zero_()
                graph.replay()
                torch.cuda.synchronize()
                assert torch.equal(xg, xe) and torch.equal(itg, ite) and torch.equal(rg, re), precond
    finally:
        ipfb.set_max_column_run(8192)


def _check_sampled_columns(dcols, w64, sig2, M, P, G, it_cols, tol, precond):
    """Sampled columns of a long solve against the oracle's column-wise solve.
    In FP32 the true residual exceeds the recursive one (the stopping test) by the
    rounding gap of finite-precision CG, about k u ||A|| max_j ||x_j|| after k steps
    (Greenbaum 1997), u = 2^-24, ||A|| <= max_k |W_n(k)|^2 / sigma^2 + lam; near column
    N/2 that floor is ~1e-6 of ||b|| at 65536 frames.  The distance to the exact solution
    is bounded by ||A^-1|| ||b - A x||, ||A^-1|| from inverse iteration with the oracle's
    PCG (a lower estimate, hence the factor 2)."""
    J = dcols.shape[0]
    X, _, _ = oml.ml_solve_d(dcols, w64, sig2, M, P, 1.0, "wiener", 1e-11, 5000)
    B = oml.rhs(w64, dcols, sig2, M, P, 1.0)
    bn, xn = np.linalg.norm(B, axis=0), np.linalg.norm(X, axis=0)
    tr = oml.true_relative_residual(dcols, w64, sig2, M, P, 1.0, G)
    Anorm = (np.abs(oipfb.eigenvalues(w64, J)) ** 2).max(axis=0) / sig2 + 1.0
    gap = 2.0 * np.maximum(it_cols, 1) * 2.0 ** -24 * Anorm * xn / bn
    assert np.all(tr <= tol + gap), (tr, gap)
    V = np.random.default_rng(76).standard_normal(dcols.shape)
    for _ in range(8):
        V /= np.linalg.norm(V, axis=0)
        V = oml.cg(lambda U: oml.normal_operator_fft(w64, U, sig2, M, 1.0), V, np.zeros_like(V), 1e-10, 5000,
                   lambda R: oml.wiener_precond(w64, R, sig2, M, 1.0))[0]
    inv_norm = np.linalg.norm(V, axis=0)
    rel = np.linalg.norm(G - X, axis=0) / xn
    assert np.all(rel <= 2.0 * inv_norm * tr * bn / xn + 1e-6), (rel, inv_norm * tr * bn / xn)
    _, oit, _ = oml.ml_solve_d(dcols, w64, sig2, M, P, 1.0, precond, tol, 20000)
    assert np.all(np.abs(it_cols - oit) <= np.maximum(3, 0.15 * oit)), (it_cols, oit)
    return rel


@pytest.mark.parametrize("J,ntap", [(16384, 4), (32768, 4), (16384, 8)])
def test_mlbig_two_and_four_cta_runs_of_8192(J, ntap):
    """16384 and 32768 frames: residue splits C = 2, 4 with S = 8192 (the default on-chip
    run), 8 and 16 tiles per pair; an 8-tap window takes the generic-tap transform and the
    15-tap stencil; lblock 256 (128 at 32768 frames), 10 % prior; sampled columns against
    the oracle, the stopping test and true residuals on every column."""
    N = 256 if J <= 16384 else 128
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 26, nchunks=32, ntap=ntap)
    ipfb.set_max_column_run(8192)
    xg, it, res = _solve(codes, scale, w, sig2, mask, prior, precond="wiener", tol=1e-6, max_iter=500)
    assert np.all(res[0] <= 1e-6) and np.all(res[1] <= 1e-5)
    cols = np.array([0, 1, N // 2 - 1, N // 2, N // 2 + 1, N - 1, N // 3, 3 * N // 4])
    M = mask.reshape(J, N)[:, cols].astype(np.float64)
    P = prior.reshape(J, N)[:, cols].astype(np.float64)
    G = xg.reshape(J, N)[:, cols]
    rel = _check_sampled_columns(d[:, cols], w[:, cols], sig2, M, P, G, it[cols], 1e-6, "wiener")
    assert np.all(rel[[0, 1, 5, 6, 7]] < 1e-5), rel   # the well-conditioned columns


@pytest.mark.parametrize("N,precond", [(2048, "wiener"), (2048, "none"), (4096, "wiener")])
def test_mlbig_paper_size_sampled_columns(N, precond):
    """The paper's size (lblock 2048, ntap 4, 65536 frames: 2^27 samples) and the
    benchmark's pipeline geometry (lblock 4096: 2^28 samples), 10 % of the samples saved
    as 256 chunks; random 4-bit codes and channel steps, a Gaussian prior of the data's
    scale, sigma^2 = 0.0141 var(d).  Every column's own stopping test and true residual;
    sampled columns (the edges, the worst-conditioned column N/2 and its neighbours,
    seeded ones) against the oracle's column-wise solve."""
    J = 65536
    ipfb.set_max_column_run(8192)
    dev = torch.device("cuda", 0)
    codes = synth.random_code_bytes(J, N // 2, 71)
    scale = synth.random_scale(N // 2 + 1, 72)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    rng = np.random.default_rng(73)
    cols = np.array([0, 1, N // 2 - 1, N // 2, N // 2 + 1, N - 1] + [int(c) for c in rng.integers(2, N - 2, size=3)])
    dcols = oipfb.data_columns(codes, scale, N, cols)
    dstd = float(np.std(dcols))
    sig2 = 0.0141 * dstd ** 2
    starts, L = synth.prior_chunks(N * J, 256, 0.1, 74)
    mask = synth.mask_from_chunks(N * J, starts, L)
    prior = synth.gaussian_stream_torch(N * J, 75, dev) * dstd
    tol = 1e-6
    xg, it, res = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w), sig2, cuda(mask), prior, precond=precond, tol=tol,
                                max_iter=3000)
    torch.cuda.synchronize()
    res = res.cpu().numpy()
    it = it.cpu().numpy()
    assert np.all(res[0] <= tol)
    assert np.all(res[1] <= 1e-5), res[1].max()
    M = mask.reshape(J, N)[:, cols].astype(np.float64)
    P = prior.reshape(J, N)[:, cols].double().cpu().numpy()
    w64 = w.astype(np.float64)[:, cols]
    G = xg.reshape(J, N)[:, cols].double().cpu().numpy()
    rel = _check_sampled_columns(dcols, w64, sig2, M, P, G, it[cols], tol, precond)
    assert np.all(rel[[0, 1, 5]] < 1e-5), rel   # the edge columns are well conditioned
