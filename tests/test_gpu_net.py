"""GPU parity of the learned preconditioner (net forward, gradients, Adam, training
pairs, flexible CG) against the FP64 oracle with BF16 emulation, through the C ABI.

Tolerances: net outputs within 5e-3 and gradients within 1e-2 relative (RMS over
each parameter group) of the oracle with the same BF16 rounding of weights and
activations; the remaining differences are FP32 accumulation order and the rare
BF16 rounding decision that flips between an FP32 and an FP64 pre-activation."""
import numpy as np
import pytest

from oracle import ml as oml
from oracle import net as onet
from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402


def cuda(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def _theta(seed, scale3=1.0, jitter=0.05):
    rng = np.random.default_rng(seed + 100)
    p = onet.init_params(seed, scale3=scale3)
    for k in p:
        p[k] = p[k] + jitter * rng.standard_normal(p[k].shape)
    return onet.flatten(p)


def _xin(ns, J, seed):
    rng = np.random.default_rng(seed)
    x = np.empty((ns, 2, J))
    x[:, 0] = rng.standard_normal((ns, J))
    x[:, 1] = (rng.uniform(size=(ns, J)) < 0.2)
    return x


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("ns,J", [(3, 500), (2, 37), (1, 8192), (2, 240)])
def test_net_forward_matches_oracle(ns, J):
    th = _theta(1).astype(np.float32)
    xin = _xin(ns, J, 2).astype(np.float32)
    y = ipfb.net_forward(cuda(th), cuda(xin)).cpu().numpy().astype(np.float64)
    ref = onet.forward(onet.unflatten(th.astype(np.float64)), xin.astype(np.float64), emulate_bf16=True)
    assert y.shape == ref.shape
    assert _rel(y, ref) <= 5e-3, _rel(y, ref)
    # every position computed (ragged last tile, wrap-around halos)
    assert np.all(np.abs(y - ref) <= 0.05 * np.abs(ref).max())


def test_zero_output_layer_gives_bias():
    th = _theta(3).astype(np.float32)
    p = onet.unflatten(th.astype(np.float64))
    p["w3"][:] = 0.0
    p["b3"][:] = 0.25
    th = onet.flatten(p).astype(np.float32)
    y = ipfb.net_forward(cuda(th), cuda(_xin(2, 300, 4).astype(np.float32))).cpu().numpy()
    assert np.all(y == np.float32(0.25))


@pytest.mark.parametrize("ns,J", [(2, 300), (1, 100), (3, 448)])
def test_net_grad_matches_oracle(ns, J):
    th = _theta(5, scale3=1.0).astype(np.float32)
    xin = _xin(ns, J, 6).astype(np.float32)
    tgt = np.random.default_rng(7).standard_normal((ns, J)).astype(np.float32)
    loss, grad = ipfb.net_grad(cuda(th), cuda(xin), cuda(tgt))
    loss = float(loss.cpu().numpy()[0])
    grad = grad.cpu().numpy().astype(np.float64)
    L, g = onet.loss_and_grad(onet.unflatten(th.astype(np.float64)), xin.astype(np.float64),
                              tgt.astype(np.float64), emulate_bf16=True)
    assert abs(loss - L) <= 5e-3 * abs(L), (loss, L)
    gu = onet.unflatten(grad)
    for k in ("w1", "b1", "w2", "b2", "w3", "b3"):
        assert _rel(gu[k], g[k]) <= 1e-2, (k, _rel(gu[k], g[k]))


def test_net_grad_is_deterministic():
    th = cuda(_theta(8).astype(np.float32))
    xin = cuda(_xin(4, 700, 9).astype(np.float32))
    tgt = cuda(np.random.default_rng(10).standard_normal((4, 700)).astype(np.float32))
    l1, g1 = ipfb.net_grad(th, xin, tgt)
    l2, g2 = ipfb.net_grad(th, xin, tgt)
    assert torch.equal(l1, l2) and torch.equal(g1, g2)


def test_adam_matches_oracle():
    rng = np.random.default_rng(11)
    n = ipfb.NET_NPARAMS
    th0 = rng.standard_normal(n)
    grads = [rng.standard_normal(n) for _ in range(3)]
    th = cuda(th0.astype(np.float32))
    m = torch.zeros(n, dtype=torch.float32, device="cuda")
    v = torch.zeros(n, dtype=torch.float32, device="cuda")
    opt = onet.Adam(n, lr=1e-2)
    ref = th0.astype(np.float32).astype(np.float64)
    for k, gk in enumerate(grads):
        g32 = gk.astype(np.float32)
        ipfb.net_adam(th, m, v, cuda(g32), step=k + 1, lr=1e-2)
        ref = opt.step(ref, g32.astype(np.float64))
    out = th.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(out - ref)) <= 1e-5


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


def test_training_pairs_match_oracle():
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 21)
    w32 = cuda(w.astype(np.float32))
    xs, _, _ = ipfb.ml_solve(cuda(codes), cuda(scale), w32, sig2, cuda(mask), cuda(prior), precond="wiener",
                             tol=1e-6, max_iter=500)
    xk, _, _ = ipfb.ml_solve(cuda(codes), cuda(scale), w32, sig2, cuda(mask), cuda(prior), precond="wiener",
                             tol=0.0, max_iter=2)
    pairs = np.array([N // 4, 0, N // 2 - 1, 5], dtype=np.int32)
    xin, tgt = ipfb.ml_training_pairs(w32, sig2, cuda(mask), xs, xk, pairs)
    xin = xin.cpu().numpy().astype(np.float64)
    tgt = tgt.cpu().numpy().astype(np.float64)
    Xs = xs.cpu().numpy().reshape(J, N).astype(np.float64)
    Xk = xk.cpu().numpy().reshape(J, N).astype(np.float64)
    M = mask.reshape(J, N).astype(np.float64)
    cols = np.stack([2 * pairs, 2 * pairs + 1], axis=1).reshape(-1)
    E = (Xs - Xk)[:, cols]
    A = lambda V: oml.normal_operator_fft(w[:, cols], V, sig2, M[:, cols], 1.0)  # noqa: E731
    U = oml.wiener_precond(w[:, cols], A(E), sig2, M[:, cols], 1.0)
    ref_in, s = onet.net_input(U, M[:, cols])
    ref_t = ((E - U) / s).T
    assert np.array_equal(xin[:, 1], ref_in[:, 1])
    for c in range(len(cols)):
        assert _rel(xin[c, 0], ref_in[c, 0]) <= 1e-4, c
        assert np.max(np.abs(tgt[c] - ref_t[c])) <= 1e-4 * np.sqrt(np.mean((E[:, c] / s[c]) ** 2)), c


def _oracle_precond(pr, Mw, M, lam_mbar, net_from):
    """The learned preconditioner of the oracle FCG, with the net joining from the
    net_from-th application (the earlier ones are the Wiener step alone)."""
    calls = [0]

    def pre(R):
        k = calls[0]
        calls[0] += 1
        u = Mw(R)
        return u if k < net_from else onet.apply_precond(pr, u, M, Mw, lam_mbar, emulate_bf16=True)
    return pre


@pytest.mark.parametrize("net_from", [0, 2])
def test_learned_with_zero_net_is_wiener_pcg(net_from):
    """A zero-output net leaves the Wiener term alone: the learned solve is Wiener-PCG
    (with net_from >= 1 its first iterations run in the on-chip CG kernel, which hands
    its state over to the flexible-CG kernels)."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 22)
    p = onet.unflatten(_theta(23))
    p["w3"][:] = 0.0
    p["b3"][:] = 0.0
    th = cuda(onet.flatten(p).astype(np.float32))
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    xw, itw, rw = ipfb.ml_solve(*args, precond="wiener", tol=1e-6, max_iter=500)
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=500, net_from=net_from)
    itw, itl = itw.cpu().numpy(), itl.cpu().numpy()
    assert np.all(np.abs(itw - itl) <= 1), np.abs(itw - itl).max()
    assert np.all(rl.cpu().numpy()[0] <= 1e-6)
    assert _rel(xl.cpu().numpy(), xw.cpu().numpy()) <= 1e-4


@pytest.mark.parametrize("max_iter", [0, 3, 500])
def test_learned_net_never_joining_is_wiener_pcg_bit_for_bit(max_iter):
    """With net_from beyond the iterations any column takes (or beyond max_iter), the
    learned solve never asks the net: every iteration runs in the on-chip CG kernel,
    whose state goes through the hand-over, the flexible-CG finish and back to time
    order.  Solution, iterations and both residuals equal Wiener-PCG's bit for bit."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 32)
    th = cuda(_theta(33, scale3=0.2, jitter=0.01).astype(np.float32))
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    xw, itw, rw = ipfb.ml_solve(*args, precond="wiener", tol=1e-6, max_iter=max_iter)
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=max_iter, net_from=1000)
    assert torch.equal(itl, itw), (itl.max(), itw.max())
    assert torch.equal(xl, xw)
    assert torch.equal(rl, rw)


@pytest.mark.parametrize("N,J,net_from", [(64, 128, 0), (64, 512, 0), (64, 512, 3), (64, 1024, 1)])
def test_learned_fcg_matches_oracle(N, J, net_from):
    """Learned FCG against the oracle's FCG with the BF16-emulating net; with
    net_from >= 1 the Wiener-only iterations run on chip and are handed over."""
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 24)
    th = _theta(25, scale3=0.2, jitter=0.01)
    tol = 1e-6
    xl, itl, rl = ipfb.ml_solve(cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask),
                                cuda(prior), precond="learned", net=cuda(th.astype(np.float32)), tol=tol,
                                max_iter=2000, net_from=net_from)
    xl = xl.cpu().numpy().reshape(J, N).astype(np.float64)
    itl, rl = itl.cpu().numpy(), rl.cpu().numpy()
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)
    A = lambda V: oml.normal_operator_fft(w, V, sig2, M, 1.0)  # noqa: E731
    B = oml.rhs(w, d, sig2, M, P, 1.0)
    pr = onet.unflatten(th.astype(np.float32).astype(np.float64))
    lam_mbar = 1.0 * M.mean(axis=0)
    Mw = lambda R: oml.wiener_precond(w, R, sig2, M, 1.0)  # noqa: E731
    pre = _oracle_precond(pr, Mw, M, lam_mbar, net_from)
    Xo, ito, _ = onet.fcg(A, B, np.zeros_like(B), pre, tol, 2000)
    assert np.all(rl[0] <= tol)
    tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, xl)
    assert np.all(tr <= 5 * tol), tr.max()
    assert np.all(np.abs(itl - ito) <= np.maximum(3, 0.25 * ito)), (itl, ito)
    # the same reconstruction as the oracle's solve (both at tol)
    xt = x.reshape(J, N)
    e_gpu = np.linalg.norm(xl - xt) / np.linalg.norm(xt)
    e_or = np.linalg.norm(Xo - xt) / np.linalg.norm(xt)
    assert abs(e_gpu - e_or) <= 1e-3 * e_or


@pytest.mark.parametrize("net_from", [0, 2])
def test_learned_initial_guess(net_from):
    """x0 enters in frame order and the solution leaves in frame order: with no
    iteration the output is x0 bit for bit; from x0 the learned FCG reaches the same
    reconstruction as the oracle's FCG started from the same x0 (net_from >= 1: through
    the on-chip Wiener iterations and the hand-over)."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 27)
    th = _theta(28, scale3=0.2, jitter=0.01)
    rng = np.random.default_rng(29)
    x0 = (x + 0.3 * rng.standard_normal(x.shape)).astype(np.float32)
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    x_same, it0, _ = ipfb.ml_solve(*args, precond="learned", net=cuda(th.astype(np.float32)), tol=1e-6,
                                   max_iter=0, x0=cuda(x0), net_from=net_from)
    assert np.array_equal(x_same.cpu().numpy(), x0)
    assert np.all(it0.cpu().numpy() == 0)
    tol = 1e-6
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=cuda(th.astype(np.float32)), tol=tol,
                                max_iter=2000, x0=cuda(x0), net_from=net_from)
    xl = xl.cpu().numpy().reshape(J, N).astype(np.float64)
    itl, rl = itl.cpu().numpy(), rl.cpu().numpy()
    M = mask.reshape(J, N).astype(np.float64)
    P = prior.reshape(J, N).astype(np.float64)
    A = lambda V: oml.normal_operator_fft(w, V, sig2, M, 1.0)  # noqa: E731
    B = oml.rhs(w, d, sig2, M, P, 1.0)
    pr = onet.unflatten(th.astype(np.float32).astype(np.float64))
    lam_mbar = 1.0 * M.mean(axis=0)
    Mw = lambda R: oml.wiener_precond(w, R, sig2, M, 1.0)  # noqa: E731
    pre = _oracle_precond(pr, Mw, M, lam_mbar, net_from)
    Xo, ito, _ = onet.fcg(A, B, x0.reshape(J, N).astype(np.float64), pre, tol, 2000)
    assert np.all(rl[0] <= tol)
    tr = oml.true_relative_residual(d, w, sig2, M, P, 1.0, xl)
    assert np.all(tr <= 5 * tol), tr.max()
    assert np.all(np.abs(itl - ito) <= np.maximum(3, 0.25 * ito)), (itl, ito)
    xt = x.reshape(J, N)
    e_gpu = np.linalg.norm(xl - xt) / np.linalg.norm(xt)
    e_or = np.linalg.norm(Xo - xt) / np.linalg.norm(xt)
    assert abs(e_gpu - e_or) <= 1e-3 * e_or


def test_learned_nonfinite_net_falls_back_to_plain_cg():
    """A net that returns NaN: flexible CG ends with non-finite residuals, and the call
    hands back plain CG's solve from the same start, bit for bit."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 30)
    th = _theta(31).astype(np.float32)
    th[:] = np.nan
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    xp, itp, rp = ipfb.ml_solve(*args, precond="none", tol=1e-6, max_iter=500)
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=cuda(th), tol=1e-6, max_iter=500)
    assert torch.equal(xl, xp) and torch.equal(itl, itp) and torch.equal(rl, rp)
    assert bool(torch.isfinite(xl).all())


def test_learned_requires_net_and_ntap4():
    N, J = 64, 128
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 26)
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    with pytest.raises(ValueError):
        ipfb.ml_solve(*args, precond="learned", net=None)
    L = ipfb.lib()
    g = ipfb.geom(N, 8, J)
    n = ipfb.ctypes.c_size_t(0)
    assert L.ipfb_workspace_size(ipfb.ctypes.byref(g), ipfb.OP_ML_LEARNED, ipfb.ctypes.byref(n)) == \
        ipfb.ERR_UNSUPPORTED


def test_learned_fullsize_config4_properties():
    """lblock 4096, ntap 4, 8192 spectra, 10 % prior: the learned FCG (an untrained,
    small-output net) reaches the per-column tolerance, the true residual recomputed
    from its final x stays within 5x of it, and it reconstructs the stream as well as
    Wiener-PCG (same system, same tolerance: errors equal within 1e-3 relative)."""
    from paper_2608_23441_b300 import precond_train as pt
    dev = torch.device("cuda", 0)
    inst = pt.instance(torch, dev, 4, fraction=0.1)
    args = (inst["codes"], inst["scale"], inst["w"], inst["sig2"], inst["mask"], inst["x"])
    th = cuda(_theta(31, scale3=0.1, jitter=0.0).astype(np.float32))
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=4000)
    xw, itw, rw = ipfb.ml_solve(*args, precond="wiener", tol=1e-6, max_iter=4000)
    rl = rl.cpu().numpy()
    assert np.all(rl[0] <= 1e-6)
    assert np.all(rl[1] <= 5e-6), rl[1].max()
    x = inst["x"]
    el = float(torch.linalg.norm(xl - x) / torch.linalg.norm(x))
    ew = float(torch.linalg.norm(xw - x) / torch.linalg.norm(x))
    assert abs(el - ew) <= 1e-3 * ew, (el, ew)
    assert int(itl.max()) < 4000


def test_trained_net_gain_over_its_zero_output_form():
    """What the trained net gains over the method without it.  Trained on plain-CG
    iterates of seeds 1000-1007 (the benchmark's training recipe), the learned solve of
    a held-out lblock-4096, 8192-spectrum instance (seed 4, 10 % prior in 64 chunks),
    with the net joining from the third preconditioner application, reaches 1e-6 per
    column in fewer iterations than the same solve with a zero-output net (g = 0, i.e.
    the Wiener preconditioner) and than Wiener-PCG itself: a lower worst-column count
    (by 4 or more), a lower mean, at least 15 % fewer iterations over the slow columns
    (those Wiener-PCG needs 10 or more for), and the same reconstruction error within
    1e-3 relative.  With the net joining late (the default net_from, where the learned
    solve is faster than plain CG) it still lowers the worst column and the mean
    against its zero-output form."""
    from paper_2608_23441_b300 import precond_train as pt
    dev = torch.device("cuda", 0)
    xin, tgt, _ = pt.make_training_set(torch, dev, list(range(1000, 1008)))
    theta, hist = pt.train(torch, dev, xin, tgt, epochs=pt.EPOCHS)
    assert hist[-1] < hist[0], hist
    del xin, tgt
    N, J = 4096, 8192
    x = torch.from_numpy(synth.stream_config(N, J, 4).astype(np.float32)).to(dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(N, 4)).to(dev)
    codes, scale, _ = ipfb.pfb_forward(x, w)
    starts, L = synth.prior_chunks(N * J, 64, 0.1, 4)
    mask = torch.from_numpy(synth.mask_from_chunks(N * J, starts, L)).to(dev)
    sig2 = pt.noise_var(torch, ipfb, codes, scale, w, x, N, J)
    args = (codes, scale, w, sig2, mask, x)
    zero = torch.from_numpy(pt.init_theta(0, scale3=0.0)).to(dev)
    xw, itw, rw = ipfb.ml_solve(*args, precond="wiener", tol=1e-6, max_iter=4000)
    nf = pt.NET_FROM_EARLY
    x0, it0, r0 = ipfb.ml_solve(*args, precond="learned", net=zero, tol=1e-6, max_iter=4000, net_from=nf)
    xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=theta, tol=1e-6, max_iter=4000, net_from=nf)
    for r in (rw, r0, rl):
        assert bool((r[0] <= 1e-6).all())
    itw, it0, itl = itw.cpu().numpy(), it0.cpu().numpy(), itl.cpu().numpy()
    slow = itw >= 10
    print(f"worst column: learned {itl.max()}, g = 0 {it0.max()}, Wiener-PCG {itw.max()}; mean {itl.mean():.3f}, "
          f"{it0.mean():.3f}, {itw.mean():.3f}; slow columns ({slow.sum()}) {itl[slow].sum()}, {it0[slow].sum()}, "
          f"{itw[slow].sum()}")
    for ref in (it0, itw):
        assert itl.max() + 4 <= ref.max(), (itl.max(), ref.max())
        assert itl.mean() < ref.mean(), (itl.mean(), ref.mean())
        assert itl[slow].sum() <= 0.85 * ref[slow].sum(), (itl[slow].sum(), ref[slow].sum())
    ew = float(torch.linalg.norm(xw - x) / torch.linalg.norm(x))
    el = float(torch.linalg.norm(xl - x) / torch.linalg.norm(x))
    assert abs(el - ew) <= 1e-3 * ew, (el, ew)
    # the net joining late
    _, it0l, r0l = ipfb.ml_solve(*args, precond="learned", net=zero, tol=1e-6, max_iter=4000, net_from=pt.NET_FROM)
    xll, itll, rll = ipfb.ml_solve(*args, precond="learned", net=theta, tol=1e-6, max_iter=4000,
                                   net_from=pt.NET_FROM)
    assert bool((rll[0] <= 1e-6).all()) and bool((r0l[0] <= 1e-6).all())
    it0l, itll = it0l.cpu().numpy(), itll.cpu().numpy()
    print(f"net from application {pt.NET_FROM + 1}: worst column {itll.max()} against {it0l.max()}, "
          f"mean {itll.mean():.4f} against {it0l.mean():.4f}")
    assert itll.max() < it0l.max() and itll.mean() < it0l.mean(), (itll.max(), it0l.max())
    ell = float(torch.linalg.norm(xll - x) / torch.linalg.norm(x))
    assert abs(ell - ew) <= 1e-3 * ew, (ell, ew)


def test_training_resumes_exactly_from_a_checkpoint(tmp_path):
    """Two epochs, a checkpoint written and read back, two more epochs: the same
    parameters, bit for bit, as four epochs in one run (Adam moments, step count and
    batch order all restored)."""
    from paper_2608_23441_b300 import precond_train as pt
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(41)
    xin = cuda(_xin(64, 512, 42).astype(np.float32))
    tgt = cuda(rng.standard_normal((64, 512)).astype(np.float32))
    th4, h4 = pt.train(torch, dev, xin, tgt, epochs=4, batch=16, seed=3)
    th2, h2, st = pt.train(torch, dev, xin, tgt, epochs=2, batch=16, seed=3, return_state=True)
    p = str(tmp_path / "net.ckpt")
    pt.save_checkpoint(p, st["theta"], st["m"], st["v"], step=st["step"], rng_state=st["rng"])
    thr, hr = pt.train(torch, dev, xin, tgt, epochs=2, batch=16, state=pt.load_checkpoint(p))
    assert torch.equal(thr, th4)
    assert h2 + hr == h4


def test_learned_solve_enqueues_without_host_sync():
    """The learned solve is one graph whose loop ends on the device: it can be
    recorded inside a caller's CUDA-graph capture (any host synchronisation or
    read-back would break the capture), and replaying the captured graph gives the
    eager call's answer bit for bit."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 33)
    th = cuda(_theta(34, scale3=0.2, jitter=0.01).astype(np.float32))
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    g = ipfb.geom(N, 4, J)
    ws = torch.empty(ipfb.workspace_size(g, ipfb.OP_ML_LEARNED), dtype=torch.uint8, device="cuda")
    xe, ite, re = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=500, workspace=ws)
    xe, ite, re = xe.clone(), ite.clone(), re.clone()
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            xg, itg, rg = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=500, workspace=ws)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        xg.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(xg, xe) and torch.equal(itg, ite) and torch.equal(rg, re)


def test_net_wait_that_runs_out_falls_back_to_plain_cg():
    """A bounded device wait that expires (failure detection without a fault): with the
    net forward's accumulator wait bound set to zero, every CTA gives up at once, marks
    its output, lets its MMAs in flight finish and stops; the learned solve sees the
    give-up on the device and returns plain CG's solve from the same start, bit for bit.
    The standalone forward shows the mark (NaN) in its output.  The bound is restored."""
    N, J = 64, 256
    x, w, codes, scale, d, sig2, mask, prior = _instance(N, J, 35)
    th = cuda(_theta(36, scale3=0.2, jitter=0.01).astype(np.float32))
    args = (cuda(codes), cuda(scale), cuda(w.astype(np.float32)), sig2, cuda(mask), cuda(prior))
    xp, itp, rp = ipfb.ml_solve(*args, precond="none", tol=1e-6, max_iter=500)
    xin = cuda(_xin(3, 500, 37).astype(np.float32))
    ipfb.set_net_wait_limit(0)
    try:
        xl, itl, rl = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=500)
        y = ipfb.net_forward(th, xin)
        torch.cuda.synchronize()
    finally:
        ipfb.set_net_wait_limit(-1)
    assert torch.equal(xl, xp) and torch.equal(itl, itp) and torch.equal(rl, rp)
    assert not bool(torch.isfinite(y).all())
    # the bound restored: the same calls work normally again
    xl2, itl2, rl2 = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=500)
    y2 = ipfb.net_forward(th, xin)
    assert bool(torch.isfinite(y2).all()) and bool((rl2[0] <= 1e-6).all())


def test_learned_solve_returns_before_the_device_finishes():
    """The learned solve enqueues its graph and returns: on a config-4 instance (device
    time ~10 ms) the call's host time is a small fraction of the device time, also on
    later calls (a launched graph is released only once it has finished, by a later call,
    never by waiting for it)."""
    import time
    from paper_2608_23441_b300 import precond_train as pt
    dev = torch.device("cuda", 0)
    inst = pt.instance(torch, dev, 4, fraction=0.1)
    args = (inst["codes"], inst["scale"], inst["w"], inst["sig2"], inst["mask"], inst["x"])
    th = torch.from_numpy(pt.init_theta(0, scale3=0.0)).to(dev)
    g = ipfb.geom(4096, 4, 8192)
    ws = torch.empty(ipfb.workspace_size(g, ipfb.OP_ML_LEARNED), dtype=torch.uint8, device=dev)
    ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=4000, workspace=ws)
    torch.cuda.synchronize()
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        t0 = time.perf_counter()
        x, it, r = ipfb.ml_solve(*args, precond="learned", net=th, tol=1e-6, max_iter=4000, workspace=ws)
        host_ms = 1e3 * (time.perf_counter() - t0)
        e1.record()
        torch.cuda.synchronize()
        dev_ms = e0.elapsed_time(e1)
        assert host_ms < 0.3 * dev_ms, (host_ms, dev_ms)
        assert bool((r[0] <= 1e-6).all())
