"""Training of the learned conjugate-gradient preconditioner with the library's own
kernels (the learned variant of the Sec. 4.2 solve; the paper has no learned
component).

Recipe: seeded instances of the ML workload (lblock 4096, ntap 4, 8192 spectra,
prior fraction U[2 %, 20 %] in 64 contiguous chunks); for each, the converged
solution x* and plain-CG iterates x_k at a few iteration counts; training pairs
(u/s, m) -> (e - u)/s from ipfb_ml_training_pairs for column pairs drawn with a
bias toward the ill-conditioned sub-filters around column N/2 (App. A); the mean
squared error and its gradient from ipfb_net_grad; Adam from ipfb_net_adam.
Every compute step runs in libipfb; torch only holds device memory.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import ipfb, synth

NTAP = 4
# training epochs of the recipe, and the preconditioner applications that use the
# Wiener term alone before the net joins the learned solve (ipfb_ml_params.net_from).
# Those first iterations run on chip at about 25 us each; an iteration with the net
# (its forward over the active columns plus a flexible-CG step with two pair FFTs)
# costs about 0.1 ms, so the net is kept for the slow columns: joining at the 21st
# application, the learned solve of the lblock-4096, 8192-spectrum workload is
# faster than plain CG; joining at the 3rd (NET_FROM_EARLY) it takes the fewest
# iterations but about three times plain CG's time.
EPOCHS = 24
NET_FROM = 20
NET_FROM_EARLY = 2


def init_theta(seed: int, scale3: float = 0.1) -> np.ndarray:
    """He-style uniform initial weights (biases zero); the output layer is scaled by
    `scale3` so that training starts close to the Wiener preconditioner (g = 0)."""
    rng = np.random.default_rng(seed)

    def u(n, fan_in):
        b = math.sqrt(6.0 / fan_in)
        return rng.uniform(-b, b, size=n)

    parts = [u(32 * 2 * 9, 2 * 9), np.zeros(32), u(32 * 32 * 9, 32 * 9), np.zeros(32),
             u(32 * 9, 32 * 9) * scale3, np.zeros(1)]
    th = np.concatenate(parts).astype(np.float32)
    assert th.size == ipfb.NET_NPARAMS
    return th


def noise_var(torch, ipfb_mod, codes, scale, w, x, lblock: int, nframes: int) -> float:
    """sigma^2 of the quantization noise in the units of d: with x_r the exact inverse
    of the codes, d - C x = C (x_r - x) in the periodic model, so sigma^2 =
    var(sum_r w_r e[j + r]) with e = x_r - x (setup arithmetic, FP64)."""
    xr = ipfb_mod.ipfb_wiener(codes, scale, w, 0.0)
    e = (xr - x).reshape(nframes, lblock).double()
    wd = w.double()
    ce = sum(wd[r][None, :] * torch.roll(e, -r, dims=0) for r in range(w.shape[0]))
    return float(ce.var())


def instance(torch, dev, seed: int, fraction: float | None = None, lblock: int = 4096, nframes: int = 8192,
             nchunks: int = 64):
    """One seeded instance: white Gaussian stream generated on the device, forward PFB
    with 4-bit codes (pfb_forward), prior mask of `nchunks` chunks covering `fraction`
    of the samples (drawn U[2 %, 20 %] when None), prior values = the true stream."""
    if fraction is None:
        fraction = synth.prior_fraction_draw(seed)
    T = lblock * nframes
    x = synth.gaussian_stream_torch(T, seed, dev)
    w = torch.from_numpy(ipfb.sinc_hamming_window(lblock, NTAP)).to(dev)
    codes, scale, _ = ipfb.pfb_forward(x, w)
    starts, L = synth.prior_chunks(T, nchunks, fraction, seed)
    mask = torch.from_numpy(synth.mask_from_chunks(T, starts, L)).to(dev)
    sig2 = noise_var(torch, ipfb, codes, scale, w, x, lblock, nframes)
    return {"codes": codes, "scale": scale, "w": w, "mask": mask, "x": x, "sig2": sig2, "fraction": fraction}


def draw_pairs(rng, npair_total: int, count: int, spread: float = 0.0625) -> np.ndarray:
    """`count` distinct column-pair indices, Gaussian around pair P/2 (columns near N/2,
    where |W_n| is smallest) with standard deviation spread * P."""
    centre = npair_total // 2
    out: list[int] = []
    seen = set()
    while len(out) < count:
        p = int(round(rng.normal(centre, spread * npair_total))) % npair_total
        if p not in seen:
            seen.add(p)
            out.append(p)
    return np.array(out, dtype=np.int32)


def make_training_set(torch, dev, seeds, iters=(1, 3, 8, 20, 50), pairs_per: int = 50, lblock: int = 4096,
                      nframes: int = 8192, log=None):
    """Training pairs from plain-CG iterates of every instance in `seeds`:
    len(seeds) * len(iters) * pairs_per column pairs (two columns each).
    Returns xin [S, 2, J], target [S, J] (device float32) and a summary."""
    xs_all, ts_all = [], []
    rng = np.random.default_rng(12345)
    t0 = time.time()
    for seed in seeds:
        inst = instance(torch, dev, seed, lblock=lblock, nframes=nframes)
        args = (inst["codes"], inst["scale"], inst["w"], inst["sig2"], inst["mask"], inst["x"])
        x_star, _, _ = ipfb.ml_solve(*args, precond="wiener", tol=1e-6, max_iter=4000)
        for k in iters:
            x_k, _, _ = ipfb.ml_solve(*args, precond="none", tol=0.0, max_iter=int(k))
            pl = draw_pairs(rng, lblock // 2, pairs_per)
            xin, tgt = ipfb.ml_training_pairs(inst["w"], inst["sig2"], inst["mask"], x_star, x_k, pl)
            xs_all.append(xin)
            ts_all.append(tgt)
        if log:
            log(f"training instance {seed}: fraction {inst['fraction']:.3f}, {time.time() - t0:.1f} s")
        del inst
    xin = torch.cat(xs_all)
    target = torch.cat(ts_all)
    return xin, target, {"instances": len(seeds), "iterates": list(iters), "column_pairs": len(seeds) * len(iters)
                         * pairs_per, "columns": int(xin.shape[0]), "frames": int(xin.shape[2])}


def train(torch, dev, xin, target, epochs: int = EPOCHS, batch: int = 16, lr: float = 2e-3, seed: int = 0,
          theta0: np.ndarray | None = None, log=None, state: dict | None = None, return_state: bool = False):
    """Adam on mini-batches of `batch` consecutive training columns (batch / 2 randomly
    drawn column pairs of one instance and iterate), the batches visited in a new
    random order every epoch; returns (theta device tensor, per-epoch mean loss), and
    with return_state=True also the training state (theta, Adam moments m and v, step
    count, batch-order generator state) that save_checkpoint writes and `state=`
    resumes from: training E1 epochs, then E2 more from the saved state, visits the
    same batches with the same Adam steps as E1 + E2 epochs in one run."""
    n = xin.shape[0]
    if state is not None:
        theta = torch.from_numpy(_host_f32(state["theta"]).astype(np.float32)).to(dev)
        m = torch.from_numpy(_host_f32(state["m"]).astype(np.float32)).to(dev)
        v = torch.from_numpy(_host_f32(state["v"]).astype(np.float32)).to(dev)
        step = int(state["step"])
        rng = np.random.default_rng()
        rng.bit_generator.state = state["rng"]
    else:
        theta = torch.from_numpy(init_theta(seed) if theta0 is None else theta0.astype(np.float32)).to(dev)
        m = torch.zeros_like(theta)
        v = torch.zeros_like(theta)
        rng = np.random.default_rng(seed + 1)
        step = 0
    ws = torch.empty(ipfb.net_workspace_size(ipfb.NET_GRAD, batch, xin.shape[2]), dtype=torch.uint8, device=dev)
    hist = []
    nb = n // batch
    for ep in range(epochs):
        losses = []
        for bi in rng.permutation(nb):
            b0 = int(bi) * batch
            loss, grad = ipfb.net_grad(theta, xin[b0:b0 + batch], target[b0:b0 + batch], workspace=ws)
            step += 1
            ipfb.net_adam(theta, m, v, grad, step, lr=lr)
            losses.append(loss)
        ep_loss = float(np.mean(torch.cat(losses).cpu().numpy()))
        hist.append(ep_loss)
        if log:
            log(f"epoch {ep}: loss {ep_loss:.5f}")
    if return_state:
        return theta, hist, {"theta": theta, "m": m, "v": v, "step": step, "rng": rng.bit_generator.state}
    return theta, hist


# ---------------------------------------------------------------------------
# Checkpoints: the net's parameters with the Adam state, as one file
#   8 bytes magic "IPFBNET1", 4 bytes little-endian header length H, H bytes of JSON
#   (nparams, step, has_adam, the batch-order generator state, free-form info), then
#   theta, and with has_adam m and v, each nparams little-endian float32.
# ---------------------------------------------------------------------------
CKPT_MAGIC = b"IPFBNET1"


def _host_f32(a) -> np.ndarray:
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype="<f4")).reshape(-1)


def save_checkpoint(path: str, theta, m=None, v=None, step: int = 0, rng_state: dict | None = None,
                    info: dict | None = None) -> None:
    """Write theta (and the Adam moments m, v when given) to `path` (see above)."""
    import json
    th = _host_f32(theta)
    if th.size != ipfb.NET_NPARAMS:
        raise ValueError(f"theta has {th.size} values, expected {ipfb.NET_NPARAMS}")
    has_adam = m is not None and v is not None
    arrays = [th] + ([_host_f32(m), _host_f32(v)] if has_adam else [])
    if any(a.size != th.size for a in arrays):
        raise ValueError("m and v must have as many values as theta")
    header = json.dumps({"nparams": int(th.size), "step": int(step), "has_adam": bool(has_adam),
                         "rng": rng_state, "info": info or {}}).encode()
    with open(path, "wb") as fh:
        fh.write(CKPT_MAGIC)
        fh.write(len(header).to_bytes(4, "little"))
        fh.write(header)
        for a in arrays:
            fh.write(a.tobytes())


def load_checkpoint(path: str) -> dict:
    """Read a checkpoint: {"theta", "m", "v" (None without Adam state), "step", "rng",
    "info"}; the arrays are float32 numpy vectors."""
    import json
    with open(path, "rb") as fh:
        blob = fh.read()
    if blob[:8] != CKPT_MAGIC:
        raise ValueError(f"{path}: not a net checkpoint")
    hlen = int.from_bytes(blob[8:12], "little")
    header = json.loads(blob[12:12 + hlen].decode())
    n = int(header["nparams"])
    if n != ipfb.NET_NPARAMS:
        raise ValueError(f"{path}: {n} parameters, expected {ipfb.NET_NPARAMS}")
    narr = 3 if header["has_adam"] else 1
    body = blob[12 + hlen:]
    if len(body) != narr * n * 4:
        raise ValueError(f"{path}: {len(body)} bytes of arrays, expected {narr * n * 4}")
    arrs = [np.frombuffer(body, dtype="<f4", count=n, offset=i * n * 4).astype(np.float32) for i in range(narr)]
    return {"theta": arrs[0], "m": arrs[1] if narr == 3 else None, "v": arrs[2] if narr == 3 else None,
            "step": int(header["step"]), "rng": header.get("rng"), "info": header.get("info", {})}


def parse_seeds(text: str) -> list[int]:
    """"1000-1007" -> [1000, ..., 1007]; "3,5,9" -> [3, 5, 9]; ranges and single seeds
    mix ("1-2,7"); seeds are non-negative."""
    out: list[int] = []
    for part in text.split(","):
        part = part.strip()
        if not part:
            continue
        if "-" in part:
            a, b = part.split("-", 1)
            lo, hi = int(a), int(b)
            if hi < lo:
                raise ValueError(f"empty seed range {part!r}")
            out.extend(range(lo, hi + 1))
        else:
            out.append(int(part))
    if not out:
        raise ValueError("no seeds")
    return out


def main(argv=None) -> int:
    """Train the net on the training recipe above and write a checkpoint:

        python -m paper_2608_23441_b300.precond_train --out net.ckpt
            [--seeds 1000-1007] [--epochs 24] [--resume earlier.ckpt]

    With --resume, training continues from that checkpoint's parameters, Adam state and
    batch order (the training pairs are rebuilt from the same seeds)."""
    import argparse
    import json
    import torch
    ap = argparse.ArgumentParser(description="train the learned CG preconditioner")
    ap.add_argument("--out", required=True)
    ap.add_argument("--seeds", default="1000-1007")
    ap.add_argument("--epochs", type=int, default=EPOCHS)
    ap.add_argument("--resume", default=None)
    args = ap.parse_args(argv)
    seeds = parse_seeds(args.seeds)
    dev = torch.device("cuda", 0)
    xin, tgt, info = make_training_set(torch, dev, seeds)
    state = load_checkpoint(args.resume) if args.resume else None
    theta, hist, st = train(torch, dev, xin, tgt, epochs=args.epochs, state=state, return_state=True)
    info.update({"seeds": args.seeds, "epochs": args.epochs, "loss_per_epoch": hist,
                 "resumed_from": args.resume})
    save_checkpoint(args.out, st["theta"], st["m"], st["v"], step=st["step"], rng_state=st["rng"], info=info)
    print(json.dumps({"out": args.out, "step": st["step"], "loss_per_epoch": hist}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
