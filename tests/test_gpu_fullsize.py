"""GPU parity at the benchmark's full sizes, in the launch configurations the
benchmark times, on outputs the FP64 oracle can evaluate one by one, plus
properties that hold at any size.

- Pipeline (lblock 4096, ntap 4, 65536 spectra, upfactor 64; the J = 65536 column
  transform runs on 8-CTA clusters and the 262144-sample up-channelizer on 16-CTA
  clusters): sampled reconstructed columns against the oracle's column-wise inverse
  (Eq. decorrelation, Eq. wiener weights) at 1e-4; sampled up-channelized blocks
  against an FP64 real DFT of the reconstructed stream at 1e-5; Parseval on every
  block.
- Batched (256 uneven streams, the benchmark's shapes): sampled streams against
  the oracle's per-stream inverse at 1e-4."""
import numpy as np
import pytest

from oracle import ipfb as oipfb
from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402


def relrms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


def test_config2_pipeline_sampled_columns_and_blocks():
    N, J, U, phi2 = 4096, 65536, 64, 0.0141
    ipfb.set_max_column_run(8192)
    codes = synth.random_code_bytes(J, N // 2, 51)
    scale = synth.random_scale(N // 2 + 1, 52)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
    out, xo = ipfb.ipfb_wiener_upchannelize(torch.from_numpy(codes).cuda(), torch.from_numpy(scale).cuda(),
                                            torch.from_numpy(w).cuda(), phi2, U, want_x=True)
    torch.cuda.synchronize()
    L = U * N
    nb = J * N // L
    assert tuple(out.shape) == (nb, L // 2 + 1)
    # sampled columns of the reconstruction (edge columns, the worst-conditioned
    # column N/2, and a few seeded ones)
    rng = np.random.default_rng(53)
    cols = [0, 1, N // 2 - 1, N // 2, N - 1] + [int(c) for c in rng.integers(2, N - 2, size=3)]
    ref = oipfb.ipfb_columns(codes, scale, w.astype(np.float64), cols, phi2)
    got = xo.reshape(J, N)[:, cols].cpu().numpy()
    for i, c in enumerate(cols):
        assert relrms(got[:, i], ref[:, i]) < 1e-4, c
    # sampled blocks of the up-channelizer against an FP64 real DFT of the GPU stream
    for b in (0, nb // 2, nb - 1):
        seg = xo[b * L:(b + 1) * L].double().cpu().numpy()
        refb = np.fft.rfft(seg)
        gb = out[b].cpu().numpy().astype(np.complex128)
        assert np.sqrt(np.mean(np.abs(gb - refb) ** 2) / np.mean(np.abs(refb) ** 2)) < 1e-5, b
    # Parseval on every block: sum_k c_k |X_k|^2 = L sum_t x_t^2 (c = 1 at DC and
    # Nyquist, 2 elsewhere)
    X = out.to(torch.complex128)
    e_f = 2.0 * (X.abs() ** 2).sum(dim=1) - (X[:, 0].abs() ** 2) - (X[:, -1].abs() ** 2)
    e_t = L * (xo.double().reshape(nb, L) ** 2).sum(dim=1)
    assert float(((e_f - e_t).abs() / e_t).max()) < 1e-5


def test_config3_batched_sampled_streams():
    geoms = synth.batched_geometries(256, 3)
    dev = torch.device("cuda", 0)
    streams = []
    for i, (N, J) in enumerate(geoms):
        x = synth.gaussian_stream_torch(N * J, 3 * 100003 + i, dev)
        w = torch.from_numpy(ipfb.sinc_hamming_window(N, 4)).to(dev)
        codes, scale, _ = ipfb.pfb_forward(x, w)
        del x
        streams.append({"codes": codes, "scale": scale, "window": w, "noise_level": 0.0141})
    plan = ipfb.BatchedPlan(streams)
    plan.prepare()
    xs = plan.run()
    torch.cuda.synchronize()
    # the smallest streams of each lblock, one with odd J, and the largest J among
    # streams small enough for the FP64 oracle
    sizes = [N * J for N, J in geoms]
    order = np.argsort(sizes)
    picks = set(int(i) for i in order[:3])
    picks.add(int(next(i for i in order if geoms[i][1] % 2 == 1)))
    for lb in (1024, 2048, 4096):
        picks.add(int(next(i for i in order if geoms[i][0] == lb)))
    for i in sorted(picks):
        N, J = geoms[i]
        st = streams[i]
        ref = oipfb.ipfb_wiener(st["codes"].cpu().numpy(), st["scale"].cpu().numpy(),
                                st["window"].cpu().numpy().astype(np.float64), 0.0141)
        assert relrms(xs[i].cpu().numpy(), ref) < 1e-4, (i, N, J)
    plan.close()
