"""GPU parity of the batched inverse PFB (many uneven streams, any integer number
of frames via Bluestein column transforms) against the FP64 oracle, run stream by
stream.  Tolerance: the Wiener relative RMS 1e-4 of the single-stream tests; the
Bluestein path adds two length-M FFT round trips (M < 4J), still ~1e-6."""
import os
import tempfile

import numpy as np
import pytest

from oracle import batched as obatched
from oracle import ipfb as oipfb
from oracle import pfb as opfb
from paper_2608_23441_b300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2608_23441_b300 import ipfb  # noqa: E402

SHAPES = [(1024, 1031), (2048, 1500), (4096, 1024), (1024, 2310), (2048, 4099), (1024, 1024), (4096, 1111),
          (2048, 3000), (1024, 8191)]


# column-kernel variants (cluster size, threads, largest radix) and their cluster sizes
VARIANTS = {"c4_t256_r32": 4, "c4_t256_r16": 4, "c2_t256_r32": 2, "c8_t256_r32": 8, "c1_t512_r32": 1,
            "c2_ts16_r32": 2, "c4_ts16_r32": 4, "c2_t512_r32": 2, "c1_ts16_r32": 1, "c1_t256_r32": 1,
            "c1_t1024_r32": 1, "c2_t1024_r32": 2}


def _in_range(M, C, name=""):
    # a CTA of a cluster holds up to 8192 elements, a single CTA up to 16384; the
    # "ts16" variants (S / 16 threads) serve S = 512 .. 2048
    if name == "c1_ts16_r32":
        return 2048 <= M <= 4096
    if name == "c1_t256_r32":
        return M == 8192
    if name.endswith("t1024_r32"):
        return M // C == 16384
    if "ts16" in name:
        return 512 <= M // C <= 2048
    if name == "c2_t512_r32":
        return M // C == 16384
    return 512 <= M // C <= (16384 if C == 1 else 8192)


def relrms(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.sqrt(np.mean((a - b) ** 2) / np.mean(b ** 2)))


def _streams(shapes, seed0):
    out, host = [], []
    for i, (N, J) in enumerate(shapes):
        codes = synth.random_code_bytes(J, N // 2, seed0 + i)
        scale = synth.random_scale(N // 2 + 1, seed0 + 100 + i)
        w = opfb.sinc_hamming_window(N, 4).astype(np.float32)
        nl = 0.01 + 0.001 * i
        out.append({"codes": torch.from_numpy(codes).cuda(), "scale": torch.from_numpy(scale).cuda(),
                    "window": torch.from_numpy(w).cuda(), "noise_level": nl})
        host.append((codes, scale, w.astype(np.float64), nl))
    return out, host


def test_batched_matches_oracle_per_stream():
    streams, host = _streams(SHAPES, 300)
    plan = ipfb.BatchedPlan(streams)
    xs = plan.run()
    torch.cuda.synchronize()
    refs = obatched.ipfb_batched(host)
    for (N, J), x, ref in zip(SHAPES, xs, refs):
        assert relrms(x.cpu().numpy(), ref) < 1e-4, (N, J)
    plan.close()


def test_batched_autotune_cache_and_graph_replay():
    shapes = SHAPES[:5]
    streams, host = _streams(shapes, 400)
    plan = ipfb.BatchedPlan(streams)
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.txt")
        plan.autotune(cache)
        assert os.path.exists(cache)
        lines = open(cache).read().split()
        assert len(lines) == 10
        names = {plan.variant(2048 << c) for c in range(5)}
        assert names <= set(VARIANTS)
        # a plan that loads the cache picks the same variants
        plan2 = ipfb.BatchedPlan(streams, tune_cache=cache)
        for c in range(5):
            assert plan2.variant(2048 << c) == plan.variant(2048 << c)
        plan2.close()
    refs = obatched.ipfb_batched(host)
    plan.prepare()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    torch.cuda.current_stream().wait_stream(s)
    for x in plan.x:
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    for (N, J), x, ref in zip(shapes, plan.x, refs):
        assert relrms(x.cpu().numpy(), ref) < 1e-4, (N, J)
    g.replay()
    torch.cuda.synchronize()
    for (N, J), x, ref in zip(shapes, plan.x, refs):
        assert relrms(x.cpu().numpy(), ref) < 1e-4, (N, J)
    plan.close()


@pytest.mark.parametrize("name", sorted(VARIANTS))
def test_batched_each_variant_matches_oracle(name):
    # one stream per Bluestein length class M = 4096 .. 32768, every class forced to
    # `name` through a tune cache (classes outside the variant's range, M / C in
    # [512, 8192] for a cluster and up to 16384 for one CTA, keep the default variant)
    shapes = [(1024, 1031), (2048, 1500), (1024, 2310), (2048, 4099), (1024, 15000)]
    streams, host = _streams(shapes, 700)
    C = VARIANTS[name]
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.txt")
        with open(cache, "w") as f:
            for c in range(5):
                f.write(f"{2048 << c} {name}\n")
        plan = ipfb.BatchedPlan(streams, tune_cache=cache)
        for c in range(5):
            M = 2048 << c
            if _in_range(M, C, name):
                assert plan.variant(M) == name, M
    xs = plan.run()
    torch.cuda.synchronize()
    refs = obatched.ipfb_batched(host)
    for (N, J), x, ref in zip(shapes, xs, refs):
        assert relrms(x.cpu().numpy(), ref) < 1e-4, (name, N, J)
    plan.close()


def test_batched_odd_bluestein_lengths_match_oracle():
    """Above J = 8192 the Bluestein length is the smallest of 5 x 4096, 6 x 4096 and
    32768 that holds 2J - 1 (clusters of 5 and 6 CTAs with a direct C-point cross
    stage): each stream still matches the oracle's exact J-point circulant inverse."""
    shapes = [(1024, 8193), (2048, 10240), (1024, 10241), (1024, 12288), (1024, 12289)]
    want_M = [20480, 20480, 24576, 24576, 32768]
    for (_, J), M in zip(shapes, want_M):
        assert M >= 2 * J - 1 and all(c * 4096 < 2 * J - 1 for c in (5, 6) if c * 4096 < M), (J, M)
    streams, host = _streams(shapes, 800)
    plan = ipfb.BatchedPlan(streams)
    for c in (5, 6):
        assert plan.variant(c * 4096) == f"c{c}_t256_r32"
    xs = plan.run()
    torch.cuda.synchronize()
    refs = obatched.ipfb_batched(host)
    for (N, J), x, ref in zip(shapes, xs, refs):
        assert relrms(x.cpu().numpy(), ref) < 1e-4, (N, J)
    plan.close()


def test_batched_matches_single_stream_path_for_pow2():
    # J = 2048 is a power of two: the Bluestein path and ipfb_wiener agree
    N, J = 1024, 2048
    streams, host = _streams([(N, J)], 500)
    plan = ipfb.BatchedPlan(streams)
    xb = plan.run()[0]
    xs = ipfb.ipfb_wiener(streams[0]["codes"], streams[0]["scale"], streams[0]["window"], streams[0]["noise_level"])
    torch.cuda.synchronize()
    assert relrms(xb.cpu().numpy(), xs.cpu().numpy()) < 1e-5
    plan.close()


def test_batched_rejects_unsupported():
    streams, _ = _streams([(512, 1024)], 600)
    with pytest.raises(ipfb.IpfbError):
        ipfb.BatchedPlan(streams)
    streams, _ = _streams([(1024, 1000)], 601)
    with pytest.raises(ipfb.IpfbError):
        ipfb.BatchedPlan(streams)
