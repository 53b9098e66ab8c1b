"""The benchmark's torch.fft comparison arm computes the same step as the library:
run on CPU tensors (torch.fft's CPU backend) against the FP64 oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench  # noqa: E402
from oracle import ipfb as oipfb  # noqa: E402
from oracle import pfb as opfb  # noqa: E402
from oracle import upchan as oup  # noqa: E402
from paper_2608_23441_b300 import synth  # noqa: E402


@pytest.mark.parametrize("N,J,U,phi2", [(64, 256, 4, 0.0141), (128, 128, 2, 0.1)])
def test_cufft_comparison_step_matches_the_oracle(N, J, U, phi2):
    x = synth.stream_config(N, J, 5, ntones=3)
    w = opfb.sinc_hamming_window(N, 4).astype(np.float32).astype(np.float64)
    codes, scale, _ = opfb.pfb_forward(x, w)
    step = bench.cufft_pipeline(torch, torch.from_numpy(codes), torch.from_numpy(scale),
                                torch.from_numpy(w.astype(np.float32)), phi2, U)
    got = step().numpy().astype(np.complex128)
    ref = oup.upchannelize(oipfb.ipfb_wiener(codes, scale, w, phi2), U * N)
    assert got.shape == ref.shape
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
