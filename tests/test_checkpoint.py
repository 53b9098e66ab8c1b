"""Net checkpoints (parameters + Adam state + batch-order generator state): file
format round trip and rejection of foreign or truncated files (host only)."""
import json

import numpy as np
import pytest

from paper_2608_23441_b300 import ipfb, precond_train as pt


def _state(seed=0):
    rng = np.random.default_rng(seed)
    n = ipfb.NET_NPARAMS
    gen = np.random.default_rng(seed + 1)
    gen.permutation(10)
    return (rng.standard_normal(n).astype(np.float32), rng.standard_normal(n).astype(np.float32),
            np.abs(rng.standard_normal(n)).astype(np.float32), gen.bit_generator.state)


def test_round_trip_is_bit_exact(tmp_path):
    th, m, v, rs = _state()
    p = tmp_path / "net.ckpt"
    pt.save_checkpoint(str(p), th, m, v, step=1234, rng_state=rs, info={"loss": 0.17})
    d = pt.load_checkpoint(str(p))
    assert np.array_equal(d["theta"], th) and np.array_equal(d["m"], m) and np.array_equal(d["v"], v)
    assert d["step"] == 1234 and d["info"] == {"loss": 0.17}
    # the generator resumes where it stopped
    g1 = np.random.default_rng()
    g1.bit_generator.state = d["rng"]
    g2 = np.random.default_rng()
    g2.bit_generator.state = rs
    assert np.array_equal(g1.permutation(50), g2.permutation(50))
    # layout: magic, header length, JSON header, then float32 arrays
    blob = p.read_bytes()
    hlen = int.from_bytes(blob[8:12], "little")
    assert blob[:8] == b"IPFBNET1" and json.loads(blob[12:12 + hlen])["nparams"] == ipfb.NET_NPARAMS
    assert len(blob) == 12 + hlen + 3 * 4 * ipfb.NET_NPARAMS


def test_parameters_only(tmp_path):
    th, _, _, _ = _state(3)
    p = tmp_path / "theta.ckpt"
    pt.save_checkpoint(str(p), th)
    d = pt.load_checkpoint(str(p))
    assert np.array_equal(d["theta"], th) and d["m"] is None and d["v"] is None and d["step"] == 0


def test_rejects_bad_files(tmp_path):
    th, m, v, rs = _state(5)
    with pytest.raises(ValueError):
        pt.save_checkpoint(str(tmp_path / "a"), th[:-1])
    with pytest.raises(ValueError):
        pt.save_checkpoint(str(tmp_path / "a"), th, m[:-1], v)
    p = tmp_path / "ok.ckpt"
    pt.save_checkpoint(str(p), th, m, v, step=2, rng_state=rs)
    blob = p.read_bytes()
    (tmp_path / "trunc").write_bytes(blob[:-4])
    with pytest.raises(ValueError):
        pt.load_checkpoint(str(tmp_path / "trunc"))
    (tmp_path / "magic").write_bytes(b"XXXXXXXX" + blob[8:])
    with pytest.raises(ValueError):
        pt.load_checkpoint(str(tmp_path / "magic"))


def test_parse_seeds():
    assert pt.parse_seeds("1000-1003") == [1000, 1001, 1002, 1003]
    assert pt.parse_seeds("3, 5,9") == [3, 5, 9]
    assert pt.parse_seeds("1-2,7") == [1, 2, 7]
    for bad in ("", "5-3", "-4", "a"):
        with pytest.raises(ValueError):
            pt.parse_seeds(bad)
