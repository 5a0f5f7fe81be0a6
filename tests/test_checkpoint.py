"""On-disk checkpoint format (host only): a nested training state round-trips bit for bit; the fixed
header reads back with a plain struct unpack; damaged files are refused."""
import struct

import numpy as np
import pytest
import torch

from paper_2509_12138_gb300 import checkpoint


def _state():
    rng = np.random.default_rng(4)
    g = torch.Generator().manual_seed(9)
    return {
        "params": torch.from_numpy(rng.standard_normal((15, 101, 4)).astype(np.float32)),
        "opt": {"m": torch.from_numpy(rng.standard_normal((15, 101, 4)).astype(np.float32)),
                "v": torch.from_numpy(rng.uniform(0, 1, (15, 101, 4)).astype(np.float32)),
                "step": torch.tensor([37], dtype=torch.int32)},
        "t": 37, "steps_done": 12,
        "rng": np.random.default_rng(11).bit_generator.state,  # holds 128-bit integers
        "order": np.array([5, 2, 7, 0], dtype=np.int64),
        "densify": {"grad_accum": torch.zeros(101, dtype=torch.float64), "gen": g.get_state(),
                    "flags": torch.tensor([True, False])},
        "empty": {},
    }


def _equal(a, b):
    if isinstance(a, dict):
        assert isinstance(b, dict) and set(a) == set(b)
        for k in a:
            _equal(a[k], b[k])
    elif isinstance(a, torch.Tensor):
        assert isinstance(b, torch.Tensor) and a.dtype == b.dtype and torch.equal(a, b)
    elif isinstance(a, np.ndarray):
        assert isinstance(b, np.ndarray) and a.dtype == b.dtype and np.array_equal(a, b)
    else:
        assert a == b


def test_roundtrip_bit_exact(tmp_path):
    st = _state()
    p = str(tmp_path / "ck.bin")
    checkpoint.save(p, st, 101, 3, 37)
    back, h = checkpoint.load(p)
    _equal(st, back)
    assert h == {"version": 1, "json_bytes": h["json_bytes"], "n_gauss": 101, "sh_degree": 3, "step": 37}
    # the fixed header is plain little-endian fields
    raw = open(p, "rb").read()
    magic, ver, jlen, n, deg, step = struct.unpack_from("<8sIIqiq", raw, 0)
    assert (magic, ver, n, deg, step) == (b"GSCKPT\x00\x01", 1, 101, 3, 37)
    # the first array starts at a 64-byte boundary and holds the parameters as stored in memory
    start = (36 + jlen + 63) // 64 * 64
    got = np.frombuffer(raw[start:start + st["params"].numel() * 4], "<f4").reshape(15, 101, 4)
    assert np.array_equal(got, st["params"].numpy())
    # the generator state restores the same stream
    r = np.random.default_rng()
    r.bit_generator.state = back["rng"]
    assert np.array_equal(r.integers(0, 1 << 30, 8), np.random.default_rng(11).integers(0, 1 << 30, 8))


def test_damaged_files_are_refused(tmp_path):
    p = str(tmp_path / "ck.bin")
    checkpoint.save(p, _state(), 101, 3, 37)
    raw = open(p, "rb").read()
    bad = tmp_path / "bad.bin"
    bad.write_bytes(b"XXXXXXXX" + raw[8:])
    with pytest.raises(ValueError, match="not a checkpoint"):
        checkpoint.load(str(bad))
    bad.write_bytes(raw[:len(raw) - 64])
    with pytest.raises(ValueError, match="truncated"):
        checkpoint.load(str(bad))
    bad.write_bytes(raw[:20])
    with pytest.raises(ValueError, match="too short"):
        checkpoint.load(str(bad))
    with pytest.raises(TypeError):
        checkpoint.save(str(bad), {"x": object()}, 1, 0, 0)
