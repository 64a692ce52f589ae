"""Checkpoint file format on the host (no GPU): round trip of links, seed and next
trajectory; the FNV-1a hash against its published test vectors; rejection of a
flipped payload bit, a truncated file, a wrong magic and a wrong version."""
import struct

import numpy as np
import pytest

from paper_2602_20516_b300 import checkpoint as ck


def _links(dims, seed):
    rng = np.random.default_rng(seed)
    V = int(np.prod(dims))
    return rng.standard_normal((V, 4, 3, 3)) + 1j * rng.standard_normal((V, 4, 3, 3))


def test_fnv1a_reference_values():
    # FNV-1a 64 of the empty input is the offset basis; of the single byte "a" it is
    # 0xaf63dc4c8601ec8c (published test vector).  Over one 64-bit word w the recurrence
    # is the same step with the whole word xored in: for w = 0x61 it equals the
    # one-byte value.
    assert ck.fnv1a_words([]) == 0xCBF29CE484222325
    assert ck.fnv1a_words([0x61]) == 0xAF63DC4C8601EC8C


def test_round_trip(tmp_path):
    dims = (4, 2, 2, 6)
    U = _links(dims, 1)
    p = tmp_path / "c.lgt"
    ck.write(p, dims, 1234567890123, 17, U)
    d = ck.read(p)
    assert d["dims"] == list(dims) and d["seed"] == 1234567890123 and d["next_traj"] == 17
    assert np.array_equal(d["links"], U)
    assert p.stat().st_size == 56 + U.nbytes + 8


def test_corruption_is_detected(tmp_path):
    dims = (2, 2, 2, 2)
    p = tmp_path / "c.lgt"
    ck.write(p, dims, 5, 3, _links(dims, 2))
    raw = bytearray(p.read_bytes())
    bad = bytearray(raw)
    bad[56 + 100] ^= 0x04
    (tmp_path / "flip.lgt").write_bytes(bytes(bad))
    with pytest.raises(ValueError, match="checksum"):
        ck.read(tmp_path / "flip.lgt")
    (tmp_path / "short.lgt").write_bytes(bytes(raw[:-16]))
    with pytest.raises(ValueError, match="truncated"):
        ck.read(tmp_path / "short.lgt")
    bad = bytearray(raw)
    bad[0:8] = b"NOTCKPT1"
    (tmp_path / "magic.lgt").write_bytes(bytes(bad))
    with pytest.raises(ValueError, match="not a checkpoint"):
        ck.read(tmp_path / "magic.lgt")
    bad = bytearray(raw)
    bad[8:16] = struct.pack("<Q", 2)
    (tmp_path / "version.lgt").write_bytes(bytes(bad))
    with pytest.raises(ValueError, match="version"):
        ck.read(tmp_path / "version.lgt")


def test_write_replaces_atomically(tmp_path):
    """The writer goes through a temporary file renamed over the target: no .tmp is
    left behind and an existing checkpoint is replaced whole."""
    dims = (2, 2, 2, 2)
    p = tmp_path / "c.lgt"
    ck.write(p, dims, 1, 1, _links(dims, 5))
    ck.write(p, dims, 2, 7, _links(dims, 6))
    assert not (tmp_path / "c.lgt.tmp").exists()
    r = ck.read(p)
    assert r["seed"] == 2 and r["next_traj"] == 7
    assert np.array_equal(r["links"], _links(dims, 6))
