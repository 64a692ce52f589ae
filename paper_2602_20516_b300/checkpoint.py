"""Host-side reader and writer of HMC checkpoint files (the format lgt_save_checkpoint
and lgt_load_checkpoint use), for inspecting or preparing a chain's state without a
GPU.  Layout, little-endian: 7 header words of 64 bits (magic "LGTCKPT1", version 1,
dims[0] | dims[1] << 32, dims[2] | dims[3] << 32, seed, next trajectory, payload bytes),
the canonical links (complex128 [V][4][3][3]), then the FNV-1a hash of header and
payload over 64-bit words.  The hash is a sequential recurrence, computed here in
Python: fine for small lattices and tests, slow (minutes) for 32^3 x 64 files."""
import os
import struct

import numpy as np

MAGIC = b"LGTCKPT1"
VERSION = 1
_BASIS = 0xCBF29CE484222325
_PRIME = 0x100000001B3
_MASK = (1 << 64) - 1


def fnv1a_words(words, h=_BASIS):
    """FNV-1a over a sequence of unsigned 64-bit words."""
    for w in words:
        h = ((h ^ int(w)) * _PRIME) & _MASK
    return h


def _header(dims, seed, next_traj, nbytes):
    return np.array([struct.unpack("<Q", MAGIC)[0], VERSION,
                     dims[0] | (dims[1] << 32), dims[2] | (dims[3] << 32),
                     seed, next_traj, nbytes], dtype="<u8")


def write(path, dims, seed, next_traj, links):
    """links: complex128 array of shape (V, 4, 3, 3)."""
    dims = [int(d) for d in dims]
    V = int(np.prod(dims))
    links = np.ascontiguousarray(links, dtype=np.complex128)
    if links.shape != (V, 4, 3, 3):
        raise ValueError("links must have shape (V, 4, 3, 3)")
    payload = links.view("<u8").reshape(-1)
    head = _header(dims, int(seed), int(next_traj), payload.nbytes)
    h = fnv1a_words(payload, fnv1a_words(head))
    # written beside the target, flushed to disk and renamed over it, so an
    # interrupted write leaves the previous checkpoint intact
    tmp = str(path) + ".tmp"
    with open(tmp, "wb") as f:
        f.write(head.tobytes())
        f.write(payload.tobytes())
        f.write(struct.pack("<Q", h))
        f.flush()
        os.fsync(f.fileno())
    os.replace(tmp, path)


def read(path, verify=True):
    """Returns dict(dims, seed, next_traj, links); raises ValueError on a bad file."""
    raw = open(path, "rb").read()
    if len(raw) < 64 or raw[:8] != MAGIC:
        raise ValueError("not a checkpoint")
    head = np.frombuffer(raw[:56], dtype="<u8")
    if int(head[1]) & 0xFFFFFFFF != VERSION:
        raise ValueError("unknown version %d" % int(head[1]))
    dims = [int(head[2]) & 0xFFFFFFFF, int(head[2]) >> 32, int(head[3]) & 0xFFFFFFFF, int(head[3]) >> 32]
    nbytes = int(head[6])
    V = int(np.prod(dims))
    if nbytes != V * 4 * 9 * 16 or len(raw) != 56 + nbytes + 8:
        raise ValueError("truncated or too long")
    payload = np.frombuffer(raw[56:56 + nbytes], dtype="<u8")
    (h,) = struct.unpack("<Q", raw[56 + nbytes:])
    if verify and fnv1a_words(payload, fnv1a_words(head)) != h:
        raise ValueError("checksum mismatch")
    links = payload.view(np.complex128).reshape(V, 4, 3, 3).copy()
    return dict(dims=dims, seed=int(head[4]), next_traj=int(head[5]), links=links)
