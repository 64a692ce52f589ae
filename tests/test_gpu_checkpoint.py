"""HMC checkpoint / resume through the library: a chain resumed from a checkpoint
repeats the next trajectory bitwise; files written by the library and by the host
module read back in the other; damaged files and another lattice's file are refused
with the handle's links untouched."""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import checkpoint as ck

pytestmark = pytest.mark.gpu

DIMS = (4, 4, 4, 4)


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _hmc(lgt):
    ap = lgt.action_params(beta=5.7, kappa=0.15, even_odd=True)
    sp = lgt.solver("fp64", tol=1e-12)
    return ap, lgt.hmc_params("leapfrog", 10, 1.0, sp, sp)


def test_resume_repeats_next_trajectory_bitwise(lgt, tmp_path):
    ap, hp = _hmc(lgt)
    lat = lgt.Lattice(DIMS)
    lat.random_links(3, 0.3)
    lat.hmc_trajectory(ap, hp, 9, 0)
    path = tmp_path / "chain.lgt"
    lat.save_checkpoint(path, 9, 1)
    r1 = lat.hmc_trajectory(ap, hp, 9, 1)
    U1 = lat.get_links()
    other = lgt.Lattice(DIMS)
    other.random_links(4, 0.5)
    seed, nxt = other.load_checkpoint(path)
    assert (seed, nxt) == (9, 1)
    r2 = other.hmc_trajectory(ap, hp, seed, nxt)
    assert r1["dH"] == r2["dH"] and r1["accepted"] == r2["accepted"]
    assert torch.equal(other.get_links(), U1)


def test_library_and_host_module_agree(lgt, tmp_path):
    lat = lgt.Lattice(DIMS)
    lat.random_links(5, 0.4)
    p = tmp_path / "lib.lgt"
    lat.save_checkpoint(p, 77, 12)
    d = ck.read(p)
    assert d["dims"] == list(DIMS) and d["seed"] == 77 and d["next_traj"] == 12
    assert np.array_equal(d["links"], lat.get_links().cpu().numpy())
    # written on the host, loaded by the library
    U = lgt.Lattice(DIMS)
    U.random_links(6, 0.4)
    q = tmp_path / "host.lgt"
    ck.write(q, DIMS, 8, 2, U.get_links().cpu().numpy())
    seed, nxt = lat.load_checkpoint(q)
    assert (seed, nxt) == (8, 2)
    assert torch.equal(lat.get_links(), U.get_links())


def test_bad_files_are_refused(lgt, tmp_path):
    lat = lgt.Lattice(DIMS)
    lat.random_links(7, 0.4)
    good = tmp_path / "good.lgt"
    lat.save_checkpoint(good, 1, 1)
    before = lat.get_links().clone()
    raw = bytearray(good.read_bytes())
    raw[56 + 8 * 11] ^= 0x10
    (tmp_path / "flip.lgt").write_bytes(bytes(raw))
    (tmp_path / "short.lgt").write_bytes(good.read_bytes()[:-9])
    for name in ("flip.lgt", "short.lgt", "missing.lgt"):
        with pytest.raises(lgt.LGTError):
            lat.load_checkpoint(tmp_path / name)
    big = lgt.Lattice((4, 4, 4, 6))
    big.random_links(1, 0.4)
    big.save_checkpoint(tmp_path / "other.lgt", 1, 1)
    with pytest.raises(lgt.LGTError):
        lat.load_checkpoint(tmp_path / "other.lgt")
    assert torch.equal(lat.get_links(), before)
