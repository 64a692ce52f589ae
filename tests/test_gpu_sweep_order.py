"""Sweep order of the even-odd CG launches: walking the sites of every launch in the
direction opposite to the launch before it changes the order of the work only, so the
iterates are bitwise those of the forward order (the reductions index their partials
by site block)."""
import pytest
import torch

from paper_2602_20516_b300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _lat(lgt, dims, seed):
    lat = lgt.Lattice(dims)
    lat.set_links(synth.random_links(dims, 0.5, seed))
    return lat


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_alternate_sweep_order_same_iterates(lgt, precision):
    dims = (8, 8, 8, 16)
    kappa = 0.156
    lat = _lat(lgt, dims, 77)
    b = lat.pack_spinor(synth.gaussian_spinor(dims, 78, parity_mask=1), lgt.EVEN, lgt.FP64)
    sp = lgt.solver(precision, tol=1e-10, delta=1e-3)
    res = []
    for alternate in (False, True):
        lat.set_sweep_order(alternate)
        res.append(lat.cg_solve(b, kappa, True, sp))
    (x0, s0), (x1, s1) = res
    assert s0["iters"] == s1["iters"] and s0["reliable_updates"] == s1["reliable_updates"]
    assert torch.equal(x0, x1)
