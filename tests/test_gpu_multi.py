"""Several right-hand sides on shared links (lgt_hop_multi, lgt_cg_solve_multi).

Sharing the link loads must not change any system's arithmetic: the multi-source
hop equals the single-source FP32 hop bit for bit, and a system solved among
others has the same solution (bit for bit), iteration count and number of
reliable updates as the same system solved alone.  Against the FP64 oracle the
solutions agree within the bound the solver tolerance sets (cond(A) * tol).
"""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

DIMS = (8, 6, 4, 10)   # Vh = 960: 7.5 blocks of 128, a ragged tail, the time wrap


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _lat(lgt, dims, seed, alpha=0.5):
    lat = lgt.Lattice(dims)
    lat.set_links(synth.random_links(dims, alpha, seed))
    return lat


@pytest.mark.parametrize("nrhs", [1, 2, 3, 4])
@pytest.mark.parametrize("out_parity,dagger", [(0, False), (1, False), (0, True), (1, True)])
def test_hop_multi_equals_single_hops(lgt, nrhs, out_parity, dagger):
    lat = _lat(lgt, DIMS, 41)
    src_par = 1 - out_parity
    ins = [lat.pack_spinor(synth.gaussian_spinor(DIMS, 50 + k, parity_mask=1 << src_par), src_par, lgt.FP32)
           for k in range(nrhs)]
    outs = lat.hop_multi(ins, out_parity, dagger)
    for k in range(nrhs):
        one = lat.dslash(ins[k], lgt.OP_HOP, out_parity, dagger, 0.0, lgt.FP32)
        assert torch.equal(outs[k], one), k


def _sources(lgt, lat, n, seed, dims=DIMS):
    return [lat.pack_spinor(synth.gaussian_spinor(dims, seed + k, parity_mask=1), lgt.EVEN, lgt.FP64)
            for k in range(n)]


def test_multi_solve_equals_each_alone(lgt):
    """Mixed CG, three sources with different kappa: every solution, iteration count
    and reliable-update count equals the single-source solve."""
    lat = _lat(lgt, DIMS, 42)
    kappas = [0.14, 0.15, 0.156]
    bs = _sources(lgt, lat, 3, 60)
    sp = lgt.solver("mixed", tol=1e-10, delta=1e-3)
    xs, sts = lat.cg_solve_multi(bs, kappas, sp)
    for k in range(3):
        x1, st1 = lat.cg_solve(bs[k], kappas[k], True, sp)
        assert torch.equal(xs[k], x1), k
        assert sts[k]["iters"] == st1["iters"] and sts[k]["reliable_updates"] == st1["reliable_updates"], k
        assert sts[k]["true_rel_residual"] <= 1e-10
    # the systems converge at different iteration counts (kappa sets the conditioning)
    assert len({s["iters"] for s in sts}) > 1


def test_multi_solve_vs_oracle(lgt, ora):
    lat = _lat(lgt, DIMS, 43)
    U = synth.random_links(DIMS, 0.5, 43)
    kappas = [0.145, 0.155, 0.157, 0.15]
    srcs = [synth.gaussian_spinor(DIMS, 70 + k, parity_mask=1) for k in range(4)]
    bs = [lat.pack_spinor(b, lgt.EVEN, lgt.FP64) for b in srcs]
    xs, sts = lat.cg_solve_multi(bs, kappas, lgt.solver("mixed", tol=1e-10, delta=1e-4))
    for k in range(4):
        xo, _, _ = ora.cg(DIMS, U, kappas[k], srcs[k], eo=True, tol=1e-13)
        got = lat.unpack_spinor(xs[k], lgt.EVEN, lgt.FP64).cpu().numpy()
        # cond(Dhat^+ Dhat) is O(1e2) on these fields: solution error <= cond * tol
        assert H.rel(got, xo) < 1e-7, k


def test_multi_fp64_and_zero_source(lgt):
    """FP64 systems are solved one after another (equal to lgt_cg_solve); a zero
    source returns x = 0 after no iterations while the others converge."""
    lat = _lat(lgt, DIMS, 44)
    bs = _sources(lgt, lat, 3, 80)
    bs[1].zero_()
    sp = lgt.solver("fp64", tol=1e-12)
    xs, sts = lat.cg_solve_multi(bs, [0.15, 0.15, 0.155], sp)
    for k in (0, 2):
        x1, st1 = lat.cg_solve(bs[k], [0.15, 0.15, 0.155][k], True, sp)
        assert torch.equal(xs[k], x1) and sts[k]["iters"] == st1["iters"]
    assert not torch.any(xs[1]) and sts[1]["iters"] == 0
    xs, sts = lat.cg_solve_multi(bs, [0.15, 0.15, 0.155], lgt.solver("mixed", tol=1e-10))
    assert not torch.any(xs[1]) and sts[1]["iters"] == 0 and sts[0]["iters"] > 0
    assert max(sts[0]["true_rel_residual"], sts[2]["true_rel_residual"]) <= 1e-10


def test_multi_rejects_bad_arguments(lgt):
    lat = _lat(lgt, (4, 4, 4, 4), 45)
    bs = _sources(lgt, lat, 2, 90, dims=(4, 4, 4, 4))
    with pytest.raises(lgt.LGTError):
        lat.cg_solve_multi(bs, [0.15, 0.15], xs=[bs[1], torch.zeros_like(bs[0])])   # x aliases b
    with pytest.raises(lgt.LGTError):
        lat.cg_solve_multi(bs * 3, [0.15] * 6)                                       # nrhs > 4
