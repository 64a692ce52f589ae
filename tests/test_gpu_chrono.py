"""Chronological initial guesses (lgt_solver_params.chrono): a solve starts from the
combination of earlier solutions of the same operator that minimises the A-norm of
the error.  The guess may change the iteration count, never the stop test: every
solve still ends on the FP64 true residual, so solutions agree with zero-guess
solves within the solver tolerance, and without usable history the solve is the
zero-guess solve bit for bit.
"""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 8)


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _md_sequence(lgt, sp, steps=6, eps=0.02):
    """Solves of Dhat^+Dhat x = b along a short MD link evolution."""
    lat = lgt.Lattice(DIMS)
    lat.set_links(synth.random_links(DIMS, 0.5, 61))
    b = lat.pack_spinor(synth.gaussian_spinor(DIMS, 62, parity_mask=1), lgt.EVEN, lgt.FP64)
    mom = lat.pack_momenta(synth.gaussian_momenta(DIMS, 63))
    out = []
    for _ in range(steps):
        x, st = lat.cg_solve(b, 0.156, True, sp)
        out.append((x.clone(), st))
        lat.md_update(mom, eps, lgt.UPDATE_U)
    return out


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_guess_along_md_sequence(lgt, precision):
    tol = 1e-10
    zero = _md_sequence(lgt, lgt.solver(precision, tol=tol, delta=1e-4))
    chrono = _md_sequence(lgt, lgt.solver(precision, tol=tol, delta=1e-4, chrono=4))
    # the first solve has no history: identical to the zero-guess solve
    assert torch.equal(chrono[0][0], zero[0][0])
    assert chrono[0][1]["iters"] == zero[0][1]["iters"]
    for (xc, sc), (xz, sz) in zip(chrono, zero):
        assert sc["true_rel_residual"] <= tol
        # both solutions are within cond(A) * tol of the exact one
        xc_, xz_ = xc.cpu().numpy(), xz.cpu().numpy()
        assert H.rel(xc_, xz_) < 1e-7
    its_c = sum(s["iters"] for _, s in chrono[2:])
    its_z = sum(s["iters"] for _, s in zero[2:])
    assert its_c < 0.8 * its_z, (its_c, its_z)


def test_reset_and_kappa_change_give_zero_guess_solve(lgt):
    lat = lgt.Lattice(DIMS)
    lat.set_links(synth.random_links(DIMS, 0.5, 64))
    b = lat.pack_spinor(synth.gaussian_spinor(DIMS, 65, parity_mask=1), lgt.EVEN, lgt.FP64)
    sp0 = lgt.solver("mixed", tol=1e-10, delta=1e-4)
    spc = lgt.solver("mixed", tol=1e-10, delta=1e-4, chrono=2)
    x0, s0 = lat.cg_solve(b, 0.15, True, sp0)
    lat.cg_solve(b, 0.15, True, spc)              # recorded
    x1, s1 = lat.cg_solve(b, 0.15, True, spc)     # guessed: far fewer iterations
    assert s1["iters"] < 0.6 * s0["iters"] and H.rel(x1.cpu().numpy(), x0.cpu().numpy()) < 1e-7
    lat.chrono_reset()
    x2, s2 = lat.cg_solve(b, 0.15, True, spc)
    assert torch.equal(x2, x0) and s2["iters"] == s0["iters"]
    # another kappa: the kept solutions belong to another operator
    x3, s3 = lat.cg_solve(b, 0.152, True, spc)
    x4, s4 = lat.cg_solve(b, 0.152, True, sp0)
    assert torch.equal(x3, x4) and s3["iters"] == s4["iters"]


def test_hmc_trajectory_with_guess(lgt):
    """Same start and seeds: an Omelyan trajectory whose MD solves start from the
    chronological guess reproduces the zero-guess Delta H within the effect of the
    solver tolerance, with fewer CG iterations."""
    lat = lgt.Lattice(DIMS)
    lat.random_links(7, 0.5)
    U0 = lat.get_links()
    ap = lgt.action_params(beta=5.8, kappa=0.156, even_odd=True)
    res = {}
    for c in (0, 4):
        lat.set_links(U0)
        md = lgt.solver("mixed", tol=1e-11, delta=1e-4, chrono=c)
        act = lgt.solver("mixed", tol=1e-11, delta=1e-4)
        res[c] = lat.hmc_trajectory(ap, lgt.hmc_params("omelyan", 10, 1.0, md, act), 7, 0)
    assert abs(res[4]["dH"] - res[0]["dH"]) < 1e-6 * max(1.0, abs(res[0]["dH"]))
    # measured: 1933 against 2270 iterations (10 Omelyan steps, eps = 0.1)
    assert res[4]["total"]["iters"] < 0.9 * res[0]["total"]["iters"]


def test_guess_with_nearly_parallel_history(lgt):
    """Small MD steps make the kept solutions nearly parallel (the Gram matrix close to
    singular at the FP32 level of its entries): the guess must still help, never hurt."""
    zero = _md_sequence(lgt, lgt.solver("mixed", tol=1e-10, delta=1e-4), steps=9, eps=0.002)
    chrono = _md_sequence(lgt, lgt.solver("mixed", tol=1e-10, delta=1e-4, chrono=4), steps=9, eps=0.002)
    for (xc, sc), (xz, sz) in zip(chrono, zero):
        assert sc["true_rel_residual"] <= 1e-10
        assert sc["iters"] <= sz["iters"]
        assert H.rel(xc.cpu().numpy(), xz.cpu().numpy()) < 1e-7
    # measured: 245 against 455 iterations over the last five solves
    assert sum(s["iters"] for _, s in chrono[4:]) < 0.75 * sum(s["iters"] for _, s in zero[4:])
