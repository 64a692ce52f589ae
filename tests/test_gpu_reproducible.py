"""Run-to-run reproducibility (the stand-in for a race detector, compute-sanitizer
being unavailable where these tests run): every reduction sums its partials in a fixed
order and no kernel accumulates with atomics, so the same call on the same state gives
bitwise the same result.  A race would show up here as a difference between runs."""
import pytest
import torch

from paper_2602_20516_b300 import synth

pytestmark = pytest.mark.gpu

DIMS = (8, 8, 8, 16)


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _lat(lgt):
    lat = lgt.Lattice(DIMS)
    lat.set_links(synth.random_links(DIMS, 0.5, 91))
    return lat


def test_solves_and_forces_repeat_bitwise(lgt):
    lat = _lat(lgt)
    phi = lat.gaussian_spinor(92, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    sp = lgt.solver("mixed", tol=1e-10, delta=3e-6)
    x1, s1 = lat.cg_solve(phi, 0.156, True, sp)
    x2, s2 = lat.cg_solve(phi, 0.156, True, sp)
    assert s1 == {**s2, "seconds": s1["seconds"]} and torch.equal(x1, x2)
    for arith in ("df64", "fp64", "fp32"):
        ap = lgt.action_params(beta=5.8, kappa=0.156, even_odd=True, force_arith=arith)
        F1, _ = lat.force(ap, phi, sp)
        F2, _ = lat.force(ap, phi, sp)
        assert torch.equal(F1, F2), arith
    full = lat.gaussian_spinor(93, 0, lgt.FIELD_SOURCE, lgt.FULL)
    ap = lgt.action_params(beta=5.8, kappa=0.13, csw=1.5)
    G1, _ = lat.force(ap, full, lgt.solver("fp64", tol=1e-12))
    G2, _ = lat.force(ap, full, lgt.solver("fp64", tol=1e-12))
    assert torch.equal(G1, G2)


def test_trajectory_repeats_bitwise(lgt):
    ap = lgt.action_params(beta=5.8, kappa=0.156, even_odd=True)
    sp = lgt.solver("mixed", tol=1e-10, delta=3e-6)
    hp = lgt.hmc_params("omelyan", 4, 0.2, sp, sp)
    out = []
    for _ in range(2):
        lat = _lat(lgt)
        r = lat.hmc_trajectory(ap, hp, 94, 0)
        out.append((r["dH"], r["accepted"], lat.get_links()))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert torch.equal(out[0][2], out[1][2])
