"""Clover (Sheikholeslami-Wohlert) term on the GPU against the FP64 oracle: the
operator D_sw (FP64 and FP32), full-lattice solves, the pseudofermion action, its
force (Lie and real-component forms, through every force arithmetic) and an HMC
trajectory.  Tolerances as for the Wilson operator: 1e-14 for FP64 operators,
2e-6 for FP32 ones, 1e-10 for FP64 forces with both solvers at 1e-13, 1e-6 for
the mixed path.
"""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

DIMS = (8, 6, 4, 10)
KAPPA, CSW = 0.13, 1.5


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _np(t):
    return t.detach().cpu().numpy()


def _lat(lgt, U):
    lat = lgt.Lattice(DIMS)
    lat.set_links(U)
    return lat


@pytest.mark.parametrize("dagger", [False, True])
def test_clover_dirac_vs_oracle(lgt, ora, dagger):
    U = synth.random_links(DIMS, 0.5, 101)
    psi = synth.gaussian_spinor(DIMS, 102)
    lat = _lat(lgt, U)
    lat.set_clover(CSW, KAPPA)
    want = ora.dirac_sw(DIMS, U, KAPPA, CSW, psi, dagger=dagger)
    for prec, bar in ((lgt.FP64, 1e-14), (lgt.FP32, 2e-6)):
        f = lat.pack_spinor(psi, lgt.FULL, prec)
        out = lat.dslash(f, lgt.OP_D, lgt.FULL, dagger, KAPPA, prec)
        assert H.rel(_np(lat.unpack_spinor(out, lgt.FULL, prec)), want) < bar, prec
    # detaching restores the Wilson operator
    lat.set_clover(0.0, KAPPA)
    f = lat.pack_spinor(psi, lgt.FULL, lgt.FP64)
    out = lat.dslash(f, lgt.OP_D, lgt.FULL, dagger, KAPPA, lgt.FP64)
    assert H.rel(_np(lat.unpack_spinor(out, lgt.FULL, lgt.FP64)), ora.dirac(DIMS, U, KAPPA, psi, dagger=dagger)) < 1e-14


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_clover_full_lattice_solve(lgt, ora, precision):
    U = synth.random_links(DIMS, 0.5, 103)
    b = synth.gaussian_spinor(DIMS, 104)
    lat = _lat(lgt, U)
    lat.set_clover(CSW, KAPPA)
    tol = 1e-12 if precision == "fp64" else 1e-10
    x, st = lat.cg_solve(lat.pack_spinor(b, lgt.FULL, lgt.FP64), KAPPA, False, lgt.solver(precision, tol=tol))
    assert st["true_rel_residual"] <= tol
    xo, _, _ = ora.cg_sw(DIMS, U, KAPPA, CSW, b, tol=1e-13)
    assert H.rel(_np(lat.unpack_spinor(x, lgt.FULL, lgt.FP64)), xo) < (1e-9 if precision == "fp64" else 1e-6)


def test_clover_action_and_force(lgt, ora):
    U = synth.random_links(DIMS, 0.5, 105)
    phi = synth.gaussian_spinor(DIMS, 106)
    lat = _lat(lgt, U)
    pf = lat.pack_spinor(phi, lgt.FULL, lgt.FP64)
    ap = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW)
    sp = lgt.solver("fp64", tol=1e-13)
    _, Sf, _ = lat.action(ap, pf, sp)
    So, _ = ora.pf_action_sw(DIMS, U, KAPPA, CSW, phi, tol=1e-13)
    assert abs(Sf - So) / abs(So) < 1e-11
    Fo = ora.gauge_force(DIMS, U, 5.7) + ora.pf_force_sw(DIMS, U, KAPPA, CSW, phi, tol=1e-13)[0]
    F, _ = lat.force(ap, pf, sp)
    assert H.rel(_np(lat.unpack_momenta(F)), Fo) < 1e-10
    Go = ora.gauge_action_grad(DIMS, U, 5.7) + ora.pf_action_grad_sw(DIMS, U, KAPPA, CSW, phi, tol=1e-13)[0]
    G, _ = lat.force(ap, pf, sp, form=lgt.GRAD_G)
    assert H.rel(_np(lat.unpack_grad(G)), Go) < 1e-10
    for arith in ("fp64", "df64", "fp32"):
        a2 = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW, force_arith=arith)
        F2, _ = lat.force(a2, pf, lgt.solver("mixed", tol=1e-10, delta=1e-4))
        assert H.rel(_np(lat.unpack_momenta(F2)), Fo) < 1e-6, arith
    # the clover force itself is not small: switching it off changes the force
    F0, _ = lat.force(lgt.action_params(beta=5.7, kappa=KAPPA), pf, sp)
    assert H.rel(_np(lat.unpack_momenta(F0)), Fo) > 1e-2


def test_clover_hmc_trajectory_matches_oracle(lgt, ora):
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3, 107)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    ap = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW)
    sp = lgt.solver("fp64", tol=1e-13)
    r = lat.hmc_trajectory(ap, lgt.hmc_params("leapfrog", 10, 1.0, sp, sp), 5, 0)
    Uo, ro = ora.hmc_trajectory(dims, U, ora.hmc_params(5.7, KAPPA, integrator="leapfrog", n_steps=10, tau=1.0,
                                                        tol_md=1e-13, tol_action=1e-13, csw=CSW), 5, 0)
    for k in ("K_old", "Sg_old", "Sf_old", "K_new", "Sg_new", "Sf_new"):
        assert abs(r[k] - ro[k]) / abs(ro[k]) < 1e-10, k
    assert abs(r["dH"] - ro["dH"]) < 1e-8 * max(1.0, abs(ro["dH"]))
    assert r["accepted"] == ro["accepted"]
    assert H.rel(_np(lat.get_links()), Uo) < 1e-10


def test_clover_rejects_even_odd(lgt):
    U = synth.random_links((4, 4, 4, 4), 0.5, 108)
    lat = lgt.Lattice((4, 4, 4, 4))
    lat.set_links(U)
    phi = lat.pack_spinor(synth.gaussian_spinor((4, 4, 4, 4), 109, parity_mask=1), lgt.EVEN, lgt.FP64)
    with pytest.raises(lgt.LGTError):
        lat.force(lgt.action_params(kappa=KAPPA, csw=CSW, even_odd=True), phi, lgt.solver("fp64"))
    lat.set_clover(CSW, KAPPA)
    with pytest.raises(lgt.LGTError):
        lat.cg_solve(phi, KAPPA, True, lgt.solver("fp64"))
