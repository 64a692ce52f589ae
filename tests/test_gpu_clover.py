"""Clover (Sheikholeslami-Wohlert) term on the GPU against the FP64 oracle: the
operator D_sw (FP64 and FP32), full-lattice solves, the pseudofermion action, its
force (Lie and real-component forms, through every force arithmetic) and an HMC
trajectory; and the same for the even-odd form (Schur complement with M_oo^{-1} and
the odd-site determinant in the action).  Tolerances as for the Wilson operator: 1e-14 for FP64 operators,
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


def test_even_odd_clover_dhat_vs_oracle(lgt, ora):
    """Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe (M = 1 + A; M_oo^{-1} from the Cholesky
    factors of the chiral blocks) and its normal operator against the oracle's dense
    inverse, FP64 and FP32."""
    U = synth.random_links(DIMS, 0.5, 111)
    psi = synth.gaussian_spinor(DIMS, 112, parity_mask=1)
    lat = _lat(lgt, U)
    lat.set_clover(CSW, KAPPA)
    ev = synth.parity(DIMS) == 0
    for dag in (False, True):
        want = ora.dhat_sw(DIMS, U, KAPPA, CSW, psi, dagger=dag)[ev]
        for prec, bar in ((lgt.FP64, 1e-13), (lgt.FP32, 3e-6)):
            f = lat.pack_spinor(psi, lgt.EVEN, prec)
            out = lat.dslash(f, lgt.OP_DHAT, lgt.EVEN, dag, KAPPA, prec)
            assert H.rel(_np(lat.unpack_spinor(out, lgt.EVEN, prec))[ev], want) < bar, (prec, dag)
    want = ora.dhat_sw(DIMS, U, KAPPA, CSW, ora.dhat_sw(DIMS, U, KAPPA, CSW, psi), dagger=True)[ev]
    f = lat.pack_spinor(psi, lgt.EVEN, lgt.FP64)
    out = lat.dslash(f, lgt.OP_DHAT_NORMAL, lgt.EVEN, False, KAPPA, lgt.FP64)
    assert H.rel(_np(lat.unpack_spinor(out, lgt.EVEN, lgt.FP64))[ev], want) < 1e-13


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_even_odd_clover_solve(lgt, ora, precision):
    U = synth.random_links(DIMS, 0.5, 113)
    b = synth.gaussian_spinor(DIMS, 114, parity_mask=1)
    lat = _lat(lgt, U)
    lat.set_clover(CSW, KAPPA)
    tol = 1e-12 if precision == "fp64" else 1e-10
    x, st = lat.cg_solve(lat.pack_spinor(b, lgt.EVEN, lgt.FP64), KAPPA, True, lgt.solver(precision, tol=tol))
    assert st["true_rel_residual"] <= tol
    xo, _, _ = ora.cg_sw_eo(DIMS, U, KAPPA, CSW, b, tol=1e-13)
    ev = synth.parity(DIMS) == 0
    assert H.rel(_np(lat.unpack_spinor(x, lgt.EVEN, lgt.FP64))[ev], xo[ev]) < (1e-9 if precision == "fp64" else 1e-6)


def test_even_odd_clover_action_and_force(lgt, ora):
    """S_f = phi_e^+ (Dhat^+ Dhat)^{-1} phi_e - 2 ln det M_oo and its force (hopping and
    clover insertions on the even-odd X, Y plus the determinant insertion), Lie and
    real-component forms, every force arithmetic."""
    U = synth.random_links(DIMS, 0.5, 115)
    phi = synth.gaussian_spinor(DIMS, 116, parity_mask=1)
    lat = _lat(lgt, U)
    pf = lat.pack_spinor(phi, lgt.EVEN, lgt.FP64)
    ap = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW, even_odd=True)
    sp = lgt.solver("fp64", tol=1e-13)
    _, Sf, _ = lat.action(ap, pf, sp)
    So, _ = ora.pf_action_sw_eo(DIMS, U, KAPPA, CSW, phi, tol=1e-13)
    assert abs(Sf - So) / abs(So) < 1e-11
    Fo = ora.gauge_force(DIMS, U, 5.7) + ora.pf_force_sw_eo(DIMS, U, KAPPA, CSW, phi, tol=1e-13)[0]
    F, _ = lat.force(ap, pf, sp)
    assert H.rel(_np(lat.unpack_momenta(F)), Fo) < 1e-10
    Go = ora.gauge_action_grad(DIMS, U, 5.7) + ora.pf_action_grad_sw_eo(DIMS, U, KAPPA, CSW, phi, tol=1e-13)[0]
    G, _ = lat.force(ap, pf, sp, form=lgt.GRAD_G)
    assert H.rel(_np(lat.unpack_grad(G)), Go) < 1e-10
    for arith in ("fp64", "df64", "fp32"):
        a2 = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW, even_odd=True, force_arith=arith)
        F2, _ = lat.force(a2, pf, lgt.solver("mixed", tol=1e-10, delta=1e-4))
        assert H.rel(_np(lat.unpack_momenta(F2)), Fo) < 1e-6, arith
    # the determinant term alone (phi = 0): the force of -2 sum_odd ln det M
    z = lat.pack_spinor(np.zeros_like(phi), lgt.EVEN, lgt.FP64)
    a0 = lgt.action_params(beta=0.0, kappa=KAPPA, csw=CSW, even_odd=True)
    Fd, _ = lat.force(a0, z, sp)
    Fdo = ora.pf_force_sw_eo(DIMS, U, KAPPA, CSW, np.zeros_like(phi), tol=1e-13)[0]
    assert H.rel(_np(lat.unpack_momenta(Fd)), Fdo) < 1e-10


def test_even_odd_clover_hmc_trajectory_matches_oracle(lgt, ora):
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3, 117)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    ap = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW, even_odd=True)
    sp = lgt.solver("fp64", tol=1e-13)
    r = lat.hmc_trajectory(ap, lgt.hmc_params("leapfrog", 10, 1.0, sp, sp), 5, 0)
    Uo, ro = ora.hmc_trajectory(dims, U, ora.hmc_params(5.7, KAPPA, eo=True, integrator="leapfrog", n_steps=10,
                                                        tau=1.0, tol_md=1e-13, tol_action=1e-13, csw=CSW), 5, 0)
    for k in ("K_old", "Sg_old", "Sf_old", "K_new", "Sg_new", "Sf_new"):
        assert abs(r[k] - ro[k]) / abs(ro[k]) < 1e-10, k
    assert abs(r["dH"] - ro["dH"]) < 1e-8 * max(1.0, abs(ro["dH"]))
    assert r["accepted"] == ro["accepted"]
    assert H.rel(_np(lat.get_links()), Uo) < 1e-10


@pytest.mark.parametrize("recompute", [0, 1])
def test_even_odd_clover_with_stout_force_vs_oracle(lgt, ora, recompute):
    """Even-odd clover on 2-level stout links (the clover field, its odd-site inverse and
    the determinant built from the top level): the force through the stout adjoint
    against the oracle's MD force, with the smeared levels stored or recomputed."""
    U = synth.random_links(DIMS, 0.5, 121)
    phi = synth.gaussian_spinor(DIMS, 122, parity_mask=1)
    lat = _lat(lgt, U)
    pf = lat.pack_spinor(phi, lgt.EVEN, lgt.FP64)
    ap = lgt.action_params(beta=5.7, kappa=KAPPA, csw=CSW, even_odd=True, n_stout=2, rho=0.1,
                           stout_recompute=recompute)
    F, _ = lat.force(ap, pf, lgt.solver("fp64", tol=1e-13))
    p = ora.hmc_params(5.7, KAPPA, eo=True, tol_md=1e-13, n_stout=2, rho=0.1, csw=CSW)
    Fo = ora.md_force(DIMS, U, p, phi)
    assert H.rel(_np(lat.unpack_momenta(F)), Fo) < 1e-10
    _, Sf, _ = lat.action(ap, pf, lgt.solver("fp64", tol=1e-13))
    Hs = ora.hamiltonian(DIMS, U, np.zeros((int(np.prod(DIMS)), 4, 8)), phi, p) - ora.gauge_action(DIMS, U, 5.7)
    assert abs(Sf - Hs) / abs(Hs) < 1e-11
