"""HMC pins of the oracle: reversibility, Delta H ~ dt^2 (the validation of the
paper's dynamical test, Sec. III B), energy conservation and heatbath identities."""
import numpy as np
import pytest

from paper_2602_20516_b300 import synth
from tests import helpers as H

D4 = (4, 4, 4, 4)


def _setup(seed=1, alpha=0.3):
    U = synth.random_links(D4, alpha, seed)
    mom = synth.gaussian_momenta(D4, seed + 100)
    return U, mom


@pytest.mark.parametrize("integrator,eo", [("leapfrog", False), ("omelyan", True)])
def test_reversibility(ora, integrator, eo):
    U, mom = _setup()
    phi = synth.gaussian_spinor(D4, 3, parity_mask=1 if eo else 3)
    p = ora.hmc_params(5.7, 0.15, eo=eo, integrator=integrator, n_steps=5, tau=0.5,
                       tol_md=1e-14)
    U1, m1, _ = ora.md_integrate(D4, U, mom, phi, p)
    U2, m2, _ = ora.md_integrate(D4, U1, -m1, phi, p)
    assert H.rel(U2, U) < 1e-11
    assert H.rel(-m2, mom) < 1e-10


def _dH(U, mom, phi, p):
    H0 = ora_energy(U, mom, phi, p)
    U1, m1, _ = ORA.md_integrate(D4, U, mom, phi, p)
    return ora_energy(U1, m1, phi, p) - H0


ORA = None


def ora_energy(U, mom, phi, p):
    S = ORA.gauge_action(D4, U, p.beta, p.c1) + ORA.momentum_energy(D4, mom)
    if p.fermions:
        S += ORA.pf_action(D4, U, p.kappa, phi, eo=bool(p.eo), tol=1e-14)[0]
    return S


@pytest.mark.parametrize("integrator", ["leapfrog", "omelyan"])
def test_delta_h_scales_as_dt_squared(ora, integrator):
    global ORA
    ORA = ora
    U, mom = _setup(seed=2)
    phi = synth.gaussian_spinor(D4, 4)
    dh = []
    ns = [8, 16, 32]
    for n in ns:
        p = ora.hmc_params(5.7, 0.15, integrator=integrator, n_steps=n, tau=1.0, tol_md=1e-14)
        dh.append(abs(_dH(U, mom, phi, p)))
    slope = np.polyfit(np.log(1.0 / np.array(ns)), np.log(dh), 1)[0]
    assert abs(slope - 2) < 0.2, (dh, slope)


def test_pure_gauge_energy_conservation(ora):
    global ORA
    ORA = ora
    U, mom = _setup(seed=5)
    phi = np.zeros((256, 4, 3), np.complex128)
    p1 = ora.hmc_params(5.7, 0.0, fermions=False, n_steps=20, tau=1.0)
    p2 = ora.hmc_params(5.7, 0.0, fermions=False, n_steps=40, tau=1.0)
    d1, d2 = abs(_dH(U, mom, phi, p1)), abs(_dH(U, mom, phi, p2))
    # halving the step divides Delta H by ~4 for a second-order integrator
    assert 3.2 < d1 / d2 < 4.8


def test_trajectory_heatbath_and_metropolis(ora):
    U = synth.random_links(D4, 0.3, 7)
    p = ora.hmc_params(5.7, 0.15, n_steps=10, tau=1.0, tol_md=1e-12, tol_action=1e-12)
    U1, r = ora.hmc_trajectory(D4, U, p, 1, 0)
    # the pseudofermion heatbath phi = D^+ xi gives S_f(old) = xi^+ xi exactly; check it
    # against an independent action evaluation on the starting field
    xi = ora.gaussian_spinor(D4, 1, 0, ora.FIELD_XI, 3)
    phi = ora.dirac(D4, U, 0.15, xi, dagger=True)
    S, _ = ora.pf_action(D4, U, 0.15, phi, tol=1e-13)
    assert abs(S - r["Sf_old"]) / S < 1e-11
    assert abs(r["K_old"] - 0.5 * (ora.gaussian_momenta(D4, 1, 0) ** 2).sum()) < 1e-9
    assert r["force_evals"] == 11
    u = ora.uniform(1, 0, 0, 0, ora.FIELD_METROPOLIS)
    assert r["accepted"] == int(u < np.exp(-r["dH"]))
    if not r["accepted"]:
        assert H.rel(U1, U) < 1e-14
    assert np.abs(U1 @ np.conj(np.swapaxes(U1, -1, -2)) - np.eye(3)).max() < 1e-14


# ------------------------------------------------------------------ stout + Sexton-Weingarten
def _sw_params(ora, n_steps, n_inner=10, tau=1.0, tol=1e-13):
    return ora.hmc_params(5.7, 0.15, eo=False, integrator="sexton_weingarten", n_steps=n_steps,
                          tau=tau, tol_md=tol, tol_action=tol, n_inner=n_inner, n_stout=1, rho=0.3)


def test_stout_md_force_finite_difference(ora):
    """The MD force of S_G(U) + S_f(stout(U)) (rho 0.3) against central differences
    of that action in Lie directions."""
    U, _ = _setup(seed=6)
    phi = synth.gaussian_spinor(D4, 7)
    p = _sw_params(ora, 4)
    F = ora.md_force(D4, U, p, phi)
    zero = np.zeros((256, 4, 8))
    h = 1e-4   # |S| ~ 7e3: rounding / h and truncation h^2 balance near here
    for (s, mu, a) in ((0, 0, 1), (77, 2, 4), (255, 3, 7), (130, 1, 0)):
        Sp = ora.hamiltonian(D4, H.lie_perturb(U, s, mu, a, h), zero, phi, p)
        Sm = ora.hamiltonian(D4, H.lie_perturb(U, s, mu, a, -h), zero, phi, p)
        assert abs((Sp - Sm) / (2 * h) - F[s, mu, a]) < 5e-7 * max(1.0, abs(F[s, mu, a]))
    # the parts add up
    Fg = ora.md_force(D4, U, p, phi, part=1)
    Ff = ora.md_force(D4, U, p, phi, part=2)
    assert H.rel(Fg + Ff, F) < 1e-14


def test_sexton_weingarten_reversible_and_reduces_to_leapfrog(ora):
    U, mom = _setup(seed=8)
    phi = synth.gaussian_spinor(D4, 9)
    p = _sw_params(ora, 3, n_inner=4, tau=0.5, tol=1e-14)
    U1, m1, _ = ora.md_integrate(D4, U, mom, phi, p)
    U2, m2, _ = ora.md_integrate(D4, U1, -m1, phi, p)
    assert H.rel(U2, U) < 1e-11 and H.rel(-m2, mom) < 1e-10
    # one inner step: the same kicks as leapfrog, merged differently
    p1 = _sw_params(ora, 4, n_inner=1, tau=0.5, tol=1e-14)
    pl = ora.hmc_params(5.7, 0.15, integrator="leapfrog", n_steps=4, tau=0.5, tol_md=1e-14, n_stout=1, rho=0.3)
    Ua, ma, _ = ora.md_integrate(D4, U, mom, phi, p1)
    Ub, mb, _ = ora.md_integrate(D4, U, mom, phi, pl)
    assert H.rel(Ua, Ub) < 1e-12 and H.rel(ma, mb) < 1e-11


def test_sexton_weingarten_stout_delta_h_dt_squared(ora):
    """The paper's second dynamical check (stout rho 0.3, Sexton-Weingarten with 10
    inner steps): |Delta H| scales as dt^2 in the outer step."""
    global ORA
    ORA = ora
    U, mom = _setup(seed=10)
    phi = synth.gaussian_spinor(D4, 11)
    ns = [4, 8, 16]
    dh = []
    for n in ns:
        p = _sw_params(ora, n)
        H0 = ora.hamiltonian(D4, U, mom, phi, p)
        U1, m1, _ = ora.md_integrate(D4, U, mom, phi, p)
        dh.append(abs(ora.hamiltonian(D4, U1, m1, phi, p) - H0))
    slope = np.polyfit(np.log(1.0 / np.array(ns)), np.log(dh), 1)[0]
    assert abs(slope - 2) < 0.25, (dh, slope)


def test_improved_gauge_energy_conservation(ora):
    """Pure-gauge HMC with the Iwasaki action: Delta H falls by ~4 when the step halves
    (second-order integrator on the rectangle force), and the oracle's force is the
    gradient of the action it integrates."""
    global ORA
    ORA = ora
    U, mom = _setup(seed=8)
    phi = np.zeros((256, 4, 3), np.complex128)
    p1 = ora.hmc_params(2.5, 0.0, fermions=False, n_steps=20, tau=1.0, c1=-0.331)
    p2 = ora.hmc_params(2.5, 0.0, fermions=False, n_steps=40, tau=1.0, c1=-0.331)
    d1, d2 = abs(_dH(U, mom, phi, p1)), abs(_dH(U, mom, phi, p2))
    assert 3.2 < d1 / d2 < 4.8


def test_clover_hmc_reversible_and_dt_squared(ora):
    """Wilson-clover fermions (c_sw = 1.5, full lattice): the integrator is reversible
    and Delta H falls by ~4 when the leapfrog step halves."""
    global ORA
    ORA = ora
    U, mom = _setup(seed=9)
    phi = synth.gaussian_spinor(D4, 10)
    p = ora.hmc_params(5.7, 0.13, integrator="leapfrog", n_steps=5, tau=0.5, tol_md=1e-14, csw=1.5)
    U1, m1, _ = ora.md_integrate(D4, U, mom, phi, p)
    U2, m2, _ = ora.md_integrate(D4, U1, -m1, phi, p)
    assert H.rel(U2, U) < 1e-11 and H.rel(-m2, mom) < 1e-10

    def energy(Ux, mx, pp):
        return (ora.gauge_action(D4, Ux, pp.beta) + ora.momentum_energy(D4, mx)
                + ora.pf_action_sw(D4, Ux, pp.kappa, pp.csw, phi, tol=1e-14)[0])

    dh = []
    for n in (10, 20):
        pp = ora.hmc_params(5.7, 0.13, integrator="leapfrog", n_steps=n, tau=1.0, tol_md=1e-14, csw=1.5)
        Ux, mx, _ = ora.md_integrate(D4, U, mom, phi, pp)
        dh.append(abs(energy(Ux, mx, pp) - energy(U, mom, pp)))
    assert 3.2 < dh[0] / dh[1] < 4.8, dh


def test_even_odd_clover_hmc_reversible_and_dt_squared(ora):
    """Even-odd Wilson-clover fermions (c_sw = 1.5; the action carries -2 ln det M_oo):
    the integrator is reversible, Delta H falls by ~4 when the leapfrog step halves, and a
    trajectory's S_f(old) is xi^+ xi - 2 ln det M_oo."""
    global ORA
    ORA = ora
    U, mom = _setup(seed=11)
    phi = synth.gaussian_spinor(D4, 12, parity_mask=1)
    p = ora.hmc_params(5.7, 0.13, eo=True, integrator="leapfrog", n_steps=5, tau=0.5, tol_md=1e-14, csw=1.5)
    U1, m1, _ = ora.md_integrate(D4, U, mom, phi, p)
    U2, m2, _ = ora.md_integrate(D4, U1, -m1, phi, p)
    assert H.rel(U2, U) < 1e-11 and H.rel(-m2, mom) < 1e-10

    def energy(Ux, mx, pp):
        return (ora.gauge_action(D4, Ux, pp.beta) + ora.momentum_energy(D4, mx)
                + ora.pf_action_sw_eo(D4, Ux, pp.kappa, pp.csw, phi, tol=1e-14)[0])

    dh = []
    for n in (10, 20):
        pp = ora.hmc_params(5.7, 0.13, eo=True, integrator="leapfrog", n_steps=n, tau=1.0, tol_md=1e-14, csw=1.5)
        Ux, mx, _ = ora.md_integrate(D4, U, mom, phi, pp)
        dh.append(abs(energy(Ux, mx, pp) - energy(U, mom, pp)))
    assert 3.2 < dh[0] / dh[1] < 4.8, dh
    pt = ora.hmc_params(5.7, 0.13, eo=True, integrator="leapfrog", n_steps=4, tau=0.4, tol_md=1e-13,
                        tol_action=1e-13, csw=1.5)
    _, r = ora.hmc_trajectory(D4, U, pt, 21, 0)
    xi = ora.gaussian_spinor(D4, 21, 0, ora.FIELD_XI, 1)
    S_old = float(np.vdot(xi, xi).real) - 2 * ora.clover_logdet_odd(D4, U, 0.13, 1.5)
    assert abs(r["Sf_old"] - S_old) < 1e-10 * abs(S_old)
