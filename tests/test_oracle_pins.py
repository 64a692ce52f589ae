"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, library routines, algebraic identities,
dense brute force on tiny lattices, finite differences and symmetries.
"""
import os

import numpy as np
import pytest
import scipy.linalg

from paper_2602_20516_b300 import synth
from tests import helpers as H

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ random numbers
def test_philox_known_answers(ora):
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = ora.philox4x32_10(v[0:4], v[4:6])
        assert [int(o) for o in out] == v[6:10]


def test_gaussian_moments(ora):
    g = np.array([ora.gauss_pair(7, i, 0, 0, 1) for i in range(20000)]).ravel()
    assert abs(g.mean()) < 0.03 and abs(g.var() - 1) < 0.03
    # fourth moment of N(0,1) is 3
    assert abs((g ** 4).mean() - 3) < 0.15


# ------------------------------------------------------------------ small matrices
def test_gamma_algebra(ora):
    g = [ora.gamma(m) for m in range(4)]
    g5 = ora.gamma(4)
    for m in range(4):
        assert np.allclose(g[m], g[m].conj().T)
        for n in range(4):
            assert np.allclose(g[m] @ g[n] + g[n] @ g[m], 2 * (m == n) * np.eye(4))
        assert np.allclose(g5 @ g[m] + g[m] @ g5, 0)
    assert np.allclose(g5, np.diag([1, 1, -1, -1]))


def test_gellmann(ora):
    T = [ora.gellmann_T(a) for a in range(8)]
    for a in range(8):
        assert np.allclose(T[a], T[a].conj().T) and abs(np.trace(T[a])) < 1e-15
        for b in range(8):
            assert abs(np.trace(T[a] @ T[b]) - 0.5 * (a == b)) < 1e-15
    # structure constants f_123 = 1, f_458 = sqrt(3)/2
    assert np.allclose(T[0] @ T[1] - T[1] @ T[0], 1j * T[2])
    assert np.allclose(T[3] @ T[4] - T[4] @ T[3], 1j * (0.5 * T[2] + np.sqrt(3) / 2 * T[7]))


@pytest.mark.parametrize("n", [3, 6])
def test_expm_matches_library(ora, n):
    rng = np.random.default_rng(n)
    for scale in (1e-3, 0.5, 3.0):
        A = scale * (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
        assert H.rel(ora.expm(A), scipy.linalg.expm(A)) < 1e-13
    assert np.allclose(ora.expm(np.zeros((3, 3))), np.eye(3), atol=0)
    th = np.array([0.3, -1.1, 0.8])
    assert np.allclose(ora.expm(np.diag(1j * th)), np.diag(np.exp(1j * th)), atol=1e-15)


# ------------------------------------------------------------------ seeded links
def test_random_links_distribution(ora):
    d = (8, 8, 8, 8)
    U = ora.random_links(d, 11, 0.3)
    I3 = np.eye(3)
    assert np.abs(U @ np.conj(np.swapaxes(U, -1, -2)) - I3).max() < 1e-14
    assert np.abs(np.linalg.det(U) - 1).max() < 1e-14
    # independent links from an Ad-invariant law: <plaq> = c^4, c = E[Re tr U / 3],
    # with c estimated from an independent generator (numpy + eigh)
    W = synth.random_links((4, 4, 4, 4), 0.3, 5).reshape(-1, 3, 3)
    c = np.real(np.trace(W, axis1=-2, axis2=-1)).mean() / 3
    assert abs(ora.plaquette(d, U) - c ** 4) < 0.01


# ------------------------------------------------------------------ Wilson-Dirac operator
@pytest.mark.parametrize("n", [(0, 0, 0, 0), (1, 0, 2, 1), (3, 1, 1, 0)])
def test_free_field_plane_wave(ora, n):
    d = (4, 4, 4, 4)
    kappa = 0.15
    U = np.broadcast_to(np.eye(3), (256, 4, 3, 3)).copy()
    u = np.random.default_rng(1).standard_normal((4, 3)) + 0j
    psi, p = H.plane_wave(d, n, u)
    g = [ora.gamma(m) for m in range(4)]
    # D e^{ipx} u = [(1 - 2 kappa sum cos p) + 2 i kappa sum gamma sin p] e^{ipx} u
    M = (1 - 2 * kappa * np.cos(p).sum()) * np.eye(4) + 2j * kappa * sum(
        g[m] * np.sin(p[m]) for m in range(4))
    expect = np.einsum("ab,xbc->xac", M, psi)
    assert H.rel(ora.dirac(d, U, kappa, psi), expect) < 1e-14


def test_gamma5_hermiticity_and_adjoint(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 3)
    kappa = 0.15
    phi = synth.gaussian_spinor(d, 4)
    psi = synth.gaussian_spinor(d, 5)
    g5 = np.diag([1, 1, -1, -1])
    g5psi = np.einsum("ab,xbc->xac", g5, psi)
    lhs = np.einsum("ab,xbc->xac", g5, ora.dirac(d, U, kappa, g5psi))
    assert H.rel(lhs, ora.dirac(d, U, kappa, psi, dagger=True)) < 1e-14
    a = np.vdot(phi, ora.dirac(d, U, kappa, psi))
    b = np.vdot(ora.dirac(d, U, kappa, phi, dagger=True), psi)
    assert abs(a - b) / abs(a) < 1e-13


def test_gauge_covariance_of_D(ora):
    d = (4, 4, 4, 4)
    V = 256
    U = synth.random_links(d, 0.5, 6)
    g = synth.random_su3(V, 7)
    psi = synth.gaussian_spinor(d, 8)
    Ug = H.gauge_transform_links(d, U, g)
    lhs = ora.dirac(d, Ug, 0.13, H.gauge_transform_spinor(psi, g))
    rhs = H.gauge_transform_spinor(ora.dirac(d, U, 0.13, psi), g)
    assert H.rel(lhs, rhs) < 1e-14


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 2, 2, 2)])
def test_even_odd_determinant_and_schur(ora, dims):
    V = synth.volume(dims)
    U = synth.random_links(dims, 0.6, 9)
    kappa = 0.2
    Dm = H.dense_operator(lambda e: ora.dirac(dims, U, kappa, e), V)
    even = np.where(synth.parity(dims) == 0)[0]
    Dh = H.dense_operator(lambda e: ora.dhat(dims, U, kappa, e), V, sites=even)
    Dh = Dh.reshape(V, 12, -1)[even].reshape(len(even) * 12, -1)
    s1, l1 = np.linalg.slogdet(Dm)
    s2, l2 = np.linalg.slogdet(Dh)
    assert abs(l1 - l2) < 1e-10 and abs(s1 - s2) < 1e-10
    # full solve equals the even-odd reconstruction
    b = synth.gaussian_spinor(dims, 10)
    x_full = np.linalg.solve(Dm, b.ravel()).reshape(V, 4, 3)
    be = b.copy(); be[synth.parity(dims) == 1] = 0
    bo = b - be
    rhs = be + kappa * ora.hop(dims, U, bo, out_mask=1)
    xe = np.linalg.solve(Dh, rhs[even].ravel()).reshape(-1, 4, 3)
    x = np.zeros_like(b); x[even] = xe
    x = x + bo + kappa * ora.hop(dims, U, x, out_mask=2)
    assert H.rel(x, x_full) < 1e-12
    # Dhat^+ = gamma5 Dhat gamma5
    g5 = np.diag([1, 1, -1, -1])
    psi = synth.gaussian_spinor(dims, 11, parity_mask=1)
    lhs = np.einsum("ab,xbc->xac", g5, ora.dhat(dims, U, kappa, np.einsum("ab,xbc->xac", g5, psi)))
    assert H.rel(lhs, ora.dhat(dims, U, kappa, psi, dagger=True)) < 1e-14


# ------------------------------------------------------------------ solver and S_F
@pytest.mark.parametrize("eo", [False, True])
def test_cg_true_residual(ora, eo):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 12)
    b = synth.gaussian_spinor(d, 13, parity_mask=1 if eo else 3)
    x, it, res = ora.cg(d, U, 0.15, b, eo=eo, tol=1e-12)
    assert it > 0 and res <= 1e-12
    M = (lambda v, dag=False: ora.dhat(d, U, 0.15, v, dag)) if eo else \
        (lambda v, dag=False: ora.dirac(d, U, 0.15, v, dag))
    assert H.rel(M(M(x), True), b) <= 1.5e-12


def test_pf_action_free_field_closed_form(ora):
    d = (4, 4, 4, 6)
    kappa = 0.12
    V = synth.volume(d)
    U = np.broadcast_to(np.eye(3), (V, 4, 3, 3)).copy()
    phi = synth.gaussian_spinor(d, 14)
    S, _ = ora.pf_action(d, U, kappa, phi, tol=1e-13)
    # unitary DFT with antiperiodic time: phi~(p) = V^-1/2 sum_x e^{-ipx} phi(x)
    c = synth.coords(d)
    f = phi * np.exp(-1j * np.pi * c[:, 3] / d[3])[:, None, None]
    f = f.reshape(d[3], d[2], d[1], d[0], 12)
    ft = np.fft.fftn(f, axes=(0, 1, 2, 3), norm="ortho")
    k = [2 * np.pi * np.fft.fftfreq(L) for L in (d[3], d[2], d[1], d[0])]
    p3, p2, p1, p0 = np.meshgrid(k[0] + np.pi / d[3], k[1], k[2], k[3], indexing="ij")
    cs = np.cos(p0) + np.cos(p1) + np.cos(p2) + np.cos(p3)
    s2 = np.sin(p0) ** 2 + np.sin(p1) ** 2 + np.sin(p2) ** 2 + np.sin(p3) ** 2
    lam = (1 - 2 * kappa * cs) ** 2 + 4 * kappa ** 2 * s2
    S_exact = (np.abs(ft) ** 2 / lam[..., None]).sum()
    assert abs(S - S_exact) / S_exact < 1e-12


@pytest.mark.parametrize("eo", [False, True])
def test_pf_action_dense_and_heatbath(ora, eo):
    d = (2, 2, 2, 4)
    V = synth.volume(d)
    U = synth.random_links(d, 0.5, 15)
    kappa = 0.16
    mask = 1 if eo else 3
    phi = synth.gaussian_spinor(d, 16, parity_mask=mask)
    if eo:
        even = np.where(synth.parity(d) == 0)[0]
        M = H.dense_operator(lambda e: ora.dhat(d, U, kappa, e), V, sites=even)
        M = M.reshape(V, 12, -1)[even].reshape(len(even) * 12, -1)
        pv = phi[even].ravel()
    else:
        M = H.dense_operator(lambda e: ora.dirac(d, U, kappa, e), V)
        pv = phi.ravel()
    S_dense = np.real(np.vdot(pv, np.linalg.solve(M.conj().T @ M, pv)))
    S, _ = ora.pf_action(d, U, kappa, phi, eo=eo, tol=1e-13)
    assert abs(S - S_dense) / S_dense < 1e-12
    # heatbath identity: phi = M^+ xi gives S_f = xi^+ xi
    xi = synth.gaussian_spinor(d, 17, parity_mask=mask)
    ph = ora.dhat(d, U, kappa, xi, True) if eo else ora.dirac(d, U, kappa, xi, True)
    S2, _ = ora.pf_action(d, U, kappa, ph, eo=eo, tol=1e-13)
    assert abs(S2 - np.vdot(xi, xi).real) / S2 < 1e-12


def test_gauge_invariance_of_actions(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 18)
    g = synth.random_su3(256, 19)
    Ug = H.gauge_transform_links(d, U, g)
    assert abs(ora.gauge_action(d, U, 5.7) - ora.gauge_action(d, Ug, 5.7)) < 1e-10
    for eo in (False, True):
        phi = synth.gaussian_spinor(d, 20, parity_mask=1 if eo else 3)
        S1, _ = ora.pf_action(d, U, 0.15, phi, eo=eo, tol=1e-13)
        S2, _ = ora.pf_action(d, Ug, 0.15, H.gauge_transform_spinor(phi, g), eo=eo, tol=1e-13)
        assert abs(S1 - S2) / abs(S1) < 1e-12
    # S_G(U = 1) = 0
    one = np.broadcast_to(np.eye(3), (256, 4, 3, 3)).copy()
    assert ora.gauge_action(d, one, 5.7) == 0.0


# ------------------------------------------------------------------ forces
LINKS = [(0, 0), (37, 1), (100, 2), (255, 3), (3, 3), (64 + 5, 3)]


def test_gauge_force_finite_difference(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 21)
    beta = 5.7
    F = ora.gauge_force(d, U, beta)
    h = 1e-5
    for (s, mu) in LINKS:
        for a in (0, 3, 7):
            Sp = ora.gauge_action(d, H.lie_perturb(U, s, mu, a, h), beta)
            Sm = ora.gauge_action(d, H.lie_perturb(U, s, mu, a, -h), beta)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 1e-6 * max(1.0, abs(F[s, mu, a]))


@pytest.mark.parametrize("eo", [False, True])
def test_fermion_force_finite_difference(ora, eo):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 22)
    kappa = 0.15
    phi = synth.gaussian_spinor(d, 23, parity_mask=1 if eo else 3)
    F, _ = ora.pf_force(d, U, kappa, phi, eo=eo, tol=1e-14)
    h = 1e-5
    for (s, mu) in LINKS:
        for a in (1, 4, 7):
            Sp, _ = ora.pf_action(d, H.lie_perturb(U, s, mu, a, h), kappa, phi, eo=eo, tol=1e-14)
            Sm, _ = ora.pf_action(d, H.lie_perturb(U, s, mu, a, -h), kappa, phi, eo=eo, tol=1e-14)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 2e-6 * max(1.0, abs(F[s, mu, a]))


def test_force_covariance(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 24)
    g = synth.random_su3(256, 25)
    Ug = H.gauge_transform_links(d, U, g)
    phi = synth.gaussian_spinor(d, 26)
    F = ora.gauge_force(d, U, 5.7) + ora.pf_force(d, U, 0.15, phi, tol=1e-13)[0]
    Fg = ora.gauge_force(d, Ug, 5.7) + ora.pf_force(d, Ug, 0.15, H.gauge_transform_spinor(phi, g), tol=1e-13)[0]
    assert H.rel(Fg, H.gauge_transform_adjoint(F, g)) < 1e-11


def test_real_component_gradients(ora):
    """G = dS/dReU + i dS/dImU (Eq. S2.11) by finite differences on matrix entries,
    and F_a = Re tr(G^+ i T^a U) reproduces the Lie force."""
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 27)
    phi = synth.gaussian_spinor(d, 28)
    # S_f is a global sum of ~1e3: its rounding (~1e-11) over 2h sets the step
    beta, kappa, h = 5.7, 0.15, 3e-5
    Gg = ora.gauge_action_grad(d, U, beta)
    Gf, _ = ora.pf_action_grad(d, U, kappa, phi, tol=1e-14)
    for (s, mu) in LINKS[:3]:
        for (i, j) in ((0, 0), (1, 2), (2, 1)):
            for part, unit in (("re", 1.0), ("im", 1j)):
                Up = U.copy(); Up[s, mu, i, j] += h * unit
                Um = U.copy(); Um[s, mu, i, j] -= h * unit
                fd_g = (ora.gauge_action(d, Up, beta) - ora.gauge_action(d, Um, beta)) / (2 * h)
                fd_f = (ora.pf_action(d, Up, kappa, phi, tol=1e-14)[0]
                        - ora.pf_action(d, Um, kappa, phi, tol=1e-14)[0]) / (2 * h)
                ga = Gg[s, mu, i, j].real if part == "re" else Gg[s, mu, i, j].imag
                fa = Gf[s, mu, i, j].real if part == "re" else Gf[s, mu, i, j].imag
                assert abs(fd_g - ga) < 2e-6 * max(1, abs(ga))
                assert abs(fd_f - fa) < 3e-6 * max(1, abs(fa))
    assert H.rel(ora.grad_to_force(d, U, Gg), ora.gauge_force(d, U, beta)) < 1e-13
    assert H.rel(ora.grad_to_force(d, U, Gf), ora.pf_force(d, U, kappa, phi, tol=1e-14)[0]) < 1e-12


# ------------------------------------------------------------------ link update
def test_link_update_unitarity_and_inverse(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 29)
    mom = synth.gaussian_momenta(d, 30)
    U1 = ora.update_links(d, U, mom, 0.3)
    I3 = np.eye(3)
    assert np.abs(U1 @ np.conj(np.swapaxes(U1, -1, -2)) - I3).max() < 1e-14
    assert np.abs(np.linalg.det(U1) - 1).max() < 1e-14
    assert H.rel(ora.update_links(d, U1, mom, -0.3), U) < 1e-14
    # independent route: scipy expm of i eps Pi
    P = np.einsum("xma,aij->xmij", mom, H.GELLMANN_T)
    s, mu = 77, 2
    assert H.rel(U1[s, mu], scipy.linalg.expm(0.3j * P[s, mu]) @ U[s, mu]) < 1e-14


def test_reunitarise(ora):
    d = (2, 2, 2, 2)
    U = synth.random_links(d, 0.5, 31)
    assert H.rel(ora.reunitarise(d, U), U) < 1e-15
    W = U + 1e-6 * (np.random.default_rng(0).standard_normal(U.shape))
    R = ora.reunitarise(d, W)
    assert np.abs(R @ np.conj(np.swapaxes(R, -1, -2)) - np.eye(3)).max() < 1e-15
    assert np.abs(np.linalg.det(R) - 1).max() < 1e-15


# ------------------------------------------------------------------ stout smearing
def test_stout_identity_at_rho_zero(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 32)
    G = synth.random_links(d, 1.0, 33)  # any complex matrices
    assert H.rel(ora.stout_forward(d, U, 0.0), U) < 1e-15
    assert H.rel(ora.stout_backward(d, U, 0.0, G), G) < 1e-14


def test_stout_unitary_and_covariant(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 34)
    S = ora.stout_forward(d, U, 0.1)
    assert np.abs(S @ np.conj(np.swapaxes(S, -1, -2)) - np.eye(3)).max() < 1e-14
    assert np.abs(np.linalg.det(S) - 1).max() < 1e-14
    g = synth.random_su3(256, 35)
    lhs = ora.stout_forward(d, H.gauge_transform_links(d, U, g), 0.1)
    assert H.rel(lhs, H.gauge_transform_links(d, S, g)) < 1e-13


def test_stout_rho_derivative_is_gauge_flow(ora):
    """One stout level is U' = exp(rho P[(U V)^+]) U with V the force staple, i.e. a
    step of the gradient flow of S_G: dS_G(smear_rho U)/drho at rho = 0 equals
    sum_{x,mu,a} F_a (-2 Im tr T^a U V) = -(6 / beta) sum F_a^2, with F the gauge
    force (itself pinned by finite differences).  A central difference in rho checks
    the sign and scale of Q, the staple orientation and the projection."""
    d = (4, 4, 4, 4)
    beta = 5.8
    U = synth.random_links(d, 0.5, 39)
    F = ora.gauge_force(d, U, beta)
    want = -(6.0 / beta) * float(np.sum(F * F))
    h = 1e-4
    fd = (ora.gauge_action(d, ora.stout_forward(d, U, h), beta)
          - ora.gauge_action(d, ora.stout_forward(d, U, -h), beta)) / (2 * h)
    assert abs(fd - want) < 1e-6 * abs(want), (fd, want)
    # a flow step lowers the action
    assert ora.gauge_action(d, ora.stout_forward(d, U, 0.01), beta) < ora.gauge_action(d, U, beta)


def test_stout_closed_form_abelian_field(ora):
    """Diagonal (abelian) links U_mu(x) = diag(exp(i th_mu,k(x))), sum_k th = 0: every
    product is diagonal, so one stout level moves each phase by
    rho sum_nu [sin phi_munu,k(x - nu) - sin phi_munu,k(x)] minus its colour mean,
    phi_munu(x) = th_mu(x) + th_nu(x + mu) - th_mu(x + nu) - th_nu(x) the plaquette
    angle (scalar trigonometry; no matrix code)."""
    d = (4, 6, 4, 8)
    V = synth.volume(d)
    rng = np.random.default_rng(41)
    th = rng.uniform(-1.2, 1.2, size=(V, 4, 3))
    th -= th.mean(axis=2, keepdims=True)
    U = np.zeros((V, 4, 3, 3), np.complex128)
    for k in range(3):
        U[:, :, k, k] = np.exp(1j * th[:, :, k])
    rho = 0.13
    shift = np.zeros_like(th)
    for mu in range(4):
        xpmu = H.neighbour(d, mu, +1)
        for nu in range(4):
            if nu == mu:
                continue
            xpnu, xmnu = H.neighbour(d, nu, +1), H.neighbour(d, nu, -1)
            phi = th[:, mu] + th[xpmu, nu] - th[xpnu, mu] - th[:, nu]
            shift[:, mu] += rho * (np.sin(phi[xmnu]) - np.sin(phi))
    shift -= shift.mean(axis=2, keepdims=True)
    want = np.zeros_like(U)
    for k in range(3):
        want[:, :, k, k] = np.exp(1j * (th[:, :, k] + shift[:, :, k]))
    assert H.rel(ora.stout_forward(d, U, rho), want) < 1e-14


def test_stout_backward_finite_difference(ora):
    """L(U) = Re tr sum A^+ smear(U): its gradient is the backward of G' = A."""
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 36)
    rho = 0.1
    A = synth.random_links(d, 1.0, 37) + 0.3 * synth.random_links(d, 1.0, 38)

    def L(W):
        return np.real(np.vdot(A, ora.stout_forward(d, W, rho)))

    G = ora.stout_backward(d, U, rho, A)
    h = 1e-4  # central-difference error is smallest here (truncation ~ rounding)
    for (s, mu) in LINKS[:4]:
        for (i, j) in ((0, 1), (2, 2)):
            for unit, part in ((1.0, np.real), (1j, np.imag)):
                Up = U.copy(); Up[s, mu, i, j] += h * unit
                Um = U.copy(); Um[s, mu, i, j] -= h * unit
                fd = (L(Up) - L(Um)) / (2 * h)
                assert abs(fd - part(G[s, mu, i, j])) < 2e-8 * max(1, abs(fd))


# ------------------------------------------------------------------ rectangle-improved gauge action
IWASAKI = -0.331


def test_improved_action_closed_form_abelian_field(ora):
    """U_1(x) = exp(i phi x_0 H), H = diag(1, -1, 0), phi = 2 pi / L_0, other links 1:
    every (0,1) plaquette is exp(i phi H) and both (0,1) rectangles exp(+-2 i phi H),
    all other loops are 1, so sum Re tr P / 3 = V (5 + (1 + 2 cos phi) / 3) and
    sum Re tr R / 3 = V (10 + 2 (1 + 2 cos 2 phi) / 3)."""
    d = (6, 4, 4, 4)
    V = int(np.prod(d))
    phi = 2 * np.pi / d[0]
    x0 = synth.coords(d)[:, 0]
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    for s in range(V):
        U[s, 1] = np.diag(np.exp(1j * phi * x0[s] * np.array([1.0, -1.0, 0.0])))
    P = V * (5 + (1 + 2 * np.cos(phi)) / 3)
    R = V * (10 + 2 * (1 + 2 * np.cos(2 * phi)) / 3)
    assert abs(ora.plaquette_sum(d, U) - P) < 1e-11 * P
    assert abs(ora.rectangle_sum(d, U) - R) < 1e-11 * R
    beta = 2.5
    for c1 in (-1.0 / 12, IWASAKI, -1.4088):
        want = beta * ((1 - 8 * c1) * (6 * V - P) + c1 * (12 * V - R))
        assert abs(ora.gauge_action(d, U, beta, c1) - want) < 1e-10 * abs(want)


def test_improved_action_invariance_and_unit_field(ora):
    d = (4, 4, 4, 6)
    V = int(np.prod(d))
    U = synth.random_links(d, 0.5, 81)
    g = synth.random_su3(V, 82)
    Ug = H.gauge_transform_links(d, U, g)
    S = ora.gauge_action(d, U, 2.5, IWASAKI)
    assert abs(S - ora.gauge_action(d, Ug, 2.5, IWASAKI)) < 1e-12 * abs(S)
    one = np.broadcast_to(np.eye(3), (V, 4, 3, 3)).copy()
    assert ora.gauge_action(d, one, 2.5, IWASAKI) == 0.0
    # the rectangle term is not the plaquette term: the two sums differ on a random field
    assert abs(ora.rectangle_sum(d, U) / (12 * V) - ora.plaquette_sum(d, U) / (6 * V)) > 1e-2


def test_improved_force_and_gradient_finite_difference(ora):
    """Lie force (central differences in Lie directions) and real-component gradient
    (central differences on matrix entries) of the Iwasaki action, including links
    whose rectangles wrap around the lattice."""
    d = (4, 4, 4, 6)
    U = synth.random_links(d, 0.5, 83)
    beta = 2.5
    F = ora.gauge_force(d, U, beta, IWASAKI)
    G = ora.gauge_action_grad(d, U, beta, IWASAKI)
    h = 1e-5
    for (s, mu) in [(0, 0), (37, 1), (100, 2), (383, 3), (3, 3)]:
        for a in (0, 4, 7):
            Sp = ora.gauge_action(d, H.lie_perturb(U, s, mu, a, h), beta, IWASAKI)
            Sm = ora.gauge_action(d, H.lie_perturb(U, s, mu, a, -h), beta, IWASAKI)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 2e-6 * max(1.0, abs(F[s, mu, a]))
    for (s, mu) in [(5, 1), (200, 3)]:
        for (i, j) in ((0, 0), (1, 2)):
            for unit, part in ((1.0, "re"), (1j, "im")):
                Up = U.copy(); Up[s, mu, i, j] += h * unit
                Um = U.copy(); Um[s, mu, i, j] -= h * unit
                fd = (ora.gauge_action(d, Up, beta, IWASAKI) - ora.gauge_action(d, Um, beta, IWASAKI)) / (2 * h)
                ga = G[s, mu, i, j].real if part == "re" else G[s, mu, i, j].imag
                assert abs(fd - ga) < 2e-6 * max(1.0, abs(ga))
    assert H.rel(ora.grad_to_force(d, U, G), F) < 1e-13


# ------------------------------------------------------------------ clover (Sheikholeslami-Wohlert) term
def _chiral_gammas():
    """g_k = [[0, -i s_k], [i s_k, 0]] (mu = k - 1), g_4 = [[0, 1], [1, 0]], built here
    from the Pauli matrices, independently of the oracle."""
    s = [np.array([[0, 1], [1, 0]], complex), np.array([[0, -1j], [1j, 0]]), np.array([[1, 0], [0, -1]], complex)]
    z = np.zeros((2, 2))
    g = [np.block([[z, -1j * sk], [1j * sk, z]]) for sk in s]
    g.append(np.block([[z, np.eye(2)], [np.eye(2), z]]))
    return g


def _abelian_field(d, n=1):
    V = int(np.prod(d))
    phi = 2 * np.pi * n / d[0]
    x0 = synth.coords(d)[:, 0]
    U = np.broadcast_to(np.eye(3, dtype=np.complex128), (V, 4, 3, 3)).copy()
    for s_ in range(V):
        U[s_, 1] = np.diag(np.exp(1j * phi * x0[s_] * np.array([1.0, -1.0, 0.0])))
    return U, phi


def test_clover_abelian_field_closed_form(ora):
    """U_1(x) = exp(i phi x_0 H): all four leaves of the (0,1) plane are exp(i phi H),
    so F_01 = sin(phi H) = diag(sin phi, -sin phi, 0) at every site and the other
    planes vanish; D_sw - D = -kappa c_sw sigma_01 (x) F_01."""
    d = (6, 4, 4, 4)
    V = int(np.prod(d))
    U, phi = _abelian_field(d)
    F01 = ora.clover_field_strength(d, U, 0, 1)
    want = np.diag([np.sin(phi), -np.sin(phi), 0.0])
    assert np.abs(F01 - want).max() < 1e-14
    for (mu, nu) in ((0, 2), (1, 3), (2, 3)):
        assert np.abs(ora.clover_field_strength(d, U, mu, nu)).max() < 1e-14
    g = _chiral_gammas()
    sig01 = 0.5j * (g[0] @ g[1] - g[1] @ g[0])
    kappa, csw = 0.13, 1.7
    psi = synth.gaussian_spinor(d, 84)
    diff = ora.dirac_sw(d, U, kappa, csw, psi) - ora.dirac(d, U, kappa, psi)
    expect = -kappa * csw * np.einsum("st,ab,xtb->xsa", sig01, want, psi)
    assert np.abs(diff - expect).max() < 1e-13


def test_clover_hermiticity_covariance_and_unit_field(ora):
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 85)
    kappa, csw = 0.13, 1.5
    phi, psi = synth.gaussian_spinor(d, 86), synth.gaussian_spinor(d, 87)
    Dpsi = ora.dirac_sw(d, U, kappa, csw, psi)
    Ddphi = ora.dirac_sw(d, U, kappa, csw, phi, dagger=True)
    assert abs(np.vdot(phi, Dpsi) - np.vdot(Ddphi, psi)) < 1e-12 * abs(np.vdot(phi, Dpsi))
    g5 = np.diag([1, 1, -1, -1])
    g5D = np.einsum("st,xtc->xsc", g5, ora.dirac_sw(d, U, kappa, csw, np.einsum("st,xtc->xsc", g5, psi)))
    assert H.rel(g5D, ora.dirac_sw(d, U, kappa, csw, psi, dagger=True)) < 1e-14
    gt = synth.random_su3(256, 88)
    Ug = H.gauge_transform_links(d, U, gt)
    lhs = ora.dirac_sw(d, Ug, kappa, csw, H.gauge_transform_spinor(psi, gt))
    assert H.rel(lhs, H.gauge_transform_spinor(Dpsi, gt)) < 1e-13
    one = np.broadcast_to(np.eye(3), (256, 4, 3, 3)).copy()
    assert H.rel(ora.dirac_sw(d, one, kappa, csw, psi), ora.dirac(d, one, kappa, psi)) < 1e-15
    # the clover term is Hermitian and traceless in spin at every site
    A = ora.clover_term(d, U, kappa, csw)
    assert np.abs(A - np.conj(np.swapaxes(A, 1, 2))).max() < 1e-15
    assert np.abs(np.einsum("xii->x", A)).max() < 1e-13


def test_clover_force_and_gradient_finite_difference(ora):
    """S_f = phi^+ (D_sw^+ D_sw)^{-1} phi: the Lie force against central differences in
    Lie directions, and the real-component gradient against differences on entries."""
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 89)
    kappa, csw = 0.13, 1.5
    phi = synth.gaussian_spinor(d, 90)
    F, _ = ora.pf_force_sw(d, U, kappa, csw, phi, tol=1e-14)
    h = 1e-5
    for (s, mu) in LINKS:
        for a in (1, 4, 7):
            Sp, _ = ora.pf_action_sw(d, H.lie_perturb(U, s, mu, a, h), kappa, csw, phi, tol=1e-14)
            Sm, _ = ora.pf_action_sw(d, H.lie_perturb(U, s, mu, a, -h), kappa, csw, phi, tol=1e-14)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 2e-6 * max(1.0, abs(F[s, mu, a]))
    G, _ = ora.pf_action_grad_sw(d, U, kappa, csw, phi, tol=1e-14)
    h = 3e-5
    for (s, mu) in LINKS[:2]:
        for (i, j) in ((0, 1), (2, 2)):
            for unit, part in ((1.0, "re"), (1j, "im")):
                Up = U.copy(); Up[s, mu, i, j] += h * unit
                Um = U.copy(); Um[s, mu, i, j] -= h * unit
                fd = (ora.pf_action_sw(d, Up, kappa, csw, phi, tol=1e-14)[0]
                      - ora.pf_action_sw(d, Um, kappa, csw, phi, tol=1e-14)[0]) / (2 * h)
                ga = G[s, mu, i, j].real if part == "re" else G[s, mu, i, j].imag
                assert abs(fd - ga) < 3e-6 * max(1.0, abs(ga))
    # c_sw = 0 is the Wilson force
    F0, _ = ora.pf_force_sw(d, U, kappa, 0.0, phi, tol=1e-14)
    assert H.rel(F0, ora.pf_force(d, U, kappa, phi, tol=1e-14)[0]) < 1e-10


# ---------------------------------------------------------------- even-odd clover
def _dense(apply, n):
    """Dense matrix of a linear map on C^n from its action on the unit vectors."""
    M = np.zeros((n, n), np.complex128)
    for k in range(n):
        e = np.zeros(n, np.complex128)
        e[k] = 1.0
        M[:, k] = apply(e)
    return M


def test_clover_even_odd_schur_complement_and_determinant(ora):
    """On a 2x2x2x4 lattice the dense clover operator D is built column by column; with
    sites ordered even then odd, its Schur complement D_ee - D_eo D_oo^{-1} D_oe (numpy)
    is the oracle's Dhat, det D = det D_oo det Dhat, and ln det D_oo is the oracle's sum
    over odd sites of ln det (1 + A) (D_oo is site-diagonal: no hop joins two odd sites)."""
    d = (2, 2, 2, 4)
    V = int(np.prod(d))
    U = synth.random_links(d, 0.5, 301)
    kappa, csw = 0.13, 1.7
    par = synth.parity(d)
    ev, od = np.where(par == 0)[0], np.where(par == 1)[0]

    def full_apply(vec):
        return ora.dirac_sw(d, U, kappa, csw, vec.reshape(V, 4, 3)).reshape(-1)

    D = _dense(full_apply, V * 12)
    idx_e = (ev[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
    idx_o = (od[:, None] * 12 + np.arange(12)[None, :]).reshape(-1)
    Dee, Deo = D[np.ix_(idx_e, idx_e)], D[np.ix_(idx_e, idx_o)]
    Doe, Doo = D[np.ix_(idx_o, idx_e)], D[np.ix_(idx_o, idx_o)]
    schur = Dee - Deo @ np.linalg.solve(Doo, Doe)

    def dhat_apply(vec):
        full = np.zeros(V * 12, np.complex128)
        full[idx_e] = vec
        return ora.dhat_sw(d, U, kappa, csw, full.reshape(V, 4, 3)).reshape(-1)[idx_e]

    Dhat = _dense(dhat_apply, len(idx_e))
    assert np.abs(Dhat - schur).max() < 1e-12 * np.abs(schur).max()
    s_full, l_full = np.linalg.slogdet(D)
    s_oo, l_oo = np.linalg.slogdet(Doo)
    s_hat, l_hat = np.linalg.slogdet(Dhat)
    assert abs(l_full - (l_oo + l_hat)) < 1e-9 * abs(l_full)
    assert abs(s_full - s_oo * s_hat) < 1e-9
    # D_oo = 1 + A_oo is Hermitian positive definite: det real positive
    assert abs(s_oo - 1.0) < 1e-12
    assert abs(ora.clover_logdet_odd(d, U, kappa, csw) - l_oo) < 1e-10 * abs(l_oo)
    # the adjoint: gamma5 Dhat gamma5 = Dhat^+
    def dhat_dag_apply(vec):
        full = np.zeros(V * 12, np.complex128)
        full[idx_e] = vec
        return ora.dhat_sw(d, U, kappa, csw, full.reshape(V, 4, 3), dagger=True).reshape(-1)[idx_e]
    assert np.abs(_dense(dhat_dag_apply, len(idx_e)) - Dhat.conj().T).max() < 1e-12 * np.abs(schur).max()


def test_clover_even_odd_action_force_finite_difference(ora):
    """S_f = phi_e^+ (Dhat^+ Dhat)^{-1} phi_e - 2 ln det M_oo: the Lie force against central
    differences in Lie directions (links on both parities, so the determinant term and both
    clover insertions are exercised), the real-component gradient against differences on
    entries, and c_sw = 0 giving the Wilson even-odd force."""
    d = (4, 4, 4, 4)
    U = synth.random_links(d, 0.5, 302)
    kappa, csw = 0.13, 1.5
    phi = synth.gaussian_spinor(d, 303, parity_mask=1)
    F, _ = ora.pf_force_sw_eo(d, U, kappa, csw, phi, tol=1e-14)
    h = 1e-5
    for (s, mu) in LINKS:
        for a in (0, 4, 7):
            Sp, _ = ora.pf_action_sw_eo(d, H.lie_perturb(U, s, mu, a, h), kappa, csw, phi, tol=1e-14)
            Sm, _ = ora.pf_action_sw_eo(d, H.lie_perturb(U, s, mu, a, -h), kappa, csw, phi, tol=1e-14)
            fd = (Sp - Sm) / (2 * h)
            assert abs(fd - F[s, mu, a]) < 2e-6 * max(1.0, abs(F[s, mu, a])), (s, mu, a, fd, F[s, mu, a])
    G, _ = ora.pf_action_grad_sw_eo(d, U, kappa, csw, phi, tol=1e-14)
    h = 3e-5
    for (s, mu) in LINKS[:2]:
        for (i, j) in ((0, 2), (1, 1)):
            for unit, part in ((1.0, "re"), (1j, "im")):
                Up = U.copy(); Up[s, mu, i, j] += h * unit
                Um = U.copy(); Um[s, mu, i, j] -= h * unit
                fd = (ora.pf_action_sw_eo(d, Up, kappa, csw, phi, tol=1e-14)[0]
                      - ora.pf_action_sw_eo(d, Um, kappa, csw, phi, tol=1e-14)[0]) / (2 * h)
                ga = G[s, mu, i, j].real if part == "re" else G[s, mu, i, j].imag
                assert abs(fd - ga) < 3e-6 * max(1.0, abs(ga))
    F0, _ = ora.pf_force_sw_eo(d, U, kappa, 0.0, phi, tol=1e-14)
    assert H.rel(F0, ora.pf_force(d, U, kappa, phi, eo=True, tol=1e-14)[0]) < 1e-10
    # the determinant term alone: its force is that of -2 sum_odd ln det M (phi = 0)
    Fd, _ = ora.pf_force_sw_eo(d, U, kappa, csw, np.zeros_like(phi), tol=1e-14)
    for (s, mu) in LINKS[:3]:
        a = 2
        Lp = ora.clover_logdet_odd(d, H.lie_perturb(U, s, mu, a, h), kappa, csw)
        Lm = ora.clover_logdet_odd(d, H.lie_perturb(U, s, mu, a, -h), kappa, csw)
        assert abs(-2 * (Lp - Lm) / (2 * h) - Fd[s, mu, a]) < 1e-6 * max(1.0, abs(Fd[s, mu, a]))
