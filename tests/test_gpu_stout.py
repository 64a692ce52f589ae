"""Stout smearing (forward and hand-written adjoint) and the autograd front end
on the GPU, against the oracle's independent adjoint (Van Loan block exponential)
and central finite differences of the action."""
import time

import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

DIMS = (8, 6, 4, 10)


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    L.lib()
    return L


def _np(t):
    return t.detach().cpu().numpy()


def _oracle_total_grad(ora, dims, U, beta, kappa, rho, n, phi, eo=False):
    levels = [U]
    for _ in range(n):
        levels.append(ora.stout_forward(dims, levels[-1], rho))
    G, _ = ora.pf_action_grad(dims, levels[-1], kappa, phi, eo=eo, tol=1e-13)
    for k in range(n, 0, -1):
        G = ora.stout_backward(dims, levels[k - 1], rho, G)
    return G + ora.gauge_action_grad(dims, U, beta)


@pytest.mark.parametrize("alpha", [0.5, 0.02])
def test_stout_forward_and_adjoint_vs_oracle(lgt, ora, alpha):
    """alpha = 0.02 makes Q small enough for the series branch of the adjoint."""
    U = synth.random_links(DIMS, alpha, 40)
    G = synth.random_links(DIMS, 1.0, 41) + 0.5 * synth.random_links(DIMS, 1.0, 42)
    lat = lgt.Lattice(DIMS)
    lat.set_links(U)
    for n in (1, 2):
        ref = U
        for _ in range(n):
            ref = ora.stout_forward(DIMS, ref, 0.1)
        assert H.rel(_np(lat.stout_smear(0.1, n)), ref) < 1e-14
        levels = [U]
        for _ in range(n):
            levels.append(ora.stout_forward(DIMS, levels[-1], 0.1))
        Gr = G
        for k in range(n, 0, -1):
            Gr = ora.stout_backward(DIMS, levels[k - 1], 0.1, Gr)
        for rc in (False, True):
            assert H.rel(_np(lat.stout_backward(0.1, n, G, recompute=rc)), Gr) < 1e-13


def test_stored_and_recomputed_stack_bitwise(lgt):
    U = synth.random_links(DIMS, 0.5, 43)
    G = synth.random_links(DIMS, 1.0, 44)
    lat = lgt.Lattice(DIMS)
    lat.set_links(U)
    for n in (2, 3):
        a = lat.stout_backward(0.1, n, G, recompute=False)
        b = lat.stout_backward(0.1, n, G, recompute=True)
        assert torch.equal(a, b)


@pytest.mark.parametrize("eo", [False, True])
def test_smeared_force_vs_oracle_and_autograd(lgt, ora, eo):
    from paper_2602_20516_b300 import autograd as AG
    beta, kappa, rho, n = 6.0, 0.15, 0.1, 2
    U = synth.random_links(DIMS, 0.5, 45)
    phi = synth.gaussian_spinor(DIMS, 46, parity_mask=1 if eo else 3)
    lat = lgt.Lattice(DIMS)
    lat.set_links(U)
    ap = lgt.action_params(beta=beta, kappa=kappa, even_odd=eo, n_stout=n, rho=rho)
    pf = lat.pack_spinor(phi, lgt.EVEN if eo else lgt.FULL, lgt.FP64)
    sp = lgt.solver("fp64", tol=1e-13)
    Gf, _ = lat.force(ap, pf, sp, form=lgt.GRAD_G)
    Gf = _np(lat.unpack_grad(Gf))
    Go = _oracle_total_grad(ora, DIMS, U, beta, kappa, rho, n, phi, eo)
    assert H.rel(Gf, Go) < 1e-10
    # Lie form of the fused path equals grad_to_lie of the G form
    F, _ = lat.force(ap, pf, sp, form=lgt.FORCE_LIE)
    assert H.rel(_np(lat.unpack_momenta(F)), ora.grad_to_force(DIMS, U, Go)) < 1e-10
    # autograd: S_G(U) + S_f(smear^2(U))
    Ut = torch.tensor(U, device="cuda", requires_grad=True)
    phit = torch.tensor(phi, device="cuda")
    S = AG.total_action(Ut, phit, lat, beta, kappa, n_stout=n, rho=rho, even_odd=eo, solver=sp)
    S.backward()
    assert H.rel(_np(Ut.grad), Gf) < 1e-12
    Sg = ora.gauge_action(DIMS, U, beta)
    Us = ora.stout_forward(DIMS, ora.stout_forward(DIMS, U, rho), rho)
    Sf, _ = ora.pf_action(DIMS, Us, kappa, phi, eo=eo, tol=1e-13)
    assert abs(S.item() - (Sg + Sf)) / (Sg + Sf) < 1e-12


def test_config3_16x4_finite_differences_and_memory(lgt, ora):
    """16^4, beta 6.0, kappa 0.15, 2-level stout rho 0.1 in front of the Wilson
    operator (full-lattice S_f): autograd gradient vs the oracle and vs central FD
    (eps = 1e-5, FP64) in Lie directions; stored vs recomputed smearing stack."""
    from paper_2602_20516_b300 import autograd as AG
    dims = (16, 16, 16, 16)
    beta, kappa, rho, n = 6.0, 0.15, 0.1, 2
    U = synth.random_links(dims, 0.5, 3)
    phi = synth.gaussian_spinor(dims, 47)
    sp = lgt.solver("fp64", tol=1e-13)
    res = {}
    for rc in (False, True):
        lat = lgt.Lattice(dims)
        Ut = torch.tensor(U, device="cuda", requires_grad=True)
        phit = torch.tensor(phi, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S = AG.total_action(Ut, phit, lat, beta, kappa, n_stout=n, rho=rho, solver=sp, recompute=rc)
        S.backward()
        torch.cuda.synchronize()
        res[rc] = (_np(Ut.grad), S.item(), lat.info()[1], time.perf_counter() - t0)
        if not rc:
            keep = lat
    assert np.array_equal(res[False][0], res[True][0])
    G = res[False][0]
    Go = _oracle_total_grad(ora, dims, U, beta, kappa, rho, n, phi)
    assert H.rel(G, Go) < 1e-10
    F = ora.grad_to_force(dims, U, G)
    lat = keep
    ap = lgt.action_params(beta=beta, kappa=kappa, n_stout=n, rho=rho)
    pf = lat.pack_spinor(phi, lgt.FULL, lgt.FP64)

    def S_of(W):
        lat.set_links(W)
        Sg, Sf, _ = lat.action(ap, pf, sp)
        return Sg + Sf

    # Central differences of the global action: the truncation error eps^2 S'''/6 is
    # ~1e-9 at eps = 1e-5, but |S| ~ 1.6e6 is rounded at ~u|S| per evaluation, so the
    # difference quotient carries ~sqrt(N)u|S|/eps.  The bound below is 20 u |S| / eps
    # (+1e-7 relative); eps = 2e-4 is checked as well, where rounding is 20x smaller.
    S0 = S_of(U)
    rng = np.random.default_rng(5)
    for eps in (1e-5, 2e-4):
        bound = 20 * 2.2e-16 * abs(S0) / eps
        for s, mu, a in zip(rng.integers(0, 65536, 8), rng.integers(0, 4, 8), rng.integers(0, 8, 8)):
            fd = (S_of(H.lie_perturb(U, s, mu, a, eps)) - S_of(H.lie_perturb(U, s, mu, a, -eps))) / (2 * eps)
            assert abs(fd - F[s, mu, a]) < bound + 1e-7 * abs(F[s, mu, a]), (eps, s, mu, a, fd, F[s, mu, a])
    print(f"\n16^4 stout stack: stored {res[False][2] / 1e6:.0f} MB {res[False][3]:.3f} s; "
          f"recomputed {res[True][2] / 1e6:.0f} MB {res[True][3]:.3f} s")


@pytest.mark.parametrize("n", [5, 7])
def test_deep_chain_checkpoint_modes_bitwise(lgt, ora, n):
    """Deep chains: every storage of the levels (all stored, recomputed from the thin
    links, checkpoints every 2 / 3 / n levels) gives the same smeared links and the
    same adjoint, bit for bit; the adjoint agrees with the oracle's."""
    U = synth.random_links(DIMS, 0.5, 45)
    G = synth.random_links(DIMS, 1.0, 46) + 0.5 * synth.random_links(DIMS, 1.0, 47)
    lat = lgt.Lattice(DIMS)
    lat.set_links(U)
    top = {m: lat.stout_smear(0.1, n, recompute=m) for m in (0, 1, 2, 3, n)}
    grad = {m: lat.stout_backward(0.1, n, G, recompute=m) for m in (0, 1, 2, 3, n)}
    for m in (1, 2, 3, n):
        assert torch.equal(top[m], top[0]), m
        assert torch.equal(grad[m], grad[0]), m
    levels = [U]
    for _ in range(n):
        levels.append(ora.stout_forward(DIMS, levels[-1], 0.1))
    Gr = G
    for k in range(n, 0, -1):
        Gr = ora.stout_backward(DIMS, levels[k - 1], 0.1, Gr)
    assert H.rel(_np(top[0]), levels[-1]) < 1e-13
    assert H.rel(_np(grad[0]), Gr) < 1e-12


def test_deep_chain_memory_and_force(lgt):
    """Level fields held for a 12-level chain: all stored 12, checkpoints every 3 levels
    3 + top + 2 segment fields, recomputed from the thin links 2 (measured against a
    1-level chain, which holds one); the force through the chain is the same in every
    mode, bit for bit."""
    n = 12
    U = synth.random_links(DIMS, 0.5, 48)
    phi = synth.gaussian_spinor(DIMS, 49)
    sp = lgt.solver("fp64", tol=1e-12)

    def run(n_levels, m):
        lat = lgt.Lattice(DIMS)
        lat.set_links(U)
        ap = lgt.action_params(beta=6.0, kappa=0.12, n_stout=n_levels, rho=0.05, stout_recompute=m)
        F, _ = lat.force(ap, lat.pack_spinor(phi, lgt.FULL, lgt.FP64), sp)
        return F, lat.info()[1]

    _, ref = run(1, 0)
    link_field = 4 * int(np.prod(DIMS)) * 9 * 16
    forces, fields = {}, {}
    for m in (0, 3, 1):
        forces[m], b = run(n, m)
        fields[m] = (b - ref) / link_field + 1
    assert fields == {0: 12, 3: 6, 1: 2}
    assert torch.equal(forces[3], forces[0]) and torch.equal(forces[1], forces[0])
