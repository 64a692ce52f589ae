"""GPU (liblgt, sm_103a) vs the FP64 oracle, element by element, on seeded inputs.

Tolerances: the FP64 path must agree within 1e-10 relative, the mixed / FP32 path
within 1e-6 relative (relative = |a-b|_2 / |b|_2 over the whole field).  Lattice
shapes cover several thread blocks, ragged tails (V/2 not a multiple of 128),
extent-2 directions and the antiperiodic time wrap.
"""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 4, 4), (6, 4, 2, 8), (8, 6, 4, 10)]


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _lat(lgt, dims, U):
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    return lat


def _np(t):
    return t.detach().cpu().numpy()


def _parity_mask(dims, p):
    return synth.parity(dims) == p


# ------------------------------------------------------------------ layouts and seeded fields
@pytest.mark.parametrize("dims", SHAPES)
def test_layout_roundtrips_bit_exact(lgt, dims):
    U = synth.random_links(dims, 0.5, 1)
    lat = _lat(lgt, dims, U)
    assert np.array_equal(_np(lat.get_links()), U)
    psi = synth.gaussian_spinor(dims, 2)
    f = lat.pack_spinor(psi, lgt.FULL, lgt.FP64)
    assert np.array_equal(_np(lat.unpack_spinor(f, lgt.FULL, lgt.FP64)), psi)
    fe = lat.pack_spinor(psi, lgt.EVEN, lgt.FP64)
    back = _np(lat.unpack_spinor(fe, lgt.EVEN, lgt.FP64))
    ev = _parity_mask(dims, 0)
    assert np.array_equal(back[ev], psi[ev]) and not back[~ev].any()
    f32 = lat.pack_spinor(psi, lgt.FULL, lgt.FP32)
    b32 = _np(lat.unpack_spinor(f32, lgt.FULL, lgt.FP32))
    assert np.array_equal(b32, psi.astype(np.complex64).astype(np.complex128))
    mom = synth.gaussian_momenta(dims, 3)
    assert np.array_equal(_np(lat.unpack_momenta(lat.pack_momenta(mom))), mom)
    G = synth.random_links(dims, 1.0, 4)
    assert np.array_equal(_np(lat.unpack_grad(lat.pack_grad(G))), G)


def test_seeded_fields_match_oracle(lgt, ora):
    dims = (6, 4, 4, 8)
    lat = lgt.Lattice(dims)
    lat.random_links(77, 0.5)
    Uo = ora.random_links(dims, 77, 0.5)
    assert H.rel(_np(lat.get_links()), Uo) < 1e-13
    m = lat.unpack_momenta(lat.gaussian_momenta(5, 3))
    assert H.rel(_np(m), ora.gaussian_momenta(dims, 5, 3)) < 1e-14
    xi = lat.unpack_spinor(lat.gaussian_spinor(5, 3, lgt.FIELD_XI, lgt.FULL), lgt.FULL, lgt.FP64)
    assert H.rel(_np(xi), ora.gaussian_spinor(dims, 5, 3, ora.FIELD_XI, 3)) < 1e-14
    xe = lat.unpack_spinor(lat.gaussian_spinor(5, 3, lgt.FIELD_XI, lgt.EVEN), lgt.EVEN, lgt.FP64)
    assert H.rel(_np(xe), ora.gaussian_spinor(dims, 5, 3, ora.FIELD_XI, 1)) < 1e-14


# ------------------------------------------------------------------ operators
@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
def test_hop_and_dirac_fp64(lgt, ora, dims, dagger):
    U = synth.random_links(dims, 0.5, 5)
    psi = synth.gaussian_spinor(dims, 6)
    lat = _lat(lgt, dims, U)
    kappa = 0.155
    f = lat.pack_spinor(psi, lgt.FULL, lgt.FP64)
    out = lat.dslash(f, lgt.OP_D, lgt.FULL, dagger, kappa, lgt.FP64)
    ref = ora.dirac(dims, U, kappa, psi, dagger)
    assert H.rel(_np(lat.unpack_spinor(out, lgt.FULL, lgt.FP64)), ref) < 1e-14
    for p in (lgt.EVEN, lgt.ODD):
        src = lat.pack_spinor(psi, 1 - p, lgt.FP64)
        h = lat.dslash(src, lgt.OP_HOP, p, dagger, 0.0, lgt.FP64)
        got = _np(lat.unpack_spinor(h, p, lgt.FP64))
        want = ora.hop(dims, U, psi, out_mask=1 << p, dagger=dagger)
        m = _parity_mask(dims, p)
        assert H.rel(got[m], want[m]) < 1e-14


@pytest.mark.parametrize("dims", SHAPES)
def test_dhat_and_normal_fp64_fp32(lgt, ora, dims):
    U = synth.random_links(dims, 0.5, 7)
    psi = synth.gaussian_spinor(dims, 8, parity_mask=1)
    lat = _lat(lgt, dims, U)
    kappa = 0.155
    ev = _parity_mask(dims, 0)
    for dag in (False, True):
        want = ora.dhat(dims, U, kappa, psi, dag)[ev]
        for prec, tol in ((lgt.FP64, 1e-14), (lgt.FP32, 2e-6)):
            f = lat.pack_spinor(psi, lgt.EVEN, prec)
            out = lat.dslash(f, lgt.OP_DHAT, lgt.EVEN, dag, kappa, prec)
            got = _np(lat.unpack_spinor(out, lgt.EVEN, prec))[ev]
            assert H.rel(got, want) < tol, (prec, dag)
    want = ora.dhat(dims, U, kappa, ora.dhat(dims, U, kappa, psi), True)[ev]
    for prec, tol in ((lgt.FP64, 1e-14), (lgt.FP32, 3e-6)):
        f = lat.pack_spinor(psi, lgt.EVEN, prec)
        out = lat.dslash(f, lgt.OP_DHAT_NORMAL, lgt.EVEN, False, kappa, prec)
        assert H.rel(_np(lat.unpack_spinor(out, lgt.EVEN, prec))[ev], want) < tol


def test_fp32_full_dirac(lgt, ora):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 9)
    psi = synth.gaussian_spinor(dims, 10)
    lat = _lat(lgt, dims, U)
    for dag in (False, True):
        f = lat.pack_spinor(psi, lgt.FULL, lgt.FP32)
        out = lat.dslash(f, lgt.OP_D, lgt.FULL, dag, 0.157, lgt.FP32)
        want = ora.dirac(dims, U, 0.157, psi, dag)
        assert H.rel(_np(lat.unpack_spinor(out, lgt.FULL, lgt.FP32)), want) < 2e-6


# ------------------------------------------------------------------ solver
@pytest.mark.parametrize("eo", [True, False])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cg_solution(lgt, ora, eo, precision):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 11)
    b = synth.gaussian_spinor(dims, 12, parity_mask=1 if eo else 3)
    lat = _lat(lgt, dims, U)
    kappa = 0.155
    par = lgt.EVEN if eo else lgt.FULL
    bf = lat.pack_spinor(b, par, lgt.FP64)
    tol = 1e-12 if precision == "fp64" else 1e-10
    x, st = lat.cg_solve(bf, kappa, eo, lgt.solver(precision, tol=tol))
    assert st["true_rel_residual"] <= tol
    xo, it, res = ora.cg(dims, U, kappa, b, eo=eo, tol=1e-13)
    got = _np(lat.unpack_spinor(x, par, lgt.FP64))
    bar = 1e-9 if precision == "fp64" else 1e-6
    assert H.rel(got, xo) < bar
    if precision == "mixed":
        assert st["reliable_updates"] >= 2


# ------------------------------------------------------------------ actions and forces
def test_plaquette_and_gauge_action(lgt, ora):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 13)
    lat = _lat(lgt, dims, U)
    assert abs(lat.plaquette() - ora.plaquette(dims, U)) < 1e-14
    Sg, _, _ = lat.action(lgt.action_params(beta=5.8, fermions=False))
    So = ora.gauge_action(dims, U, 5.8)
    assert abs(Sg - So) / So < 1e-13


@pytest.mark.parametrize("eo", [False, True])
def test_pf_action(lgt, ora, eo):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 14)
    phi = synth.gaussian_spinor(dims, 15, parity_mask=1 if eo else 3)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.8, kappa=0.155, even_odd=eo)
    pf = lat.pack_spinor(phi, lgt.EVEN if eo else lgt.FULL, lgt.FP64)
    So, _ = ora.pf_action(dims, U, 0.155, phi, eo=eo, tol=1e-13)
    _, Sf, _ = lat.action(ap, pf, lgt.solver("fp64", tol=1e-12))
    assert abs(Sf - So) / So < 1e-12
    _, Sm, _ = lat.action(ap, pf, lgt.solver("mixed", tol=1e-10))
    assert abs(Sm - So) / So < 1e-9


def test_gauge_force(lgt, ora):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 16)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.8, fermions=False)
    F, _ = lat.force(ap)
    assert H.rel(_np(lat.unpack_momenta(F)), ora.gauge_force(dims, U, 5.8)) < 1e-13
    G, _ = lat.force(ap, form=lgt.GRAD_G)
    assert H.rel(_np(lat.unpack_grad(G)), ora.gauge_action_grad(dims, U, 5.8)) < 1e-14


@pytest.mark.parametrize("eo", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_fermion_force(lgt, ora, eo, precision):
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 17)
    phi = synth.gaussian_spinor(dims, 18, parity_mask=1 if eo else 3)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=0.0, kappa=0.155, even_odd=eo)
    pf = lat.pack_spinor(phi, lgt.EVEN if eo else lgt.FULL, lgt.FP64)
    tol = 1e-13 if precision == "fp64" else 1e-10
    F, st = lat.force(ap, pf, lgt.solver(precision, tol=tol))
    Fo, _ = ora.pf_force(dims, U, 0.155, phi, eo=eo, tol=1e-13)
    bar = 1e-10 if precision == "fp64" else 1e-6
    assert H.rel(_np(lat.unpack_momenta(F)), Fo) < bar
    if precision == "fp64":
        G, _ = lat.force(ap, pf, lgt.solver("fp64", tol=1e-13), form=lgt.GRAD_G)
        Go, _ = ora.pf_action_grad(dims, U, 0.155, phi, eo=eo, tol=1e-13)
        assert H.rel(_np(lat.unpack_grad(G)), Go) < 1e-10


def test_total_force_link_level_error_cdf(lgt, ora):
    """Per-link relative Frobenius error of Eq. 10 between GPU and oracle force."""
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 19)
    phi = synth.gaussian_spinor(dims, 20, parity_mask=1)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.8, kappa=0.155, even_odd=True)
    pf = lat.pack_spinor(phi, lgt.EVEN, lgt.FP64)
    F, _ = lat.force(ap, pf, lgt.solver("fp64", tol=1e-13))
    Fo = ora.gauge_force(dims, U, 5.8) + ora.pf_force(dims, U, 0.155, phi, eo=True, tol=1e-13)[0]
    Fg = _np(lat.unpack_momenta(F))
    # Frobenius norm of sum_a F_a T^a is |F|/sqrt(2): the ratio is the same
    eps = np.linalg.norm(Fg - Fo, axis=-1) / np.linalg.norm(Fo, axis=-1)
    assert np.quantile(eps, 0.999) < 1e-10 and eps.max() < 1e-9


@pytest.mark.parametrize("eo", [False, True])
@pytest.mark.parametrize("arith", ["fp64", "fp32", "df64"])
def test_mixed_total_force(lgt, ora, eo, arith):
    """Mixed path: FP32 CG with FP64 reliable updates; force arithmetic FP64 (default),
    FP32 accumulated in FP64, or double-float (FP32 pairs) accumulated in FP64.  Within
    1e-6 of the FP64 oracle (whole field and per link); FP64 and double-float forces
    within 1e-7, where the solver tolerance (1e-10) sets the error."""
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 27)
    phi = synth.gaussian_spinor(dims, 28, parity_mask=1 if eo else 3)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.8, kappa=0.156, even_odd=eo, force_arith=arith)
    pf = lat.pack_spinor(phi, lgt.EVEN if eo else lgt.FULL, lgt.FP64)
    F, st = lat.force(ap, pf, lgt.solver("mixed", tol=1e-10, delta=1e-4))
    Fo = ora.gauge_force(dims, U, 5.8) + ora.pf_force(dims, U, 0.156, phi, eo=eo, tol=1e-13)[0]
    Fg = _np(lat.unpack_momenta(F))
    assert H.rel(Fg, Fo) < (1e-6 if arith == "fp32" else 1e-7)
    eps = np.linalg.norm(Fg - Fo, axis=-1) / np.linalg.norm(Fo, axis=-1)
    assert np.quantile(eps, 0.999) < 1e-5
    # the kick applies exactly this force: mom - eps F
    mom = synth.gaussian_momenta(dims, 29)
    m = lat.pack_momenta(mom)
    lat.md_update(m, 0.05, lgt.UPDATE_P, ap, pf, lgt.solver("mixed", tol=1e-10, delta=1e-4))
    assert H.rel(_np(lat.unpack_momenta(m)), mom - 0.05 * Fo) < 1e-6


def test_double_float_gauge_force(lgt, ora):
    """Double-float staple force (pure gauge, mixed solver selects the arithmetic):
    about 48-bit products, within 1e-13 of the FP64 oracle, per link within 1e-12."""
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 31)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.8, fermions=False, force_arith="df64")
    F, _ = lat.force(ap, None, lgt.solver("mixed", tol=1e-10))
    Fo = ora.gauge_force(dims, U, 5.8)
    Fg = _np(lat.unpack_momenta(F))
    assert H.rel(Fg, Fo) < 1e-13
    eps = np.linalg.norm(Fg - Fo, axis=-1) / np.linalg.norm(Fo, axis=-1)
    assert eps.max() < 1e-12


@pytest.mark.parametrize("eo", [False, True])
def test_double_float_fermion_force(lgt, ora, eo):
    """Double-float fermion force on the same mixed solve as the FP64 kernel: the two
    differ only by the force arithmetic (within 1e-12); against the oracle the solver
    tolerance (1e-12) sets the error."""
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 32)
    phi = synth.gaussian_spinor(dims, 33, parity_mask=1 if eo else 3)
    lat = _lat(lgt, dims, U)
    pf = lat.pack_spinor(phi, lgt.EVEN if eo else lgt.FULL, lgt.FP64)
    sp = lgt.solver("mixed", tol=1e-12, delta=1e-4)
    F64, s64 = lat.force(lgt.action_params(kappa=0.156, even_odd=eo, force_arith="fp64"), pf, sp)
    Fdf, sdf = lat.force(lgt.action_params(kappa=0.156, even_odd=eo, force_arith="df64"), pf, sp)
    assert s64["iters"] == sdf["iters"]
    assert H.rel(_np(lat.unpack_momenta(Fdf)), _np(lat.unpack_momenta(F64))) < 1e-12
    Fo = ora.pf_force(dims, U, 0.156, phi, eo=eo, tol=1e-13)[0]
    assert H.rel(_np(lat.unpack_momenta(Fdf)), Fo) < 1e-9


# ------------------------------------------------------------------ molecular dynamics
def test_link_update_and_kick(lgt, ora):
    dims = (6, 4, 4, 8)
    U = synth.random_links(dims, 0.5, 21)
    mom = synth.gaussian_momenta(dims, 22)
    lat = _lat(lgt, dims, U)
    m = lat.pack_momenta(mom)
    lat.md_update(m, 0.37, lgt.UPDATE_U)
    assert H.rel(_np(lat.get_links()), ora.update_links(dims, U, mom, 0.37)) < 1e-14
    # a kick with the gauge force: mom - eps F
    U1 = ora.update_links(dims, U, mom, 0.37)
    lat.md_update(m, 0.05, lgt.UPDATE_P, lgt.action_params(beta=5.7, fermions=False))
    want = mom - 0.05 * ora.gauge_force(dims, U1, 5.7)
    assert H.rel(_np(lat.unpack_momenta(m)), want) < 1e-14
    assert abs(lat.kinetic_energy(m) - ora.momentum_energy(dims, want)) / ora.momentum_energy(dims, want) < 1e-14


def test_small_exponent_branch(lgt, ora):
    """exp(i eps P) for tiny eps (Taylor branch) and around the branch switch."""
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.5, 23)
    mom = synth.gaussian_momenta(dims, 24)
    for eps in (0.0, 1e-9, 1e-4, 0.02, 0.03, 0.5, 2.0):
        lat = _lat(lgt, dims, U)
        m = lat.pack_momenta(mom)
        lat.md_update(m, eps, lgt.UPDATE_U)
        assert H.rel(_np(lat.get_links()), ora.update_links(dims, U, mom, eps)) < 1e-14, eps


def test_reunitarise(lgt, ora):
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.5, 25)
    W = U + 1e-7 * np.random.default_rng(1).standard_normal(U.shape)
    lat = _lat(lgt, dims, W)
    lat.reunitarise()
    assert H.rel(_np(lat.get_links()), ora.reunitarise(dims, W)) < 1e-14


@pytest.mark.parametrize("integrator,eo", [("leapfrog", False), ("omelyan", True)])
def test_hmc_trajectory_matches_oracle(lgt, ora, integrator, eo):
    """Config-1 style trajectory: 4^4, beta 5.7, kappa 0.15, alpha 0.3, tol 1e-12."""
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3, 26)
    lat = _lat(lgt, dims, U)
    ap = lgt.action_params(beta=5.7, kappa=0.15, even_odd=eo)
    sp = lgt.solver("fp64", tol=1e-13)
    hp = lgt.hmc_params(integrator, n_steps=10, tau=1.0, md_solver=sp, action_solver=sp)
    r = lat.hmc_trajectory(ap, hp, 1, 0)
    Uo, ro = ora.hmc_trajectory(dims, U, ora.hmc_params(5.7, 0.15, eo=eo, integrator=integrator,
                                                        n_steps=10, tau=1.0, tol_md=1e-13,
                                                        tol_action=1e-13), 1, 0)
    for k in ("K_old", "Sg_old", "Sf_old", "K_new", "Sg_new", "Sf_new"):
        assert abs(r[k] - ro[k]) / abs(ro[k]) < 1e-10, k
    assert abs(r["dH"] - ro["dH"]) < 1e-8 * max(1.0, abs(ro["dH"]))
    assert r["accepted"] == ro["accepted"] and r["force_evals"] == ro["force_evals"]
    assert H.rel(_np(lat.get_links()), Uo) < 1e-10


def test_hmc_mixed_vs_fp64_delta_h(lgt):
    """Same start, same seeds: the mixed path (FP32 CG, FP64 reliable updates) with
    FP64 or double-float force arithmetic reproduces the FP64 path's Delta H within
    1e-6 relative; FP32 force arithmetic moves it by O(1e-4) and is only asked to
    stay within 1e-2."""
    dims = (8, 8, 8, 8)
    lat = lgt.Lattice(dims)
    lat.random_links(4, 0.5)
    U0 = lat.get_links()
    dH = {}
    for name, prec, arith in (("fp64", "fp64", "fp64"), ("mixed", "mixed", "fp64"),
                              ("mixed_df64", "mixed", "df64"), ("mixed_f32", "mixed", "fp32")):
        lat.set_links(U0)
        sp = lgt.solver(prec, tol=1e-10, delta=1e-4)
        ap = lgt.action_params(beta=5.8, kappa=0.156, even_odd=True, force_arith=arith)
        dH[name] = lat.hmc_trajectory(ap, lgt.hmc_params("omelyan", 20, 1.0, sp, sp), 4, 0)["dH"]
    assert abs(dH["mixed"] - dH["fp64"]) <= 1e-6 * abs(dH["fp64"]) + 1e-9
    assert abs(dH["mixed_df64"] - dH["fp64"]) <= 1e-6 * abs(dH["fp64"]) + 1e-9
    assert abs(dH["mixed_f32"] - dH["fp64"]) <= 1e-2 * abs(dH["fp64"]) + 1e-6


def test_md_reversibility_gpu(lgt):
    dims = (4, 4, 4, 8)
    lat = lgt.Lattice(dims)
    lat.random_links(3, 0.3)
    U0 = _np(lat.get_links())
    ap = lgt.action_params(beta=5.7, kappa=0.15, even_odd=True)
    phi = lat.gaussian_spinor(9, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    sp = lgt.solver("fp64", tol=1e-14)
    mom = lat.gaussian_momenta(4, 0)
    m0 = mom.clone()
    eps, n = 0.1, 5

    def run():
        lat.md_update(mom, 0.5 * eps, lgt.UPDATE_P, ap, phi, sp)
        for i in range(n):
            lat.md_update(mom, eps, lgt.UPDATE_U)
            lat.md_update(mom, eps if i + 1 < n else 0.5 * eps, lgt.UPDATE_P, ap, phi, sp)

    run()
    mom.neg_()
    run()
    assert H.rel(_np(lat.get_links()), U0) < 1e-11
    assert (torch.linalg.norm(mom + m0) / torch.linalg.norm(m0)).item() < 1e-10


def test_link_grid_reductions_large_volume(lgt, ora):
    """Reductions over one thread per link (kinetic energy) use 8 Vh / 128 partial
    sums; at 16^3 x 48 that exceeds a site-sized buffer.  The energy must match the
    oracle and a following solve must still converge (reduction state intact)."""
    dims = (16, 16, 16, 48)
    lat = lgt.Lattice(dims)
    lat.random_links(5, 0.5)
    mom = lat.gaussian_momenta(6, 2)
    K = lat.kinetic_energy(mom)
    Ko = ora.momentum_energy(dims, ora.gaussian_momenta(dims, 6, 2))
    assert abs(K - Ko) / Ko < 1e-13
    assert abs(lat.plaquette() - ora.plaquette(dims, ora.random_links(dims, 5, 0.5))) < 1e-13
    b = lat.gaussian_spinor(7, 0, lgt.FIELD_SOURCE, lgt.EVEN)
    x, st = lat.cg_solve(b, 0.155, True, lgt.solver("mixed", tol=1e-10, max_iter=2000))
    assert st["true_rel_residual"] <= 1e-10 and st["iters"] < 2000


# ------------------------------------------------------------------ full size (bench workload)
def test_full_size_hop_sampled(lgt, ora):
    """32^3 x 64 lattice from the device generator (seed 4, alpha 0.5): the FP64 and
    FP32 hops agree with the oracle's hop on oracle-generated links."""
    dims = (32, 32, 32, 64)
    lat = lgt.Lattice(dims)
    lat.random_links(4, 0.5)
    Uo = ora.random_links(dims, 4, 0.5)
    psi = ora.gaussian_spinor(dims, 4, 0, ora.FIELD_SOURCE, 2)   # odd sites
    want = ora.hop(dims, Uo, psi, out_mask=1)
    ev = _parity_mask(dims, 0)
    rng = np.random.default_rng(0)
    sample = rng.choice(np.where(ev)[0], 20000, replace=False)
    for prec, tol in ((lgt.FP64, 1e-13), (lgt.FP32, 2e-6)):
        f = lat.pack_spinor(psi, lgt.ODD, prec)
        h = lat.dslash(f, lgt.OP_HOP, lgt.EVEN, False, 0.0, prec)
        got = _np(lat.unpack_spinor(h, lgt.EVEN, prec))
        assert H.rel(got[sample], want[sample]) < tol
        assert H.rel(got[ev], want[ev]) < tol


# ------------------------------------------------------------------ rectangle-improved gauge action
@pytest.mark.parametrize("c1", [-1.0 / 12, -0.331])
def test_improved_gauge_action_and_force(lgt, ora, c1):
    """Symanzik and Iwasaki actions: S_G, the mean rectangle, the Lie force (FP64 and
    FP32 arithmetic; double-float falls back to FP64 for c1 != 0) and the G-form
    gradient against the oracle."""
    dims = (8, 6, 4, 10)
    V = int(np.prod(dims))
    U = synth.random_links(dims, 0.5, 91)
    lat = _lat(lgt, dims, U)
    beta = 2.5
    ap = lgt.action_params(beta=beta, fermions=False, c1=c1)
    Sg, _, _ = lat.action(ap)
    assert abs(Sg - ora.gauge_action(dims, U, beta, c1)) < 1e-12 * abs(Sg)
    assert abs(lat.rectangle() - ora.rectangle_sum(dims, U) / (12 * V)) < 1e-13
    Fo = ora.gauge_force(dims, U, beta, c1)
    F, _ = lat.force(ap, None, lgt.solver("fp64"))
    assert H.rel(_np(lat.unpack_momenta(F)), Fo) < 1e-12
    G, _ = lat.force(ap, None, lgt.solver("fp64"), form=lgt.GRAD_G)
    assert H.rel(_np(lat.unpack_grad(G)), ora.gauge_action_grad(dims, U, beta, c1)) < 1e-12
    for arith, bar in (("fp32", 1e-6), ("df64", 1e-12)):
        a2 = lgt.action_params(beta=beta, fermions=False, c1=c1, force_arith=arith)
        F2, _ = lat.force(a2, None, lgt.solver("mixed"))
        assert H.rel(_np(lat.unpack_momenta(F2)), Fo) < bar, arith


def test_improved_hmc_trajectory_matches_oracle(lgt, ora):
    """Iwasaki gauge action + Nf=2 Wilson fermions, leapfrog: energies and Delta H of
    one trajectory against the oracle."""
    dims = (4, 4, 4, 4)
    U = synth.random_links(dims, 0.3, 92)
    lat = _lat(lgt, dims, U)
    c1 = -0.331
    ap = lgt.action_params(beta=2.3, kappa=0.14, c1=c1)
    sp = lgt.solver("fp64", tol=1e-13)
    r = lat.hmc_trajectory(ap, lgt.hmc_params("leapfrog", 10, 1.0, sp, sp), 3, 0)
    Uo, ro = ora.hmc_trajectory(dims, U, ora.hmc_params(2.3, 0.14, integrator="leapfrog", n_steps=10, tau=1.0,
                                                        tol_md=1e-13, tol_action=1e-13, c1=c1), 3, 0)
    for k in ("K_old", "Sg_old", "Sf_old", "K_new", "Sg_new", "Sf_new"):
        assert abs(r[k] - ro[k]) / abs(ro[k]) < 1e-10, k
    assert abs(r["dH"] - ro["dH"]) < 1e-8 * max(1.0, abs(ro["dH"]))
    assert r["accepted"] == ro["accepted"]
