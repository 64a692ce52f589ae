"""The double-float (FP32-pair) Wilson hop against the FP64 oracle, and the mixed
solver whose true residuals it forms.

The double-float format carries about 48 significant bits, so the hop must agree
with the oracle's FP64 hop within 1e-13 relative; the residual b - A x that the mixed
solver computes with it must agree with an FP64 recomputation within 1e-13 |b|, far
below every solver tolerance it is used with.
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


def _np(t):
    return t.detach().cpu().numpy()


def _mask(dims, p):
    return synth.parity(dims) == p


def test_df64_layout_round_trip(lgt):
    dims = (6, 4, 2, 8)
    lat = lgt.Lattice(dims)
    psi = synth.gaussian_spinor(dims, 2)
    for par in (lgt.FULL, lgt.EVEN, lgt.ODD):
        f = lat.pack_spinor(psi, par, lgt.DF64)
        back = _np(lat.unpack_spinor(f, par, lgt.DF64))
        m = np.ones(len(psi), bool) if par == lgt.FULL else _mask(dims, par)
        # a pair of FP32 numbers holds 48 significant bits of each component
        assert H.rel(back[m], psi[m]) < 1e-14
        assert not back[~m].any()


@pytest.mark.parametrize("dims", SHAPES)
@pytest.mark.parametrize("dagger", [False, True])
def test_df64_hop_vs_oracle(lgt, ora, dims, dagger):
    U = synth.random_links(dims, 0.5, 5)
    psi = synth.gaussian_spinor(dims, 6)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    for p in (lgt.EVEN, lgt.ODD):
        src = lat.pack_spinor(psi, 1 - p, lgt.DF64)
        h = lat.dslash(src, lgt.OP_HOP, p, dagger, 0.0, lgt.DF64)
        got = _np(lat.unpack_spinor(h, p, lgt.DF64))
        want = ora.hop(dims, U, psi, out_mask=1 << p, dagger=dagger)
        m = _mask(dims, p)
        assert H.rel(got[m], want[m]) < 1e-13, (p, dagger)
        assert not got[~m].any()


def test_df64_hop_full_size_sampled(lgt, ora):
    """32^3 x 64, links from the device generator (seed 4, alpha 0.5): the double-float
    hop against the oracle's hop on oracle-generated links (identical up to the
    exponential's rounding), on every even site and on a sample."""
    dims = (32, 32, 32, 64)
    lat = lgt.Lattice(dims)
    lat.random_links(4, 0.5)
    Uo = ora.random_links(dims, 4, 0.5)
    psi = ora.gaussian_spinor(dims, 4, 0, ora.FIELD_SOURCE, 2)   # odd sites
    want = ora.hop(dims, Uo, psi, out_mask=1)
    ev = _mask(dims, 0)
    f = lat.pack_spinor(psi, lgt.ODD, lgt.DF64)
    h = lat.dslash(f, lgt.OP_HOP, lgt.EVEN, False, 0.0, lgt.DF64)
    got = _np(lat.unpack_spinor(h, lgt.EVEN, lgt.DF64))
    sample = np.random.default_rng(0).choice(np.where(ev)[0], 20000, replace=False)
    assert H.rel(got[sample], want[sample]) < 1e-13
    assert H.rel(got[ev], want[ev]) < 1e-13


def test_df64_hop_rejects_other_operators(lgt):
    dims = (4, 4, 4, 4)
    lat = lgt.Lattice(dims)
    f = lat.spinor_field(lgt.FULL, lgt.DF64)
    with pytest.raises(lgt.LGTError):
        lat.dslash(f, lgt.OP_D, lgt.FULL, False, 0.15, lgt.DF64)


@pytest.mark.parametrize("dims", [(8, 6, 4, 10), (6, 4, 2, 8)])
def test_mixed_solver_true_residual_in_double_float(lgt, ora, dims):
    """A mixed solve to tol 1e-12 stops on its double-float true residual: recomputed
    with the FP64 operator, |b - A x| / |b| is still below the tolerance (to within
    the format's ~1e-14), and x agrees with the oracle's solve."""
    U = synth.random_links(dims, 0.5, 11)
    b = synth.gaussian_spinor(dims, 12, parity_mask=1)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    kappa = 0.155
    bf = lat.pack_spinor(b, lgt.EVEN, lgt.FP64)
    tol = 1e-12
    x, st = lat.cg_solve(bf, kappa, True, lgt.solver("mixed", tol=tol, delta=1e-3))
    Ax = lat.dslash(x, lgt.OP_DHAT_NORMAL, lgt.EVEN, False, kappa, lgt.FP64)
    ev = _mask(dims, 0)
    r = _np(lat.unpack_spinor(bf, lgt.EVEN, lgt.FP64))[ev] - _np(lat.unpack_spinor(Ax, lgt.EVEN, lgt.FP64))[ev]
    res64 = np.linalg.norm(r) / np.linalg.norm(b[ev])
    assert res64 <= tol * 1.01 + 1e-14, (res64, st)
    assert abs(res64 - st["true_rel_residual"]) < 1e-13
    xo, _, _ = ora.cg(dims, U, kappa, b, eo=True, tol=1e-14)
    assert H.rel(_np(lat.unpack_spinor(x, lgt.EVEN, lgt.FP64))[ev], xo[ev]) < 1e-9


@pytest.mark.parametrize("eps", [0.05, 0.7])
def test_df64_link_update_matches_fp64(lgt, eps):
    """On the mixed path with double-float force arithmetic the link update after a
    force evaluation runs in double-float from the copy of the links the evaluation
    made: it agrees with the FP64 update to 1e-13 per link and stays unitary.  eps 0.7
    with N(0,1) momenta takes the exponential's scaling-and-squaring branch."""
    dims = (8, 6, 4, 10)
    U = synth.random_links(dims, 0.5, 51)
    mom = synth.gaussian_momenta(dims, 52)
    phi = synth.gaussian_spinor(dims, 53, parity_mask=1)
    ap = lgt.action_params(beta=5.8, kappa=0.155, even_odd=True, force_arith="df64")
    sp = lgt.solver("mixed", tol=1e-10, delta=3e-3)
    a = lgt.Lattice(dims)
    a.set_links(U)
    m = a.pack_momenta(mom)
    a.md_update(m, 0.05, lgt.UPDATE_P, ap, a.pack_spinor(phi, lgt.EVEN, lgt.FP64), sp)
    b = lgt.Lattice(dims)
    b.set_links(U)
    mb = m.clone()
    a.md_update(m, eps, lgt.UPDATE_U, ap, None, sp)     # double-float
    b.md_update(mb, eps, lgt.UPDATE_U)                  # FP64
    Ua, Ub = _np(a.get_links()), _np(b.get_links())
    per_link = np.linalg.norm((Ua - Ub).reshape(-1, 9), axis=1) / np.linalg.norm(Ub.reshape(-1, 9), axis=1)
    assert per_link.max() < 1e-13, per_link.max()
    uu = Ua @ np.conj(np.swapaxes(Ua, -1, -2))
    assert np.abs(uu - np.eye(3)).max() < 1e-13
    # the FP32 copy follows the FP64 links: an FP32 operator on it agrees with one on
    # the FP32 copy derived from the FP64 links (the high word of a pair is the FP64
    # value rounded to FP32, up to exact ties)
    src = a.pack_spinor(phi, lgt.EVEN, lgt.FP32)
    ha = a.dslash(src, lgt.OP_HOP, lgt.ODD, False, 0.0, lgt.FP32)
    b.set_links(Ua)
    hb = b.dslash(b.pack_spinor(phi, lgt.EVEN, lgt.FP32), lgt.OP_HOP, lgt.ODD, False, 0.0, lgt.FP32)
    assert (torch.linalg.norm(ha - hb) / torch.linalg.norm(hb)).item() < 1e-6
