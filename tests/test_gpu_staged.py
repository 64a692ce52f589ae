"""Operand staging of the FP32 hops (lgt_set_hop_staging): each block of 128 output
sites copies its links and/or its input spinors with the neighbour halos into shared
memory by bulk copies before the arithmetic.  The arithmetic per site is unchanged, so
every staged launch must give bitwise the results of the unstaged one (hence the same
CG iterates and forces), and the FP32 hop must agree with the FP64 oracle within the
FP32 bar (2e-6 relative).

Shapes: every extent pattern the staging accepts (half-row of 1, 2, 8, 16 and 128
sites; 1 to 128 rows per block; extent-2 directions with coinciding z -+ 1 / t -+ 1
planes; the antiperiodic time wrap), plus one lattice it does not accept.
"""
import numpy as np
import pytest
import torch

from paper_2602_20516_b300 import synth
from tests import helpers as H

pytestmark = pytest.mark.gpu

STAGED = [(32, 8, 4, 4), (16, 16, 4, 4), (4, 64, 2, 4), (2, 128, 2, 2), (256, 2, 2, 2)]
MODES = [1, 2, 3]


@pytest.fixture(scope="module")
def lgt():
    from paper_2602_20516_b300 import lgt as L
    assert torch.cuda.is_available()
    L.lib()
    return L


def _np(t):
    return t.detach().cpu().numpy()


def test_staging_applies_and_rejects_bad_mode(lgt):
    assert lgt.Lattice((32, 8, 4, 4)).hop_staging_status()[0]
    assert lgt.Lattice((16, 16, 16, 32)).hop_staging_status()[0]
    assert not lgt.Lattice((8, 6, 4, 10)).hop_staging_status()[0]
    assert not lgt.Lattice((24, 24, 24, 48)).hop_staging_status()[0]
    lat = lgt.Lattice((32, 8, 4, 4))
    for bad in (-1, 4):
        with pytest.raises(lgt.LGTError):
            lat.set_hop_staging(bad)


@pytest.mark.parametrize("dims", STAGED + [(8, 6, 4, 10)])
@pytest.mark.parametrize("dagger", [False, True])
def test_staged_hop_bitwise_and_vs_oracle(lgt, ora, dims, dagger):
    U = synth.random_links(dims, 0.5, 31)
    psi = synth.gaussian_spinor(dims, 32)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    for p in (lgt.EVEN, lgt.ODD):
        src = lat.pack_spinor(psi, 1 - p, lgt.FP32)
        lat.set_hop_staging(0)
        h0 = lat.dslash(src, lgt.OP_HOP, p, dagger, 0.0, lgt.FP32)
        want = ora.hop(dims, U, psi, out_mask=1 << p, dagger=dagger)
        m = synth.parity(dims) == p
        assert H.rel(_np(lat.unpack_spinor(h0, p, lgt.FP32))[m], want[m]) < 2e-6
        for mode in MODES:
            lat.set_hop_staging(mode)
            hm = lat.dslash(src, lgt.OP_HOP, p, dagger, 0.0, lgt.FP32)
            assert torch.equal(hm, h0), (dims, p, dagger, mode)
    assert lat.hop_staging_status()[1] == 0


@pytest.mark.parametrize("dims", [(32, 8, 4, 4), (4, 64, 2, 4)])
def test_staged_normal_operator_bitwise(lgt, ora, dims):
    """Dhat^+ Dhat (xpay epilogues) on the even sites."""
    U = synth.random_links(dims, 0.5, 33)
    psi = synth.gaussian_spinor(dims, 34, parity_mask=1)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    src = lat.pack_spinor(psi, lgt.EVEN, lgt.FP32)
    out = []
    for mode in (0, 1, 2, 3):
        lat.set_hop_staging(mode)
        out.append(lat.dslash(src, lgt.OP_DHAT_NORMAL, lgt.EVEN, False, 0.15, lgt.FP32))
    for o in out[1:]:
        assert torch.equal(o, out[0])
    want = ora.dhat(dims, U, 0.15, ora.dhat(dims, U, 0.15, psi), dagger=True)
    ev = synth.parity(dims) == 0
    assert H.rel(_np(lat.unpack_spinor(out[3], lgt.EVEN, lgt.FP32))[ev], want[ev]) < 2e-6


@pytest.mark.parametrize("dims", [(16, 16, 4, 8), (32, 8, 4, 4)])
def test_staged_cg_same_iterates(lgt, dims):
    """The mixed even-odd CG (FP32 hops with the xpay + norm and residual-update
    epilogues, deferred reductions, alternating sweep) takes the same iterates."""
    lat = lgt.Lattice(dims)
    lat.set_links(synth.random_links(dims, 0.5, 35))
    b = lat.pack_spinor(synth.gaussian_spinor(dims, 36, parity_mask=1), lgt.EVEN, lgt.FP64)
    sp = lgt.solver("mixed", tol=1e-10, delta=3e-3)
    res = []
    for mode in (0, 1, 2, 3):
        lat.set_hop_staging(mode)
        res.append(lat.cg_solve(b, 0.156, True, sp))
    x0, s0 = res[0]
    for x, s in res[1:]:
        assert s["iters"] == s0["iters"] and s["reliable_updates"] == s0["reliable_updates"]
        assert torch.equal(x, x0)
    assert lat.hop_staging_status()[1] == 0


@pytest.mark.parametrize("csw", [0.0, 1.0])
def test_staged_force_bitwise(lgt, ora, csw):
    """Forces of the mixed path (Wilson and even-odd clover, whose hops carry the fused
    clover blocks) are bitwise those without staging, and the staged force agrees with
    the oracle's within the mixed-path bar."""
    dims = (16, 16, 4, 4)
    U = synth.random_links(dims, 0.5, 37)
    phi = synth.gaussian_spinor(dims, 38, parity_mask=1)
    lat = lgt.Lattice(dims)
    lat.set_links(U)
    pf = lat.pack_spinor(phi, lgt.EVEN, lgt.FP64)
    kappa = 0.13
    ap = lgt.action_params(beta=5.8, kappa=kappa, even_odd=True, force_arith="df64", csw=csw)
    sp = lgt.solver("mixed", tol=1e-10, delta=3e-3)
    F = []
    for mode in (0, 3):
        lat.set_hop_staging(mode)
        f, st = lat.force(ap, pf, sp)
        F.append(f)
    assert torch.equal(F[0], F[1])
    if csw == 0.0:
        Fo = ora.gauge_force(dims, U, 5.8) + ora.pf_force(dims, U, kappa, phi, eo=True, tol=1e-13)[0]
    else:
        Fo = ora.gauge_force(dims, U, 5.8) + ora.pf_force_sw_eo(dims, U, kappa, csw, phi, tol=1e-13)[0]
    assert H.rel(_np(lat.unpack_momenta(F[1])), Fo) < 1e-6


def test_staged_hop_full_size(lgt):
    """32^3 x 64 in the launch configuration the benchmark times: both parities and
    both signs, staged (every mode) against unstaged, bitwise."""
    dims = (32, 32, 32, 64)
    lat = lgt.Lattice(dims)
    lat.random_links(4, 0.5)
    for p in (lgt.EVEN, lgt.ODD):
        src = lat.gaussian_spinor(4, 0, lgt.FIELD_SOURCE, 1 - p)
        src32 = lat.pack_spinor(lat.unpack_spinor(src, 1 - p, lgt.FP64), 1 - p, lgt.FP32)
        for dagger in (False, True):
            lat.set_hop_staging(0)
            h0 = lat.dslash(src32, lgt.OP_HOP, p, dagger, 0.0, lgt.FP32)
            for mode in MODES:
                lat.set_hop_staging(mode)
                assert torch.equal(lat.dslash(src32, lgt.OP_HOP, p, dagger, 0.0, lgt.FP32), h0), (p, dagger, mode)
    assert lat.hop_staging_status()[1] == 0
