"""torch.autograd.Function front end: the actions and the stout smearing as
differentiable functions of the canonical link tensor U (complex128, (V, 4, 3, 3),
on the GPU).

The paper obtains the force as the adjoint of the action program (Eq. 3, Fig. 1)
by LLVM-level AD; here each adjoint is a hand-written CUDA kernel of liblgt and
autograd only chains them.  torch's gradient of a real loss with respect to a
complex tensor is dL/dReU + i dL/dImU, which is exactly the G of Eq. S2.11, so
the backward passes return the library's G-form gradients unchanged.  The Lie
force of Eq. 9 follows from G as F_a = Re tr(G^+ i T^a U).

Every Function loads its input links into the given Lattice handle on entry, so
one handle can serve a whole graph.  The pseudofermion field phi is treated as a
constant (no gradient).
"""
import torch

from . import lgt


def _links(lat, U):
    lat.set_links(U.detach())


class GaugeAction(torch.autograd.Function):
    """S_G = beta sum_{x, mu<nu} (1 - Re tr U_munu / 3); backward G = -(beta/3) V^+."""

    @staticmethod
    def forward(ctx, U, lat, beta):
        _links(lat, U)
        Sg, _, _ = lat.action(lgt.action_params(beta=beta, fermions=False))
        ctx.save_for_backward(U)
        ctx.lat, ctx.beta = lat, beta
        return torch.tensor(Sg, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_S):
        (U,) = ctx.saved_tensors
        lat = ctx.lat
        _links(lat, U)
        G, _ = lat.force(lgt.action_params(beta=ctx.beta, fermions=False), form=lgt.GRAD_G)
        return grad_S * lat.unpack_grad(G), None, None


class PseudofermionAction(torch.autograd.Function):
    """S_f = phi^+ (M^+M)^{-1} phi (Eq. S3.1; M = D, or Dhat on even sites), with
    backward from delta S_f = -2 Re[eta^+ (delta D) chi] (Eq. S3.12)."""

    @staticmethod
    def forward(ctx, U, phi, lat, kappa, even_odd, solver):
        _links(lat, U)
        par = lgt.EVEN if even_odd else lgt.FULL
        pf = lat.pack_spinor(phi.detach(), par, lgt.FP64)
        ap = lgt.action_params(beta=0.0, kappa=kappa, even_odd=even_odd)
        _, Sf, st = lat.action(ap, pf, solver)
        ctx.save_for_backward(U)
        ctx.lat, ctx.pf, ctx.ap, ctx.solver = lat, pf, ap, solver
        ctx.stats = st
        return torch.tensor(Sf, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_S):
        (U,) = ctx.saved_tensors
        lat = ctx.lat
        _links(lat, U)
        G, _ = lat.force(ctx.ap, ctx.pf, ctx.solver, form=lgt.GRAD_G)
        return grad_S * lat.unpack_grad(G), None, None, None, None, None


class StoutSmear(torch.autograd.Function):
    """n levels of stout smearing U -> U_n; backward = the adjoint of each level.
    recompute=True keeps only the top level and recomputes the others in backward."""

    @staticmethod
    def forward(ctx, U, lat, rho, n_levels, recompute=False):
        _links(lat, U)
        Un = lat.stout_smear(rho, n_levels, recompute)
        ctx.save_for_backward(U)
        ctx.lat, ctx.rho, ctx.n, ctx.rc = lat, rho, n_levels, recompute
        return Un

    @staticmethod
    def backward(ctx, grad_Un):
        (U,) = ctx.saved_tensors
        lat = ctx.lat
        _links(lat, U)
        G = lat.stout_backward(ctx.rho, ctx.n, grad_Un.contiguous(), ctx.rc)
        return G, None, None, None, None


def total_action(U, phi, lat, beta, kappa, n_stout=0, rho=0.0, even_odd=False, solver=None,
                 recompute=False):
    """S_G(U) + S_f(smear^n(U)): the gauge action on thin links, the pseudofermion
    action on the smeared links."""
    solver = solver or lgt.solver("fp64", tol=1e-12)
    S = GaugeAction.apply(U, lat, beta)
    Uf = StoutSmear.apply(U, lat, rho, n_stout, recompute) if n_stout > 0 else U
    return S + PseudofermionAction.apply(Uf, phi, lat, kappa, even_odd, solver)


def lie_force(lat, U, G):
    """Lie components F_a = Re tr(G^+ i T^a U) in the canonical (V, 4, 8) layout."""
    _links(lat, U)
    Gf = lat.pack_grad(G)
    F = lat.momentum_field()
    lgt.check(lgt.lib().lgt_grad_to_lie(lat.h, lgt._ptr(Gf), lgt._ptr(F)))
    return lat.unpack_momenta(F)
