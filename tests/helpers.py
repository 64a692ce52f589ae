"""Test-side arithmetic that pins the oracle and the CUDA path from outside.

Nothing here restates the oracle's formulas: gauge transformations, plane waves,
finite differences and dense-matrix constructions are independent checks.
"""
import numpy as np
import scipy.linalg

from paper_2602_20516_b300 import synth

GELLMANN_T = synth._T


def neighbour(dims, mu, step):
    """Index of x + step*mu for every site x (periodic)."""
    c = synth.coords(dims).copy()
    c[:, mu] = (c[:, mu] + step) % dims[mu]
    L0, L1, L2, _ = dims
    return c[:, 0] + L0 * (c[:, 1] + L1 * (c[:, 2] + L2 * c[:, 3]))


def gauge_transform_links(dims, U, g):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^+."""
    out = np.empty_like(U)
    for mu in range(4):
        fw = neighbour(dims, mu, +1)
        out[:, mu] = g @ U[:, mu] @ np.conj(np.swapaxes(g[fw], -1, -2))
    return out


def gauge_transform_spinor(psi, g):
    return np.einsum("xab,xsb->xsa", g, psi)


def gauge_transform_adjoint(F8, g):
    """Lie components of g F g^+ for F = sum_a F_a T^a (per link)."""
    Fm = np.einsum("xma,aij->xmij", F8, GELLMANN_T)
    gF = np.einsum("xab,xmbc,xdc->xmad", g, Fm, g.conj())
    return lie_components(gF)


def lie_components(M):
    """F_a = 2 Re tr(T^a M) for Hermitian traceless M."""
    return 2.0 * np.real(np.einsum("aij,...ji->...a", GELLMANN_T, M))


def plane_wave(dims, n, u):
    """psi(x) = exp(i p.x) u with p_k = 2 pi n_k / L_k (k<3), p_3 = (2 n_3 + 1) pi / L_3."""
    p = np.array([2 * np.pi * n[k] / dims[k] for k in range(3)] + [(2 * n[3] + 1) * np.pi / dims[3]])
    ph = np.exp(1j * synth.coords(dims) @ p)
    return ph[:, None, None] * u[None, :, :], p


def lie_perturb(U, site, mu, a, h):
    V = U.copy()
    V[site, mu] = scipy.linalg.expm(1j * h * GELLMANN_T[a]) @ U[site, mu]
    return V


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / np.linalg.norm(np.ravel(b)))


def dense_operator(apply, n_sites, shape=(4, 3), sites=None):
    """Dense matrix of a linear map on spinor fields by applying it to unit vectors."""
    dim = n_sites * 12
    cols = []
    idx = range(dim) if sites is None else [s * 12 + k for s in sites for k in range(12)]
    for j in idx:
        e = np.zeros(dim, np.complex128)
        e[j] = 1
        cols.append(apply(e.reshape((n_sites,) + shape)).ravel())
    return np.array(cols).T
