"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module holds no arithmetic of the method (no Dirac operator, no action, no
force, no link update).  It only draws seeded random numbers and shapes them into
the input recipe of the workloads: gauge links ``exp(i alpha H)`` with ``H`` a
Gaussian su(3) matrix per link, complex Gaussian spinors with ``Re, Im ~ N(0,1/2)``,
Gaussian momenta, and random SU(3) gauge transformations.  The exponential of a
Hermitian matrix is taken from numpy's eigendecomposition.

Arrays use the canonical full-lattice layout (site ``s = x0 + L0*(x1 + L1*(x2 +
L2*x3))``): links ``(V,4,3,3)`` complex128, spinors ``(V,4,3)`` complex128,
momenta ``(V,4,8)`` float64.
"""
import numpy as np

_SQ3 = 1.0 / np.sqrt(3.0)
# Gell-Mann basis / 2: the su(3) coordinates in which H is drawn
_T = 0.5 * np.array([
    [[0, 1, 0], [1, 0, 0], [0, 0, 0]],
    [[0, -1j, 0], [1j, 0, 0], [0, 0, 0]],
    [[1, 0, 0], [0, -1, 0], [0, 0, 0]],
    [[0, 0, 1], [0, 0, 0], [1, 0, 0]],
    [[0, 0, -1j], [0, 0, 0], [1j, 0, 0]],
    [[0, 0, 0], [0, 0, 1], [0, 1, 0]],
    [[0, 0, 0], [0, 0, -1j], [0, 1j, 0]],
    [[_SQ3, 0, 0], [0, _SQ3, 0], [0, 0, -2 * _SQ3]],
], dtype=np.complex128)


def volume(dims):
    return int(np.prod(dims))


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _expi_hermitian(H, alpha):
    """exp(i alpha H) for a stack of Hermitian matrices via eigh."""
    w, v = np.linalg.eigh(H)
    ph = np.exp(1j * alpha * w)
    return np.einsum("...ij,...j,...kj->...ik", v, ph, v.conj())


def random_links(dims, alpha, seed):
    """U_mu(x) = exp(i alpha sum_a h_a T^a), h_a ~ N(0,1), projected to det 1."""
    V = volume(dims)
    h = _rng(seed).standard_normal((V, 4, 8))
    H = np.einsum("...a,aij->...ij", h, _T)
    U = _expi_hermitian(H, alpha)
    # eigh is exact to rounding; remove the rounding phase of the determinant
    det = np.linalg.det(U)
    U = U * (det ** (-1.0 / 3.0))[..., None, None]
    return np.ascontiguousarray(U)


def gaussian_spinor(dims, seed, parity_mask=3):
    """Complex Gaussian spinor, Re/Im ~ N(0,1/2), zero outside parity_mask."""
    V = volume(dims)
    g = _rng(seed).standard_normal((V, 4, 3, 2)) * np.sqrt(0.5)
    psi = g[..., 0] + 1j * g[..., 1]
    par = parity(dims)
    keep = ((parity_mask >> par) & 1).astype(bool)
    psi[~keep] = 0
    return np.ascontiguousarray(psi)


def gaussian_momenta(dims, seed):
    return np.ascontiguousarray(_rng(seed).standard_normal((volume(dims), 4, 8)))


def random_su3(n, seed, alpha=3.0):
    """n random SU(3) matrices (exp of a wide Gaussian su(3) element)."""
    h = _rng(seed).standard_normal((n, 8))
    H = np.einsum("na,aij->nij", h, _T)
    U = _expi_hermitian(H, alpha)
    det = np.linalg.det(U)
    return U * (det ** (-1.0 / 3.0))[..., None, None]


def coords(dims):
    """(V, 4) integer coordinates of every site in canonical order."""
    L0, L1, L2, L3 = dims
    x3, x2, x1, x0 = np.meshgrid(np.arange(L3), np.arange(L2), np.arange(L1), np.arange(L0),
                                 indexing="ij")
    return np.stack([x0.ravel(), x1.ravel(), x2.ravel(), x3.ravel()], axis=1)


def parity(dims):
    return coords(dims).sum(axis=1) & 1
