"""Plain FP64 CPU oracle for the HMC hot path of arXiv:2602.20516.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and the CUDA library never calls it.

Arrays are numpy, canonical full-lattice layout, site index
``s = x0 + L0*(x1 + L1*(x2 + L2*x3))`` (mu = 3 is time):

* links     complex128 ``(V, 4, 3, 3)``
* spinors   complex128 ``(V, 4, 3)``   (spin, colour)
* momenta / forces  float64 ``(V, 4, 8)``  (coefficients of T^a = lambda^a/2)
* gradients complex128 ``(V, 4, 3, 3)`` = dS/dReU + i dS/dImU (Eq. S2.11)

Every function says which passage of the paper it follows; the conventions the
paper leaves open are stated in ``oracle.h``.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None

FIELD_MOMENTA, FIELD_XI, FIELD_LINKS, FIELD_METROPOLIS, FIELD_SOURCE = 1, 2, 3, 4, 5

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


class HMCParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("kappa", C.c_double), ("eo", C.c_int),
                ("fermions", C.c_int), ("integrator", C.c_int), ("n_steps", C.c_int),
                ("tau", C.c_double), ("tol_md", C.c_double), ("tol_action", C.c_double),
                ("max_iter", C.c_int), ("n_inner", C.c_int), ("n_stout", C.c_int), ("rho", C.c_double),
                ("c1", C.c_double), ("csw", C.c_double)]


class HMCResult(C.Structure):
    _fields_ = [("dH", C.c_double), ("Sg_old", C.c_double), ("Sg_new", C.c_double),
                ("Sf_old", C.c_double), ("Sf_new", C.c_double), ("K_old", C.c_double),
                ("K_new", C.c_double), ("plaquette", C.c_double), ("accepted", C.c_int),
                ("cg_iters", C.c_int), ("force_evals", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        sig = {
            "ora_volume": (C.c_long, [_ip]),
            "ora_philox4x32_10": (None, [np.ctypeslib.ndpointer(np.uint32), np.ctypeslib.ndpointer(np.uint32), np.ctypeslib.ndpointer(np.uint32)]),
            "ora_gauss_pair": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, _dp]),
            "ora_uniform": (C.c_double, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]),
            "ora_gamma": (None, [C.c_int, _cp]),
            "ora_gellmann_T": (None, [C.c_int, _cp]),
            "ora_expm": (None, [C.c_int, _cp, _cp]),
            "ora_random_links": (None, [_ip, C.c_uint64, C.c_double, _cp]),
            "ora_gaussian_momenta": (None, [_ip, C.c_uint64, C.c_uint32, _dp]),
            "ora_gaussian_spinor": (None, [_ip, C.c_uint64, C.c_uint32, C.c_uint32, C.c_int, _cp]),
            "ora_hop": (None, [_ip, _cp, _cp, _cp, C.c_int, C.c_int]),
            "ora_dirac": (None, [_ip, _cp, C.c_double, _cp, _cp, C.c_int]),
            "ora_dhat": (None, [_ip, _cp, C.c_double, _cp, _cp, C.c_int]),
            "ora_cg": (C.c_int, [_ip, _cp, C.c_double, C.c_int, _cp, _cp, C.c_double, C.c_int, C.POINTER(C.c_double)]),
            "ora_plaquette_sum": (C.c_double, [_ip, _cp]),
            "ora_gauge_action": (C.c_double, [_ip, _cp, C.c_double]),
            "ora_gauge_action_imp": (C.c_double, [_ip, _cp, C.c_double, C.c_double]),
            "ora_rectangle_sum": (C.c_double, [_ip, _cp]),
            "ora_clover_field_strength": (None, [_ip, _cp, C.c_int, C.c_int, _cp]),
            "ora_clover_term": (None, [_ip, _cp, C.c_double, C.c_double, _cp]),
            "ora_dirac_sw": (None, [_ip, _cp, C.c_double, C.c_double, _cp, _cp, C.c_int]),
            "ora_cg_sw": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, _cp, C.c_double, C.c_int,
                                    C.POINTER(C.c_double)]),
            "ora_pf_action_sw": (C.c_double, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int,
                                              C.POINTER(C.c_int)]),
            "ora_pf_action_grad_sw": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int, _cp]),
            "ora_pf_force_sw": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int,
                                          C.c_double, _dp]),
            "ora_dhat_sw": (None, [_ip, _cp, C.c_double, C.c_double, _cp, _cp, C.c_int]),
            "ora_clover_logdet_odd": (C.c_double, [_ip, _cp, C.c_double, C.c_double]),
            "ora_cg_sw_eo": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, _cp, C.c_double, C.c_int,
                                       C.POINTER(C.c_double)]),
            "ora_pf_action_sw_eo": (C.c_double, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int,
                                                 C.POINTER(C.c_int)]),
            "ora_pf_action_grad_sw_eo": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int,
                                                   _cp]),
            "ora_pf_force_sw_eo": (C.c_int, [_ip, _cp, C.c_double, C.c_double, _cp, C.c_double, C.c_int,
                                             C.c_double, _dp]),
            "ora_gauge_force_imp": (None, [_ip, _cp, C.c_double, C.c_double, C.c_double, _dp]),
            "ora_gauge_action_grad_imp": (None, [_ip, _cp, C.c_double, C.c_double, _cp]),
            "ora_pf_action": (C.c_double, [_ip, _cp, C.c_double, C.c_int, _cp, C.c_double, C.c_int, C.POINTER(C.c_int)]),
            "ora_momentum_energy": (C.c_double, [_ip, _dp]),
            "ora_gauge_force": (None, [_ip, _cp, C.c_double, C.c_double, _dp]),
            "ora_fermion_force_xy": (None, [_ip, _cp, C.c_double, _cp, _cp, C.c_double, _dp]),
            "ora_pf_force": (C.c_int, [_ip, _cp, C.c_double, C.c_int, _cp, C.c_double, C.c_int, C.c_double, _dp]),
            "ora_grad_to_force": (None, [_ip, _cp, _cp, _dp]),
            "ora_gauge_action_grad": (None, [_ip, _cp, C.c_double, _cp]),
            "ora_pf_action_grad": (C.c_int, [_ip, _cp, C.c_double, C.c_int, _cp, C.c_double, C.c_int, _cp]),
            "ora_update_links": (None, [_ip, _cp, _dp, C.c_double]),
            "ora_kick": (None, [_ip, _dp, _dp, C.c_double]),
            "ora_reunitarise": (None, [_ip, _cp]),
            "ora_stout_forward": (None, [_ip, _cp, C.c_double, _cp]),
            "ora_stout_backward": (None, [_ip, _cp, C.c_double, _cp, _cp]),
            "ora_md_force": (C.c_int, [_ip, _cp, C.POINTER(HMCParams), _cp, _dp]),
            "ora_md_force_part": (C.c_int, [_ip, _cp, C.POINTER(HMCParams), _cp, C.c_int, _dp]),
            "ora_hamiltonian": (C.c_double, [_ip, _cp, _dp, _cp, C.POINTER(HMCParams)]),
            "ora_md_integrate": (C.c_int, [_ip, _cp, _dp, _cp, C.POINTER(HMCParams)]),
            "ora_hmc_trajectory": (C.c_int, [_ip, _cp, C.POINTER(HMCParams), C.c_uint64, C.c_uint32, C.POINTER(HMCResult)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _dims(dims):
    d = np.ascontiguousarray(dims, dtype=np.int32)
    assert d.shape == (4,) and all(int(v) % 2 == 0 and int(v) >= 2 for v in d), "extents must be even"
    return d


def volume(dims):
    return int(np.prod(dims))


def _c(a, dtype=np.complex128):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------- random numbers
def philox4x32_10(ctr, key):
    """Philox-4x32-10 block function (Salmon et al., SC'11)."""
    out = np.zeros(4, np.uint32)
    lib().ora_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def gauss_pair(seed, c0, c1, c2, c3):
    g = np.zeros(2)
    lib().ora_gauss_pair(seed, c0, c1, c2, c3, g)
    return g


def uniform(seed, c0, c1, c2, c3):
    return lib().ora_uniform(seed, c0, c1, c2, c3)


# ---------------------------------------------------------------- small matrices
def gamma(mu):
    g = np.zeros(16, np.complex128)
    lib().ora_gamma(mu, g)
    return g.reshape(4, 4)


def gellmann_T(a):
    t = np.zeros(9, np.complex128)
    lib().ora_gellmann_T(a, t)
    return t.reshape(3, 3)


def expm(A):
    A = _c(A)
    n = A.shape[0]
    out = np.zeros_like(A)
    lib().ora_expm(n, A, out)
    return out


# ---------------------------------------------------------------- seeded fields
def random_links(dims, seed, alpha):
    d = _dims(dims)
    U = np.zeros((volume(d), 4, 3, 3), np.complex128)
    lib().ora_random_links(d, seed, alpha, U)
    return U


def gaussian_momenta(dims, seed, traj=0):
    d = _dims(dims)
    m = np.zeros((volume(d), 4, 8))
    lib().ora_gaussian_momenta(d, seed, traj, m)
    return m


def gaussian_spinor(dims, seed, traj=0, field=FIELD_SOURCE, parity_mask=3):
    d = _dims(dims)
    p = np.zeros((volume(d), 4, 3), np.complex128)
    lib().ora_gaussian_spinor(d, seed, traj, field, parity_mask, p)
    return p


# ---------------------------------------------------------------- Dirac operator
def hop(dims, U, psi, out_mask=3, dagger=False, out=None):
    d = _dims(dims)
    o = np.zeros_like(_c(psi)) if out is None else out
    lib().ora_hop(d, _c(U), _c(psi), o, out_mask, int(dagger))
    return o


def dirac(dims, U, kappa, psi, dagger=False):
    d = _dims(dims)
    o = np.zeros_like(_c(psi))
    lib().ora_dirac(d, _c(U), kappa, _c(psi), o, int(dagger))
    return o


def dhat(dims, U, kappa, psi, dagger=False):
    d = _dims(dims)
    o = np.zeros_like(_c(psi))
    lib().ora_dhat(d, _c(U), kappa, _c(psi), o, int(dagger))
    return o


def cg(dims, U, kappa, b, eo=False, tol=1e-12, max_iter=10000):
    """Solve (M^+M) x = b; returns (x, iterations, true relative residual)."""
    d = _dims(dims)
    x = np.zeros_like(_c(b))
    res = C.c_double()
    it = lib().ora_cg(d, _c(U), kappa, int(eo), _c(b), x, tol, max_iter, C.byref(res))
    return x, it, res.value


# ---------------------------------------------------------------- actions
def plaquette_sum(dims, U):
    return lib().ora_plaquette_sum(_dims(dims), _c(U))


def plaquette(dims, U):
    return plaquette_sum(dims, U) / (6.0 * volume(dims))


def gauge_action(dims, U, beta, c1=0.0):
    """beta sum [c0 (1 - Re tr P / 3) + c1 (1 - Re tr R / 3)], c0 = 1 - 8 c1 (c1 = 0: Wilson)."""
    if c1 == 0.0:
        return lib().ora_gauge_action(_dims(dims), _c(U), beta)
    return lib().ora_gauge_action_imp(_dims(dims), _c(U), beta, c1)


# ---------------------------------------------------------------- clover term (full lattice)
def clover_field_strength(dims, U, mu, nu):
    """F_munu(x) = (Q - Q^+)/(8i), Q the four leaves of the mu-nu plane at x: (V, 3, 3)."""
    d = _dims(dims)
    F = np.zeros((volume(d), 3, 3), np.complex128)
    lib().ora_clover_field_strength(d, _c(U), mu, nu, F)
    return F


def clover_term(dims, U, kappa, csw):
    """A(x) = -kappa c_sw sum_{mu<nu} sigma_munu F_munu(x) as (V, 12, 12), index 3 spin + colour."""
    d = _dims(dims)
    A = np.zeros((volume(d), 12, 12), np.complex128)
    lib().ora_clover_term(d, _c(U), kappa, csw, A)
    return A


def dirac_sw(dims, U, kappa, csw, psi, dagger=False):
    d = _dims(dims)
    out = np.zeros_like(_c(psi))
    lib().ora_dirac_sw(d, _c(U), kappa, csw, _c(psi), out, int(dagger))
    return out


def cg_sw(dims, U, kappa, csw, b, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    x = np.zeros_like(_c(b))
    res = C.c_double()
    it = lib().ora_cg_sw(d, _c(U), kappa, csw, _c(b), x, tol, max_iter, C.byref(res))
    return x, it, res.value


def pf_action_sw(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    it = C.c_int()
    S = lib().ora_pf_action_sw(_dims(dims), _c(U), kappa, csw, _c(phi), tol, max_iter, C.byref(it))
    return S, it.value


def pf_action_grad_sw(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    G = np.zeros((volume(d), 4, 3, 3), np.complex128)
    it = lib().ora_pf_action_grad_sw(d, _c(U), kappa, csw, _c(phi), tol, max_iter, G)
    return G, it


def pf_force_sw(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    it = lib().ora_pf_force_sw(d, _c(U), kappa, csw, _c(phi), tol, max_iter, 1.0, F)
    return F, it


def dhat_sw(dims, U, kappa, csw, psi, dagger=False):
    """Dhat = M_ee - kappa^2 H_eo M_oo^{-1} H_oe (M = 1 + A) on the even sites of psi."""
    d = _dims(dims)
    out = np.zeros_like(_c(psi))
    lib().ora_dhat_sw(d, _c(U), kappa, csw, _c(psi), out, int(dagger))
    return out


def clover_logdet_odd(dims, U, kappa, csw):
    """sum over odd sites x of ln det (1 + A(x))."""
    return lib().ora_clover_logdet_odd(_dims(dims), _c(U), kappa, csw)


def cg_sw_eo(dims, U, kappa, csw, b, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    x = np.zeros_like(_c(b))
    res = C.c_double()
    it = lib().ora_cg_sw_eo(d, _c(U), kappa, csw, _c(b), x, tol, max_iter, C.byref(res))
    return x, it, res.value


def pf_action_sw_eo(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    """phi_e^+ (Dhat^+ Dhat)^{-1} phi_e - 2 ln det M_oo."""
    it = C.c_int()
    S = lib().ora_pf_action_sw_eo(_dims(dims), _c(U), kappa, csw, _c(phi), tol, max_iter, C.byref(it))
    return S, it.value


def pf_action_grad_sw_eo(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    G = np.zeros((volume(d), 4, 3, 3), np.complex128)
    it = lib().ora_pf_action_grad_sw_eo(d, _c(U), kappa, csw, _c(phi), tol, max_iter, G)
    return G, it


def pf_force_sw_eo(dims, U, kappa, csw, phi, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    it = lib().ora_pf_force_sw_eo(d, _c(U), kappa, csw, _c(phi), tol, max_iter, 1.0, F)
    return F, it


def rectangle_sum(dims, U):
    """sum over x and ordered mu != nu of Re tr R_munu(x) / 3 (2 x 1 loops, long side mu)."""
    return lib().ora_rectangle_sum(_dims(dims), _c(U))


def pf_action(dims, U, kappa, phi, eo=False, tol=1e-12, max_iter=10000):
    it = C.c_int()
    S = lib().ora_pf_action(_dims(dims), _c(U), kappa, int(eo), _c(phi), tol, max_iter, C.byref(it))
    return S, it.value


def momentum_energy(dims, mom):
    return lib().ora_momentum_energy(_dims(dims), _c(mom, np.float64))


# ---------------------------------------------------------------- forces
def gauge_force(dims, U, beta, c1=0.0):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    if c1 == 0.0:
        lib().ora_gauge_force(d, _c(U), beta, 1.0, F)
    else:
        lib().ora_gauge_force_imp(d, _c(U), beta, c1, 1.0, F)
    return F


def fermion_force_xy(dims, U, kappa, X, Y):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    lib().ora_fermion_force_xy(d, _c(U), kappa, _c(X), _c(Y), 1.0, F)
    return F


def pf_force(dims, U, kappa, phi, eo=False, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    it = lib().ora_pf_force(d, _c(U), kappa, int(eo), _c(phi), tol, max_iter, 1.0, F)
    return F, it


def grad_to_force(dims, U, G):
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    lib().ora_grad_to_force(d, _c(U), _c(G), F)
    return F


def gauge_action_grad(dims, U, beta, c1=0.0):
    d = _dims(dims)
    G = np.zeros((volume(d), 4, 3, 3), np.complex128)
    if c1 == 0.0:
        lib().ora_gauge_action_grad(d, _c(U), beta, G)
    else:
        lib().ora_gauge_action_grad_imp(d, _c(U), beta, c1, G)
    return G


def pf_action_grad(dims, U, kappa, phi, eo=False, tol=1e-12, max_iter=10000):
    d = _dims(dims)
    G = np.zeros((volume(d), 4, 3, 3), np.complex128)
    it = lib().ora_pf_action_grad(d, _c(U), kappa, int(eo), _c(phi), tol, max_iter, G)
    return G, it


# ---------------------------------------------------------------- updates
def update_links(dims, U, mom, eps):
    U = _c(U).copy()
    lib().ora_update_links(_dims(dims), U, _c(mom, np.float64), eps)
    return U


def reunitarise(dims, U):
    U = _c(U).copy()
    lib().ora_reunitarise(_dims(dims), U)
    return U


def stout_forward(dims, U, rho):
    d = _dims(dims)
    out = np.zeros_like(_c(U))
    lib().ora_stout_forward(d, _c(U), rho, out)
    return out


def stout_backward(dims, U, rho, Gout):
    d = _dims(dims)
    Gin = np.zeros_like(_c(U))
    lib().ora_stout_backward(d, _c(U), rho, _c(Gout), Gin)
    return Gin


# ---------------------------------------------------------------- HMC
INTEGRATORS = {"leapfrog": 0, "omelyan": 1, "sexton_weingarten": 2}


def hmc_params(beta, kappa, eo=False, fermions=True, integrator="leapfrog", n_steps=10,
               tau=1.0, tol_md=1e-12, tol_action=1e-12, max_iter=10000, n_inner=1, n_stout=0, rho=0.0, c1=0.0,
               csw=0.0):
    return HMCParams(beta, kappa, int(eo), int(fermions), INTEGRATORS[integrator], n_steps, tau, tol_md,
                     tol_action, max_iter, n_inner, n_stout, rho, c1, csw)


def md_force(dims, U, params, phi, part=0):
    """MD force (Lie components); part 0 all, 1 gauge only, 2 fermion only."""
    d = _dims(dims)
    F = np.zeros((volume(d), 4, 8))
    lib().ora_md_force_part(d, _c(U), C.byref(params), _c(phi), part, F)
    return F


def hamiltonian(dims, U, mom, phi, params):
    return lib().ora_hamiltonian(_dims(dims), _c(U), _c(mom, np.float64), _c(phi), C.byref(params))


def md_integrate(dims, U, mom, phi, params):
    U = _c(U).copy()
    mom = _c(mom, np.float64).copy()
    it = lib().ora_md_integrate(_dims(dims), U, mom, _c(phi), C.byref(params))
    return U, mom, it


def hmc_trajectory(dims, U, params, seed, traj):
    U = _c(U).copy()
    res = HMCResult()
    lib().ora_hmc_trajectory(_dims(dims), U, C.byref(params), seed, traj, C.byref(res))
    return U, res.as_dict()
