"""Python binding of liblgt.so (argument marshalling only).

Every operation runs in the CUDA kernels of ``liblgt.so``; this module converts
torch tensors to device pointers and C structs.  PyTorch provides device memory
(its caching allocator backs the library's workspace) and the stream.  There is
no fallback: if the library or a CUDA device is missing, constructing a
``Lattice`` raises.
"""
import ctypes as C
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblgt.so")

FP64, MIXED, FP32, DF64 = 0, 1, 2, 3
EVEN, ODD, FULL = 0, 1, 2
OP_HOP, OP_D, OP_DHAT, OP_DHAT_NORMAL = 0, 1, 2, 3
LEAPFROG, OMELYAN2MN = 0, 1
FORCE_LIE, GRAD_G = 0, 1
UPDATE_U, UPDATE_P = 0, 1
FIELD_MOMENTA, FIELD_XI, FIELD_LINKS, FIELD_METROPOLIS, FIELD_SOURCE = 1, 2, 3, 4, 5

STATUS = {0: "LGT_OK", 1: "LGT_EINVAL", 2: "LGT_ENOMEM", 3: "LGT_ENOCONV", 4: "LGT_ENAN",
          5: "LGT_ECUDA", 6: "LGT_EKERNEL"}


class LGTError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class SolverParams(C.Structure):
    _fields_ = [("precision", C.c_int), ("tol", C.c_double), ("max_iter", C.c_int),
                ("delta", C.c_double), ("check_every", C.c_int), ("chrono", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iters", C.c_int), ("reliable_updates", C.c_int),
                ("true_rel_residual", C.c_double), ("seconds", C.c_double),
                ("breakdowns", C.c_int), ("diverged", C.c_int), ("handovers", C.c_int),
                ("fp64_iters", C.c_int), ("restarts", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ActionParams(C.Structure):
    _fields_ = [("beta", C.c_double), ("kappa", C.c_double), ("fermions", C.c_int),
                ("even_odd", C.c_int), ("n_stout", C.c_int), ("rho", C.c_double),
                ("stout_recompute", C.c_int), ("force_arith", C.c_int), ("c1", C.c_double),
                ("csw", C.c_double)]


class HMCParams(C.Structure):
    _fields_ = [("integrator", C.c_int), ("n_steps", C.c_int), ("tau", C.c_double),
                ("md_solver", SolverParams), ("action_solver", SolverParams), ("n_inner", C.c_int)]


class HMCResult(C.Structure):
    _fields_ = [("dH", C.c_double), ("Sg_old", C.c_double), ("Sg_new", C.c_double),
                ("Sf_old", C.c_double), ("Sf_new", C.c_double), ("K_old", C.c_double),
                ("K_new", C.c_double), ("plaquette", C.c_double), ("accepted", C.c_int),
                ("force_evals", C.c_int), ("total", SolveStats)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "total"}
        d["total"] = self.total.as_dict()
        return d


REQ_SOLVE, REQ_FORCE = 0, 1


class Request(C.Structure):
    _fields_ = [("gauge_id", C.c_int), ("kind", C.c_int), ("precision", C.c_int), ("kappa", C.c_double),
                ("beta", C.c_double), ("tol", C.c_double), ("max_iter", C.c_int),
                ("source_seed", C.c_uint64), ("keep_result", C.c_int)]


class Completion(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int), ("iters", C.c_int), ("reliable_updates", C.c_int),
                ("true_rel_residual", C.c_double), ("t_submit", C.c_double), ("t_admit", C.c_double),
                ("t_done", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


_lib = None

# (name, restype, argtypes) of every symbol declared in include/lgt.h
_P, _I, _D, _U64, _U32, _SZ = C.c_void_p, C.c_int, C.c_double, C.c_uint64, C.c_uint32, C.c_size_t
SIGNATURES = [
    ("lgt_last_error", C.c_char_p, []),
    ("lgt_version", _I, []),
    ("lgt_create_lattice", _I, [C.POINTER(C.c_int), C.POINTER(Allocator), _P, C.POINTER(_P)]),
    ("lgt_destroy_lattice", _I, [_P]),
    ("lgt_set_stream", _I, [_P, _P]),
    ("lgt_lattice_info", _I, [_P, C.POINTER(C.c_int64), C.POINTER(_SZ)]),
    ("lgt_field_bytes", _I, [_P, _I, _I, _I, C.POINTER(_SZ)]),
    ("lgt_set_links", _I, [_P, _P]),
    ("lgt_get_links", _I, [_P, _P]),
    ("lgt_random_links", _I, [_P, _U64, _D]),
    ("lgt_reunitarise", _I, [_P]),
    ("lgt_plaquette", _I, [_P, C.POINTER(_D)]),
    ("lgt_rectangle", _I, [_P, C.POINTER(_D)]),
    ("lgt_plaquette_noalloc", _I, [_P, C.POINTER(C.c_int), _P, _P]),
    ("lgt_pack_spinor", _I, [_P, _P, _P, _I, _I]),
    ("lgt_unpack_spinor", _I, [_P, _P, _P, _I, _I]),
    ("lgt_pack_momenta", _I, [_P, _P, _P]),
    ("lgt_unpack_momenta", _I, [_P, _P, _P]),
    ("lgt_pack_links_field", _I, [_P, _P, _P]),
    ("lgt_unpack_links_field", _I, [_P, _P, _P]),
    ("lgt_set_clover", _I, [_P, _D, _D]),
    ("lgt_set_sweep_order", _I, [_P, _I]),
    ("lgt_set_hop_staging", _I, [_P, _I]),
    ("lgt_hop_staging_status", _I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_uint)]),
    ("lgt_save_checkpoint", _I, [_P, C.c_char_p, C.c_uint64, C.c_uint64]),
    ("lgt_load_checkpoint", _I, [_P, C.c_char_p, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
    ("lgt_dslash", _I, [_P, _P, _P, _I, _I, _I, _D, _I]),
    ("lgt_cg_solve", _I, [_P, _P, _P, _D, _I, C.POINTER(SolverParams), C.POINTER(SolveStats)]),
    ("lgt_cg_solve_multi", _I, [_P, _I, C.POINTER(_P), C.POINTER(_P), C.POINTER(_D), C.POINTER(SolverParams),
                                C.POINTER(SolveStats)]),
    ("lgt_hop_multi", _I, [_P, _I, C.POINTER(_P), C.POINTER(_P), _I, _I]),
    ("lgt_chrono_reset", _I, [_P]),
    ("lgt_action", _I, [_P, C.POINTER(ActionParams), _P, C.POINTER(SolverParams), C.POINTER(_D),
                        C.POINTER(_D), C.POINTER(SolveStats)]),
    ("lgt_kinetic_energy", _I, [_P, _P, C.POINTER(_D)]),
    ("lgt_force", _I, [_P, C.POINTER(ActionParams), _P, C.POINTER(SolverParams), _P, _I,
                       C.POINTER(SolveStats)]),
    ("lgt_md_update", _I, [_P, _P, _D, _I, C.POINTER(ActionParams), _P, C.POINTER(SolverParams),
                           C.POINTER(SolveStats)]),
    ("lgt_grad_to_lie", _I, [_P, _P, _P]),
    ("lgt_stout_smear", _I, [_P, _D, _I, _I, _P]),
    ("lgt_stout_backward", _I, [_P, _D, _I, _I, _P, _P]),
    ("lgt_gaussian_momenta", _I, [_P, _P, _U64, _U32]),
    ("lgt_gaussian_spinor", _I, [_P, _P, _U64, _U32, _U32, _I]),
    ("lgt_hmc_trajectory", _I, [_P, C.POINTER(ActionParams), C.POINTER(HMCParams), _U64, _U32,
                                C.POINTER(HMCResult)]),
    ("lgt_server_create", _I, [C.POINTER(Allocator), _SZ, _I, _I, _D, _P, C.POINTER(_P)]),
    ("lgt_server_destroy", _I, [_P]),
    ("lgt_server_add_gauge", _I, [_P, C.POINTER(C.c_int), _U64, _D, C.POINTER(C.c_int)]),
    ("lgt_server_get_links", _I, [_P, _I, _P]),
    ("lgt_server_submit", _I, [_P, C.POINTER(Request), C.POINTER(C.c_uint64)]),
    ("lgt_server_step", _I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lgt_server_poll", _I, [_P, C.POINTER(Completion), _I, C.POINTER(C.c_int)]),
    ("lgt_server_result", _I, [_P, C.c_uint64, _P, _SZ]),
    ("lgt_server_info", _I, [_P, C.POINTER(_SZ), C.POINTER(_SZ), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    ("lgt_clock", C.c_double, []),
    ("lgt_measure_fp64_peak", _I, [C.POINTER(_D), C.POINTER(_D)]),
    ("lgt_kernel_timing_start", _I, [_I]),
    ("lgt_kernel_timing_sample", _I, [_I]),
    ("lgt_kernel_timing_stop", _I, [_D, C.POINTER(_D), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    ("lgt_launch_count", C.c_int64, [_I]),
]


def lib():
    """Load liblgt.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with python -m paper_2602_20516_b300.build")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(rc):
    if rc != 0:
        raise LGTError(rc, lib().lgt_last_error().decode())


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def solver(precision="fp64", tol=1e-10, max_iter=10000, delta=1e-3, check_every=16, chrono=0):
    """chrono = N > 0: even-odd solves start from the best combination of the handle's
    last N solutions of the same operator (chronological initial guess)."""
    prec = {"fp64": FP64, "mixed": MIXED}[precision] if isinstance(precision, str) else precision
    return SolverParams(prec, tol, max_iter, delta, check_every, chrono)


ARITH = {"fp64": 0, "fp32": 1, "df64": 2}


def action_params(beta=0.0, kappa=0.0, fermions=True, even_odd=False, n_stout=0, rho=0.0,
                  stout_recompute=False, force_arith="fp64", c1=0.0, csw=0.0):
    """force_arith: arithmetic of Lie-form forces with the mixed solver ("fp64",
    "fp32" or "df64", the double-float FP32-pair format); c1: rectangle weight of the
    gauge action (0 Wilson, -1/12 Symanzik, -0.331 Iwasaki, -1.4088 DBW2); csw:
    clover coefficient of the Wilson operator (full-lattice action only)."""
    return ActionParams(beta, kappa, int(fermions), int(even_odd), n_stout, rho, int(stout_recompute),
                        ARITH[force_arith] if isinstance(force_arith, str) else int(force_arith), c1, csw)


SEXTON_WEINGARTEN = 2


def hmc_params(integrator="leapfrog", n_steps=10, tau=1.0, md_solver=None, action_solver=None, n_inner=1):
    integ = {"leapfrog": LEAPFROG, "omelyan": OMELYAN2MN, "sexton_weingarten": SEXTON_WEINGARTEN}[integrator]
    return HMCParams(integ, n_steps, tau, md_solver or solver(), action_solver or solver(), n_inner)


def measure_fp64_peak():
    f, s = C.c_double(), C.c_double()
    check(lib().lgt_measure_fp64_peak(C.byref(f), C.byref(s)))
    return f.value


def kernel_timing_start(max_launches=65536, every=1):
    """Arm CUDA-event timing of the hop launches; every > 1 records only every
    every-th launch (a sample)."""
    check(lib().lgt_kernel_timing_sample(every))
    check(lib().lgt_kernel_timing_start(max_launches))


HOP_EPILOGUES = ["hop", "xpay", "xpay_norm", "cg_update", "residual"]
TIMING_KINDS = 15   # LGT_TIMING_KINDS
TIMING_ARITH = ["fp32", "fp64", "df64"]


def kernel_timing_stop(min_ms=0.0):
    """Per hop kind since kernel_timing_start: ({(precision, epilogue): (ms, count)},
    n_short); launches shorter than min_ms are only counted in n_short."""
    ms = (C.c_double * TIMING_KINDS)()
    n = (C.c_int64 * TIMING_KINDS)()
    short = C.c_int64()
    check(lib().lgt_kernel_timing_stop(min_ms, ms, n, C.byref(short)))
    out = {}
    for k in range(TIMING_KINDS):
        if n[k]:
            out[(TIMING_ARITH[k // 5], HOP_EPILOGUES[k % 5])] = (ms[k], n[k])
    return out, short.value


def launch_count(reset=False):
    return lib().lgt_launch_count(int(reset))


class Lattice:
    """A lattice handle: gauge field and solver workspace resident on one GPU.

    Device fields are torch tensors in the library's layouts (see include/lgt.h):
    FP64 spinor half field ``(12, Vh, 2)`` float64, full ``(2, 12, Vh, 2)``; FP32
    ``(6, Vh, 4)`` / ``(2, 6, Vh, 4)`` float32; momenta ``(2, 4, 4, Vh, 2)``; G-form
    ``(2, 4, 9, Vh, 2)``.  Canonical arrays: links ``(V, 4, 3, 3)`` complex128,
    spinors ``(V, 4, 3)`` complex128, momenta ``(V, 4, 8)`` float64.
    """

    def __init__(self, dims, device=None, stream=None, torch_allocator=True):
        if not torch.cuda.is_available():
            raise RuntimeError("liblgt needs a CUDA device")
        self.dims = tuple(int(d) for d in dims)
        self.V = int(np.prod(self.dims))
        self.Vh = self.V // 2
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        self._keep = []
        alloc = None
        if torch_allocator:
            dev = self.device.index

            def _a(ctx, nbytes, st):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st or 0)
                except RuntimeError:
                    return None

            def _f(ctx, ptr, st):
                torch.cuda.caching_allocator_delete(ptr)

            alloc = Allocator(ALLOC_FN(_a), FREE_FN(_f), None)
            self._keep.append(alloc)
        d = (C.c_int * 4)(*self.dims)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(lib().lgt_create_lattice(d, C.byref(alloc) if alloc else None,
                                           C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().lgt_destroy_lattice(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ tensors
    def _t(self, shape, dtype=torch.float64):
        return torch.zeros(shape, dtype=dtype, device=self.device)

    def spinor_field(self, parity=FULL, precision=FP64):
        if precision == FP32:
            return self._t((6, self.Vh, 4) if parity != FULL else (2, 6, self.Vh, 4), torch.float32)
        if precision == DF64:   # (re.hi, re.lo, im.hi, im.lo) per component
            return self._t((12, self.Vh, 4) if parity != FULL else (2, 12, self.Vh, 4), torch.float32)
        return self._t((12, self.Vh, 2) if parity != FULL else (2, 12, self.Vh, 2))

    def momentum_field(self):
        return self._t((2, 4, 4, self.Vh, 2))

    def grad_field(self):
        return self._t((2, 4, 9, self.Vh, 2))

    def _dev(self, a, dtype):
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a))
        return a.to(device=self.device, dtype=dtype).contiguous()

    # ------------------------------------------------------------ gauge field
    def set_links(self, U):
        U = self._dev(U, torch.complex128)
        assert U.shape == (self.V, 4, 3, 3)
        check(lib().lgt_set_links(self.h, _ptr(U)))
        self._sync()

    def get_links(self):
        U = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device=self.device)
        check(lib().lgt_get_links(self.h, _ptr(U)))
        self._sync()
        return U

    def random_links(self, seed, alpha):
        check(lib().lgt_random_links(self.h, seed, alpha))

    def reunitarise(self):
        check(lib().lgt_reunitarise(self.h))

    def rectangle(self):
        r = C.c_double()
        check(lib().lgt_rectangle(self.h, C.byref(r)))
        return r.value

    def plaquette(self):
        v = C.c_double()
        check(lib().lgt_plaquette(self.h, C.byref(v)))
        return v.value

    def info(self):
        v, b = C.c_int64(), C.c_size_t()
        check(lib().lgt_lattice_info(self.h, C.byref(v), C.byref(b)))
        return v.value, b.value

    def _sync(self):
        self.stream.synchronize()

    # ------------------------------------------------------------ layouts
    def pack_spinor(self, canon, parity=FULL, precision=FP64):
        c = self._dev(canon, torch.complex128)
        f = self.spinor_field(parity, precision)
        check(lib().lgt_pack_spinor(self.h, _ptr(c), _ptr(f), parity, precision))
        return f

    def unpack_spinor(self, field, parity=FULL, precision=FP64):
        c = torch.zeros((self.V, 4, 3), dtype=torch.complex128, device=self.device)
        check(lib().lgt_unpack_spinor(self.h, _ptr(field), _ptr(c), parity, precision))
        self._sync()
        return c

    def pack_momenta(self, canon):
        c = self._dev(canon, torch.float64)
        m = self.momentum_field()
        check(lib().lgt_pack_momenta(self.h, _ptr(c), _ptr(m)))
        return m

    def unpack_momenta(self, mom):
        c = torch.zeros((self.V, 4, 8), dtype=torch.float64, device=self.device)
        check(lib().lgt_unpack_momenta(self.h, _ptr(mom), _ptr(c)))
        self._sync()
        return c

    def pack_grad(self, canon):
        c = self._dev(canon, torch.complex128)
        g = self.grad_field()
        check(lib().lgt_pack_links_field(self.h, _ptr(c), _ptr(g)))
        return g

    def unpack_grad(self, field):
        c = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device=self.device)
        check(lib().lgt_unpack_links_field(self.h, _ptr(field), _ptr(c)))
        self._sync()
        return c

    # ------------------------------------------------------------ operators
    def set_clover(self, csw, kappa):
        """Attach (csw != 0) or detach (csw = 0) the clover term for OP_D and full-lattice solves."""
        check(lib().lgt_set_clover(self.h, csw, kappa))

    def save_checkpoint(self, path, seed, next_traj):
        """Write the links, seed and next trajectory index (lgt_save_checkpoint)."""
        check(lib().lgt_save_checkpoint(self.h, os.fsencode(path), int(seed), int(next_traj)))

    def load_checkpoint(self, path):
        """Set the links from a checkpoint; returns (seed, next trajectory index)."""
        seed, nxt = C.c_uint64(), C.c_uint64()
        check(lib().lgt_load_checkpoint(self.h, os.fsencode(path), C.byref(seed), C.byref(nxt)))
        return seed.value, nxt.value

    def set_sweep_order(self, alternate=True):
        """Alternate the site order of consecutive CG launches (default) or walk forward."""
        check(lib().lgt_set_sweep_order(self.h, int(bool(alternate))))

    def set_hop_staging(self, mode):
        """Stage the FP32 hops' operands in shared memory: bit 0 links, bit 1 spinors
        with their neighbour halos; 0 reads them through L1/L2 (lgt_set_hop_staging)."""
        check(lib().lgt_set_hop_staging(self.h, int(mode)))

    def hop_staging_status(self):
        """(staging applies to these extents, staged blocks whose copy wait gave up)."""
        ap, to = C.c_int(), C.c_uint()
        check(lib().lgt_hop_staging_status(self.h, C.byref(ap), C.byref(to)))
        return bool(ap.value), to.value

    def dslash(self, inp, op=OP_D, out_parity=FULL, dagger=False, kappa=0.0, precision=FP64, out=None):
        if out is None:
            if op == OP_D:
                out = self.spinor_field(FULL, precision)
            else:
                out = self.spinor_field(EVEN if op != OP_HOP else out_parity, precision)
        check(lib().lgt_dslash(self.h, _ptr(inp), _ptr(out), op, out_parity, int(dagger), kappa, precision))
        return out

    def cg_solve(self, b, kappa, even_odd, sp=None, x=None):
        sp = sp or solver()
        if x is None:
            x = torch.zeros_like(b)
        st = SolveStats()
        check(lib().lgt_cg_solve(self.h, _ptr(b), _ptr(x), kappa, int(even_odd), C.byref(sp), C.byref(st)))
        return x, st.as_dict()

    def cg_solve_multi(self, bs, kappas, sp=None, xs=None):
        """Solve Dhat_k^+ Dhat_k x_k = b_k (even half fields) for several sources at once."""
        sp = sp or solver()
        n = len(bs)
        if xs is None:
            xs = [torch.zeros_like(b) for b in bs]
        st = (SolveStats * n)()
        check(lib().lgt_cg_solve_multi(self.h, n, (C.c_void_p * n)(*[b.data_ptr() for b in bs]),
                                       (C.c_void_p * n)(*[x.data_ptr() for x in xs]),
                                       (C.c_double * n)(*kappas), C.byref(sp), st))
        return xs, [s.as_dict() for s in st]

    def chrono_reset(self):
        check(lib().lgt_chrono_reset(self.h))

    def hop_multi(self, ins, out_parity, dagger=False, outs=None):
        """out_k = H_{p,1-p} in_k for FP32 half fields, one link load for all of them."""
        n = len(ins)
        if outs is None:
            outs = [self.spinor_field(out_parity, FP32) for _ in ins]
        check(lib().lgt_hop_multi(self.h, n, (C.c_void_p * n)(*[t.data_ptr() for t in ins]),
                                  (C.c_void_p * n)(*[t.data_ptr() for t in outs]), out_parity, int(dagger)))
        return outs

    # ------------------------------------------------------------ actions and forces
    def action(self, ap, phi=None, sp=None):
        sp = sp or solver()
        Sg, Sf, st = C.c_double(), C.c_double(), SolveStats()
        check(lib().lgt_action(self.h, C.byref(ap), _ptr(phi) if phi is not None else None, C.byref(sp),
                               C.byref(Sg), C.byref(Sf), C.byref(st)))
        return Sg.value, Sf.value, st.as_dict()

    def force(self, ap, phi=None, sp=None, form=FORCE_LIE, out=None):
        sp = sp or solver()
        if out is None:
            out = self.momentum_field() if form == FORCE_LIE else self.grad_field()
        st = SolveStats()
        check(lib().lgt_force(self.h, C.byref(ap), _ptr(phi) if phi is not None else None, C.byref(sp),
                              _ptr(out), form, C.byref(st)))
        return out, st.as_dict()

    def kinetic_energy(self, mom):
        v = C.c_double()
        check(lib().lgt_kinetic_energy(self.h, _ptr(mom), C.byref(v)))
        return v.value

    def md_update(self, mom, eps, which, ap=None, phi=None, sp=None):
        sp = sp or solver()
        ap = ap or action_params()
        st = SolveStats()
        check(lib().lgt_md_update(self.h, _ptr(mom), eps, which, C.byref(ap),
                                  _ptr(phi) if phi is not None else None, C.byref(sp), C.byref(st)))
        return st.as_dict()

    def stout_smear(self, rho, n_levels, recompute=False):
        out = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device=self.device)
        check(lib().lgt_stout_smear(self.h, rho, n_levels, int(recompute), _ptr(out)))
        return out

    def stout_backward(self, rho, n_levels, G_top, recompute=False):
        G_top = self._dev(G_top, torch.complex128)
        out = torch.zeros((self.V, 4, 3, 3), dtype=torch.complex128, device=self.device)
        check(lib().lgt_stout_backward(self.h, rho, n_levels, int(recompute), _ptr(G_top), _ptr(out)))
        return out

    def gaussian_momenta(self, seed, traj=0, out=None):
        m = self.momentum_field() if out is None else out
        check(lib().lgt_gaussian_momenta(self.h, _ptr(m), seed, traj))
        return m

    def gaussian_spinor(self, seed, traj=0, field_id=FIELD_SOURCE, parity=FULL):
        f = self.spinor_field(parity, FP64)
        check(lib().lgt_gaussian_spinor(self.h, _ptr(f), seed, traj, field_id, parity))
        return f

    def hmc_trajectory(self, ap, hp, seed, traj):
        r = HMCResult()
        check(lib().lgt_hmc_trajectory(self.h, C.byref(ap), C.byref(hp), seed, traj, C.byref(r)))
        return r.as_dict()
