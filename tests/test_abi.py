"""The C-ABI library loads without a GPU and exports every symbol include/lgt.h declares;
host-side argument checks fail loudly with a status code."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lgt.h")


def declared_functions(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lgt_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def liblgt():
    from paper_2602_20516_b300 import build, lgt
    if not os.path.exists(lgt.LIB_PATH):
        build.build()
    return lgt.lib()


def test_every_declared_symbol_is_exported(liblgt):
    names = declared_functions()
    assert len(names) >= 29
    for n in names:
        assert hasattr(liblgt, n), n


def test_binding_covers_header():
    from paper_2602_20516_b300 import lgt
    bound = {n for n, _, _ in lgt.SIGNATURES}
    assert bound == set(declared_functions())


def test_version_and_error_strings(liblgt):
    assert liblgt.lgt_version() == 100
    assert isinstance(liblgt.lgt_last_error(), bytes)


def test_invalid_arguments_rejected_on_host(liblgt):
    from paper_2602_20516_b300 import lgt
    h = C.c_void_p()
    # odd extent -> LGT_EINVAL before any device work
    rc = liblgt.lgt_create_lattice((C.c_int * 4)(4, 4, 3, 4), None, None, C.byref(h))
    assert rc == 1 and b"even" in liblgt.lgt_last_error()
    assert liblgt.lgt_create_lattice(None, None, None, C.byref(h)) == 1
    assert liblgt.lgt_destroy_lattice(None) == 0
    assert liblgt.lgt_dslash(None, None, None, 0, 0, 0, 0.1, 0) == 1
    assert liblgt.lgt_cg_solve(None, None, None, 0.1, 1, None, None) == 1
    st = lgt.SolveStats()
    assert liblgt.lgt_force(None, None, None, None, None, 0, C.byref(st)) == 1
    assert liblgt.lgt_cg_solve_multi(None, 2, None, None, None, None, None) == 1
    assert liblgt.lgt_hop_multi(None, 2, None, None, 0, 0) == 1
    assert liblgt.lgt_set_hop_staging(None, 1) == 1
    ap, to = C.c_int(), C.c_uint()
    assert liblgt.lgt_hop_staging_status(None, C.byref(ap), C.byref(to)) == 1


def test_noalloc_volume_limit_checked_without_overflow(liblgt):
    """Extents whose product exceeds 2^63 are rejected by the volume limit on the host
    (the check runs after every factor, before any device call)."""
    buf = (C.c_double * 4)()
    big = (C.c_int * 4)(1 << 30, 1 << 30, 1 << 30, 1 << 30)
    assert liblgt.lgt_plaquette_noalloc(buf, big, buf, None) == 1
    assert b"limit" in liblgt.lgt_last_error()
    # a product that wraps to a small value modulo 2^64 (2^62 * 2^2 = 2^64 -> 0)
    wrap = (C.c_int * 4)(1 << 30, 1 << 30, 1 << 2, 1 << 2)
    assert liblgt.lgt_plaquette_noalloc(buf, wrap, buf, None) == 1
    assert b"limit" in liblgt.lgt_last_error()
