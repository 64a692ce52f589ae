"""lgt_plaquette_noalloc: the allocation-free plaquette entry point.

It exists for callers that cannot allocate device memory when they need the
result (code inside another framework's memory pool or budget, allocator-free
runtimes, hooks between someone else's launches).  Its scratch is a fixed device
array inside the library.  This test calls it through the C ABI and checks it
against the handle-based lgt_plaquette on two calls in a row, and that an
oversized volume is refused on the host.  The file is named so that pytest
collects it last.
"""
import ctypes as C

import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(lgt, U_dev, dims, out_dev):
    d = (C.c_int * 4)(*dims)
    stream = torch.cuda.current_stream()
    rc = lgt.lib().lgt_plaquette_noalloc(C.c_void_p(U_dev.data_ptr()), d, C.c_void_p(out_dev.data_ptr()),
                                         C.c_void_p(stream.cuda_stream))
    return rc


def test_noalloc_plaquette_matches_handle_path_twice():
    from paper_2602_20516_b300 import lgt
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for dims, seed, alpha in (((8, 6, 4, 10), 31, 0.5), ((16, 16, 16, 32), 32, 0.3)):
        lat = lgt.Lattice(dims)
        lat.random_links(seed, alpha)
        ref = lat.plaquette()                 # existing entry point (handle, workspace)
        U = lat.get_links()                   # canonical complex128 on the device
        for _ in range(2):                    # two calls in a row share the scratch array
            out.zero_()
            assert _noalloc(lgt, U, dims, out) == 0, lgt.lib().lgt_last_error()
            torch.cuda.synchronize()
            assert abs(out.item() - ref) <= 1e-13 * abs(ref)
        lat.close()


def test_noalloc_rejects_volume_over_limit():
    from paper_2602_20516_b300 import lgt
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    small = torch.zeros((16, 4, 3, 3), dtype=torch.complex128, device="cuda")
    # 64^4 sites exceed the 8,388,608-site limit: refused before any device work
    assert _noalloc(lgt, small, (64, 64, 64, 64), out) == 1
    assert b"8388608" in lgt.lib().lgt_last_error()
    assert _noalloc(lgt, small, (4, 4, 3, 4), out) == 1
