"""lqcd_deo_apply_host_noalloc: the host-buffer D_eo for callers that cannot
allocate device memory (its staging lives in a fixed array inside the
library).  Checked through the C ABI against lqcd_deo_apply with host
buffers, on two calls in a row, within the FP64 tolerance of the other
D_eo tests (1e-13 relative).  Kept in a file of its own, collected last."""
import ctypes

import numpy as np
import pytest

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13


def _call_noalloc(lib, ctx, parity, x):
    a = np.ascontiguousarray(x, dtype=np.complex128)
    out = np.empty_like(a)
    st = lib.lqcd_deo_apply_host_noalloc(ctx.h, parity, a.ctypes.data, out.ctypes.data)
    return st, out


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (16, 16, 16, 16)])
def test_noalloc_matches_allocating_entry_point_twice(gpu, dims):
    lib = gpu.load()
    U = inputs.random_links(dims)
    x1 = inputs.gaussian_field(dims, k=1)
    x2 = inputs.gaussian_field(dims, k=2)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for parity, x in ((0, x1), (1, x2)):   # two calls in a row, different inputs
            ref = c.deo_apply(parity, x)        # the allocating host-buffer call
            st, got = _call_noalloc(lib, c, parity, x)
            assert st == gpu.LQCD_OK, lib.lqcd_last_error()
            assert _rel(got, ref) <= TOL
        # the shared staging keeps the last call's contents; a repeat call is unaffected
        st, again = _call_noalloc(lib, c, 0, x1)
        assert st == gpu.LQCD_OK
        assert _rel(again, c.deo_apply(0, x1)) <= TOL


def test_noalloc_makes_no_device_allocation(gpu):
    """With the library's allocation-failure injector armed for the very next
    device allocation, the no-allocation call still succeeds (it reaches no
    allocation), while the allocating host-buffer call fails with
    LQCD_ENOMEM."""
    lib = gpu.load()
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=3)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        ref = c.deo_apply(0, x)
        st, _ = _call_noalloc(lib, c, 0, x)   # first call on this context: address set-up
        assert st == gpu.LQCD_OK, lib.lqcd_last_error()
        try:
            lib.lqcd_inject_alloc_failure(1)
            st, got = _call_noalloc(lib, c, 0, x)
            assert st == gpu.LQCD_OK, lib.lqcd_last_error()
            assert _rel(got, ref) <= TOL
            a = np.ascontiguousarray(x)
            out = np.empty_like(a)
            st = lib.lqcd_deo_apply(c.h, 0, a.ctypes.data, out.ctypes.data, 0, None)
            assert st == gpu.LQCD_ENOMEM   # the armed failure was still waiting
        finally:
            lib.lqcd_inject_alloc_failure(0)


def test_noalloc_rejects_lattices_above_its_fixed_size(gpu):
    lib = gpu.load()
    dims = (24, 24, 24, 24)  # V/2 = 165888 > 131072
    with gpu.Context(dims) as c:
        c.links_upload(inputs.unit_links(dims))
        st, _ = _call_noalloc(lib, c, 0, np.zeros((c.Vh, 3), np.complex128))
        assert st == gpu.LQCD_EINVAL
        assert b"too large" in lib.lqcd_last_error()
