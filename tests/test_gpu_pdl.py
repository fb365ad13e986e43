"""Programmatic dependent launch of the solver iteration (opts.pdl) through
the C ABI.

With pdl = 1 each iteration kernel starts while its predecessor drains and
streams, before it waits, only what that predecessor does not write (links,
and vectors written two or more launches back).  The arithmetic is the same
as with pdl = 0, so the bar is bitwise equality of the solutions, iteration
counts and true residuals over repeated solves.  A prologue that read data
its predecessor still writes would show up as a difference here.  Cases: the
staged FP64 kernels on a ragged lattice and on 24^4 (648 tiles, more than
the resident blocks), the per-thread FP64 kernels, the hybrid solve with its
FP32 phase and reliable updates, and a packed launch over several lattices."""
import numpy as np
import pytest

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solve(gpu, dims, U, b, shifts, reps, **opts):
    out = []
    with gpu.Context(dims, **opts) as c:
        c.links_upload(U)
        for _ in range(reps):
            out.append(c.mscg_solve(0.01, shifts, 1e-10, b))
    return out


@pytest.mark.parametrize("staged", [1, 0])
@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (24, 24, 24, 24)])
def test_fp64_solve_pdl_bitwise(gpu, dims, staged):
    shifts = inputs.log_shifts(15)
    U = inputs.random_links(dims, seed=61)
    b = inputs.gaussian_field(dims, k=6)
    (x0, i0), = _solve(gpu, dims, U, b, shifts, 1, staged=staged, pdl=0)
    for rep, (x1, i1) in enumerate(_solve(gpu, dims, U, b, shifts, 4, staged=staged, pdl=1)):
        assert i1["iters"] == i0["iters"], f"solve {rep}"
        assert i1["true_resid"] == i0["true_resid"], f"solve {rep}"
        assert np.array_equal(x1, x0), f"solve {rep}"
    assert max(i0["true_resid"]) <= 1e-10


def test_hybrid_solve_pdl_bitwise(gpu):
    dims = (8, 8, 8, 12)
    shifts = inputs.log_shifts(8)
    U = inputs.random_links(dims, seed=62)
    b = inputs.gaussian_field(dims, k=7)
    kw = dict(prec=1, recon=12, fp64_until=1e-3)
    (x0, i0), = _solve(gpu, dims, U, b, shifts, 1, pdl=0, **kw)
    for x1, i1 in _solve(gpu, dims, U, b, shifts, 2, pdl=1, **kw):
        assert np.array_equal(x1, x0)
        assert i1["iters"] == i0["iters"] and i1["reliable_updates"] == i0["reliable_updates"]
    assert max(i0["true_resid"]) <= 1e-10


def test_packed_pdl_equals_solo_without(gpu):
    sizes = [(4, 4, 4, 4), (8, 8, 8, 8), (12, 12, 12, 12), (4, 6, 8, 10)]
    shifts = [inputs.log_shifts(15), [1e-3, 0.1], inputs.log_shifts(5, 1e-4, 10.0), [0.01]]
    masses = [0.01, 0.05, 0.02, 0.1]
    ctxs, bs, solo = [], [], []
    for k, d in enumerate(sizes):
        U = inputs.random_links(d, seed=400 + k)
        b = inputs.gaussian_field(d, k=k)
        with gpu.Context(d, pdl=0) as c0:
            c0.links_upload(U)
            x, _ = c0.mscg_solve(masses[k], shifts[k], 1e-10, b)
        c = gpu.Context(d, pdl=1)
        c.links_upload(U)
        ctxs.append(c)
        bs.append(b)
        solo.append(x)
    xs, infos = gpu.mscg_solve_packed(ctxs, masses, shifts, [1e-10] * len(sizes), bs)
    for k, d in enumerate(sizes):
        assert np.array_equal(xs[k], solo[k]), f"lattice {d}"
        assert max(infos[k]["true_resid"]) <= 1e-10
    for c in ctxs:
        c.close()
