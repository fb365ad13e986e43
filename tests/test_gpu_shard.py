"""Domain decomposition in time slabs on the GPU: every rank a separate
context of its extended slab (all on the one GPU of the box), ghost faces
filled by device copies into the receiving rank's memory.  Each rank's
sharded D_eo / D_oe is compared with the unsharded oracle on its sites, and
a CG with the sharded operator and rank-ordered sums reaches the oracle's
true residual 1e-10.  The host-side rank logic is covered on CPU ranks by
test_halo_cpu.py."""
import numpy as np
import pytest
import torch

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [((4, 6, 4, 8), 1), ((4, 6, 4, 8), 2), ((4, 6, 4, 8), 4), ((8, 8, 8, 16), 2), ((8, 8, 8, 16), 4),
         ((6, 4, 10, 12), 3)]


def _errs(got, ref):
    d = np.abs(got - ref)
    return float(np.linalg.norm(d) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max())


@pytest.mark.parametrize("dims,world", CASES)
def test_sharded_deo_matches_unsharded_oracle(gpu, orc, dims, world):
    U = inputs.random_links(dims, seed=61)
    with gpu.ShardWorld(dims, world) as W:
        W.links_upload(U)
        for out_parity in (0, 1):
            x = inputs.gaussian_field(dims, k=60 + out_parity)
            xin = W.scatter(x)
            out = [torch.zeros_like(f) for f in xin]
            W.exchange(xin)
            W.deo_apply(out_parity, xin, out)
            torch.cuda.synchronize()
            got = W.gather(out)
            n, m = _errs(got, orc.deo(dims, out_parity, U, x))
            assert n <= 1e-13 and m <= 1e-13, f"world {world} parity {out_parity}: {n:.2e} {m:.2e}"


def test_sharded_deo_equals_unsharded_gpu_bits(gpu):
    """A site's output depends only on its own hops, evaluated in one fixed
    order: two ranks give bitwise the outputs of one rank over the whole
    lattice."""
    dims = (8, 8, 8, 16)
    U = inputs.random_links(dims, seed=62)
    x = inputs.gaussian_field(dims, k=62)
    with gpu.ShardWorld(dims, 2) as W, gpu.ShardWorld(dims, 1) as W1:
        W.links_upload(U)
        W1.links_upload(U)
        for out_parity in (0, 1):
            res = []
            for ww in (W, W1):
                xin = ww.scatter(x)
                out = [torch.zeros_like(f) for f in xin]
                ww.exchange(xin)
                ww.deo_apply(out_parity, xin, out)
                torch.cuda.synchronize()
                res.append(ww.gather(out))
            assert np.array_equal(res[0], res[1])


@pytest.mark.parametrize("dims,world", [((4, 6, 4, 8), 2), ((8, 8, 8, 16), 4), ((6, 4, 10, 12), 3)])
def test_sharded_cg_reaches_oracle_true_residual(gpu, orc, dims, world):
    U = inputs.random_links(dims, seed=63)
    b = inputs.gaussian_field(dims, k=63)
    mass, sigma, tol = 0.1, 0.02, 1e-10
    with gpu.ShardWorld(dims, world) as W:
        W.links_upload(U)
        x, info = W.cg_solve(mass, sigma, tol, b)
    assert info["true_resid"][0] <= tol
    assert orc.true_residual(dims, U, mass, sigma, b, x) <= tol
    ref = orc.cg(dims, U, mass, sigma, b, 1e-12)[0]
    kappa = (mass ** 2 + sigma + 16) / (mass ** 2 + sigma)
    assert np.linalg.norm(x - ref) / np.linalg.norm(ref) <= 2 * kappa * tol


def test_sharded_cg_same_result_for_every_world_size(gpu, orc):
    """The decomposition changes only the grouping of the FP64 sums: every
    world size reaches tol with iteration counts within a few of each other."""
    dims = (8, 8, 8, 16)
    U = inputs.random_links(dims, seed=64)
    b = inputs.gaussian_field(dims, k=64)
    its = []
    for world in (1, 2, 4):
        with gpu.ShardWorld(dims, world) as W:
            W.links_upload(U)
            x, info = W.cg_solve(0.1, 0.0, 1e-10, b)
        assert orc.true_residual(dims, U, 0.1, 0.0, b, x) <= 1e-10
        its.append(info["iters"])
    assert max(its) - min(its) <= 3, its


def test_shard_argument_errors(gpu):
    import ctypes
    lib = gpu.load()
    h = ctypes.c_void_p()
    o = gpu.default_opts()
    for dims, world, rank in [((4, 4, 4, 8), 3, 0), ((4, 4, 4, 6), 2, 0), ((4, 4, 4, 8), 2, 2)]:
        st = lib.lqcd_shard_create((ctypes.c_int * 4)(*dims), world, rank, ctypes.byref(o), ctypes.byref(h))
        assert st == gpu.LQCD_EINVAL
    with gpu.ShardWorld((4, 4, 4, 8), 2) as W:
        # ranks out of order are rejected
        hs = (ctypes.c_void_p * 2)(W.h[1], W.h[0])
        fp = (ctypes.c_void_p * 2)(0, 0)
        assert lib.lqcd_shard_exchange(hs, 2, fp) == gpu.LQCD_EINVAL
        with gpu.Context((4, 4, 4, 8)) as c:
            info = (ctypes.c_long * 6)()
            assert lib.lqcd_shard_geometry(c.h, info) == gpu.LQCD_EINVAL
