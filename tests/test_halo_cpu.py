"""t-slab decomposition of the even/odd lattice (host logic in
paper_1701_00426_gb300/halo.py) against the unsharded oracle.

* Index pins (no ranks): a slab of t-slices is one contiguous half-index
  range for either parity; in the extended slab a site keeps its global
  parity and its half index shifts by a constant; the antiperiodic t-links
  land in the slices `boundary_slices` names.
* World-size-2 and -4 gloo ranks: each rank holds its slab of the field, exchanges
  one face each way, applies D_eo / D_oe on its extended slab (the oracle
  stands in for the per-rank operator, with the global antiperiodic sign
  applied to the links that carry it) and reproduces the unsharded oracle's
  D_eo / D_oe on its sites bit for bit.  A CG on A = m^2 - D_eo D_oe with
  the sharded operator and rank-ordered sums reaches the oracle's solution."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1701_00426_gb300 import halo, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = (4, 6, 4, 8)


def test_slab_is_a_contiguous_half_range(orc):
    S = halo.slice_sites(DIMS)
    for ta, tb in ((0, 8), (2, 6), (4, 8), (3, 4)):
        lo, hi = halo.half_range(DIMS, ta, tb)
        for p in (0, 1):
            got = sorted(orc.idxh(DIMS, (x0, x1, x2, x3))
                         for x3 in range(ta, tb) for x2 in range(DIMS[2]) for x1 in range(DIMS[1])
                         for x0 in range(DIMS[0]) if orc.parity((x0, x1, x2, x3)) == p)
            assert got == list(range(lo, hi)) and hi - lo == (tb - ta) * S // 2


@pytest.mark.parametrize("world", [1, 2, 4])
def test_extended_slab_keeps_parity_and_order(orc, world):
    ext = halo.ext_dims(DIMS, world)
    h = halo.slice_sites(DIMS) // 2
    for rank in range(world):
        t0, nt = halo.slab(DIMS, world, rank)
        for k in range(ext[3]):
            tg = (t0 - halo.GHOST + k) % DIMS[3]
            for x in ((1, 2, 3, k), (0, 5, 1, k), (3, 0, 2, k)):
                xg = (x[0], x[1], x[2], tg)
                assert orc.parity(x) == orc.parity(xg)
                assert orc.idxh(ext, x) - k * h == orc.idxh(DIMS, xg) - tg * h


def test_boundary_slices():
    assert halo.boundary_slices(DIMS, 2, 0) == [1]      # lower ghost = global t = 7
    assert halo.boundary_slices(DIMS, 2, 1) == [5]      # top owned slice = global t = 7
    assert halo.boundary_slices(DIMS, 1, 0) == [1, 9]   # both: the wrapped ghost and the owned top
    with pytest.raises(ValueError):
        halo.slab(DIMS, 3, 0)                           # 8 not divisible by 3
    with pytest.raises(ValueError):
        halo.slab((4, 4, 4, 6), 2, 0)                   # odd slab extent


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def sharded_deo(orc, U_ext, out_parity, x_local, dims, world, rank):
    lower, upper = halo.exchange(x_local, dims, world, rank)
    x_ext = halo.extend(x_local, lower, upper, dims, world)
    return halo.interior(orc.deo(halo.ext_dims(dims, world), out_parity, U_ext, x_ext), dims, world)


def signed_ext_links(U, dims, world, rank):
    U_ext = halo.extended_links(U, dims, world, rank)
    S = halo.slice_sites(dims)
    for k in halo.boundary_slices(dims, world, rank):
        U_ext[3, k * S:(k + 1) * S] *= -1.0
    return U_ext


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle
    orc = oracle()
    U = inputs.random_links(DIMS, seed=55)
    U_ext = signed_ext_links(U, DIMS, world, rank)
    res = {}
    for out_parity in (0, 1):
        x = inputs.gaussian_field(DIMS, k=30 + out_parity)
        ref = halo.local_part(orc.deo(DIMS, out_parity, U, x), DIMS, world, rank)
        got = sharded_deo(orc, U_ext, out_parity, halo.local_part(x, DIMS, world, rank), DIMS, world, rank)
        res[f"deo{out_parity}"] = bool(np.array_equal(got, ref))
    # CG on A = m^2 - D_eo D_oe with the sharded operator (two exchanges and
    # two rank-ordered sums per iteration)
    m2 = 0.1 ** 2
    b = halo.local_part(inputs.gaussian_field(DIMS, k=40), DIMS, world, rank).copy()

    def A(v):
        t = sharded_deo(orc, U_ext, 1, v, DIMS, world, rank)
        return m2 * v - sharded_deo(orc, U_ext, 0, t, DIMS, world, rank)

    def dot(u, v):
        return halo.ordered_sum(float(np.vdot(u, v).real), world)

    x = np.zeros_like(b)
    r, p = b.copy(), b.copy()
    rr, bb = dot(r, r), dot(b, b)
    it = 0
    while rr > 1e-24 * bb and it < 500:
        qv = A(p)
        alpha = rr / dot(p, qv)
        x += alpha * p
        r -= alpha * qv
        rr_new = dot(r, r)
        p = r + (rr_new / rr) * p
        rr, it = rr_new, it + 1
    res["cg_iters"] = it
    q.put((rank, res, x))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_sharded_deo_and_cg_ranks(orc, world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, res, _ in out:
        assert res["deo0"] and res["deo1"], f"rank {rank}: sharded D differs from the unsharded oracle"
    assert len({o[1]["cg_iters"] for o in out}) == 1 and out[0][1]["cg_iters"] < 500
    x = np.concatenate([o[2] for o in out])
    U = inputs.random_links(DIMS, seed=55)
    b = inputs.gaussian_field(DIMS, k=40)
    assert orc.true_residual(DIMS, U, 0.1, 0.0, b, x) <= 1e-10
