"""Staged FP64 stencil kernels (link stream through shared memory by bulk
asynchronous copies) against the per-thread kernels, through the C ABI.

The staged kernels keep the per-thread kernels' hop order and arithmetic,
so the bar is bitwise equality: the stand-alone D_eo, the FP64 multi-shift
solve, the hybrid mixed-precision solve and the packed multi-lattice solve
give the same bits with opts.staged = 1 and 0.  Lattices cover a ragged last
tile (4x6x8x10: 960 sites per parity, 3.75 tiles), the smallest lattice
(2^4), a non-power-of-two row length (12^4) and more tiles than resident
blocks (24^4: 648 tiles, so every block walks several tiles)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DEO_DIMS = [(4, 6, 8, 10), (2, 2, 2, 2), (12, 12, 12, 12), (24, 24, 24, 24)]
STAGED_CODE = 3 * 1024 + 288   # tuner code of the staged stand-alone kernel
PER_THREAD_CODE = 256          # one thread per site, 256 per block

FORCED = r'''
import sys, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import inputs, lqcd
dims_list = [tuple(d) for d in eval(sys.argv[3])]
out = {}
for dims in dims_list:
    U = inputs.random_links(dims, seed=77)
    with lqcd.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            x = inputs.gaussian_field(dims, k=5 + parity)
            out[f"{dims}{parity}"] = c.deo_apply(parity, x)
np.savez(sys.argv[2], **out)
'''


def _forced_deo(tmp_path, code, tag):
    cache = tmp_path / f"tune_{tag}.txt"
    cache.write_text("".join(f"deo2 v0 {d[0]}x{d[1]}x{d[2]}x{d[3]} {code}\n" for d in DEO_DIMS))
    script = tmp_path / "forced.py"
    script.write_text(FORCED)
    out = tmp_path / f"out_{tag}.npz"
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, str(script), ROOT, str(out), repr([list(d) for d in DEO_DIMS])],
                       env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    return dict(np.load(out))


def test_staged_deo_bitwise_equals_per_thread(gpu, tmp_path):
    a = _forced_deo(tmp_path, STAGED_CODE, "staged")
    b = _forced_deo(tmp_path, PER_THREAD_CODE, "thread")
    assert set(a) == set(b) and len(a) == 2 * len(DEO_DIMS)
    for k in a:
        assert np.array_equal(a[k], b[k]), f"staged and per-thread D_eo differ for {k}"


def test_staged_link_stream_size(gpu):
    """opts.staged = 1 adds the tile-ordered stream: 2 parities x tiles x 8
    hops x 9 x 256 float4 (16 B)."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    with gpu.Context(dims) as c1, gpu.Context(dims, staged=0) as c0:
        c1.links_upload(U)
        c0.links_upload(U)
        ntiles = (c1.Vh + 255) // 256
        extra = c1.device_bytes() - c0.device_bytes()
        assert extra == 2 * ntiles * 8 * 9 * 256 * 16 + 16  # + the 16-byte status word


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (24, 24, 24, 24)])
def test_staged_fp64_solve_bitwise_equals_per_thread(gpu, dims):
    """Three staged solves in a row (the first captures the iteration graph
    and allocates the workspace) against one per-thread solve."""
    shifts = inputs.log_shifts(15)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=2)
    with gpu.Context(dims, staged=0) as c:
        c.links_upload(U)
        x0, i0 = c.mscg_solve(0.01, shifts, 1e-10, b)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for rep in range(3):
            x1, i1 = c.mscg_solve(0.01, shifts, 1e-10, b)
            assert i1["iters"] == i0["iters"], f"solve {rep}"
            assert i1["true_resid"] == i0["true_resid"], f"solve {rep}"
            assert np.array_equal(x1, x0), f"solve {rep}"
    assert max(i0["true_resid"]) <= 1e-10


def test_staged_hybrid_solve_bitwise_equals_per_thread(gpu):
    """FP64 phase (staged or not) then FP32 with reliable updates."""
    dims = (8, 8, 8, 12)
    shifts = inputs.log_shifts(8)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=4)
    res = {}
    for staged in (1, 0):
        with gpu.Context(dims, prec=1, recon=12, fp64_until=1e-3, staged=staged) as c:
            c.links_upload(U)
            res[staged] = c.mscg_solve(0.01, shifts, 1e-10, b)
    (x1, i1), (x0, i0) = res[1], res[0]
    assert np.array_equal(x1, x0)
    assert i1["iters"] == i0["iters"] and i1["reliable_updates"] == i0["reliable_updates"]
    assert max(i1["true_resid"]) <= 1e-10


def test_staged_packed_equals_per_thread_solo(gpu):
    """Packed launch over several lattices (staged, 64-job kernels) against
    each lattice solved alone on the per-thread kernels."""
    sizes = [(4, 4, 4, 4), (8, 8, 8, 8), (12, 12, 12, 12), (4, 6, 8, 10)]
    shifts = [inputs.log_shifts(15), [1e-3, 0.1], inputs.log_shifts(5, 1e-4, 10.0), [0.01]]
    masses = [0.01, 0.05, 0.02, 0.1]
    ctxs, bs, solo = [], [], []
    for k, d in enumerate(sizes):
        U = inputs.random_links(d, seed=300 + k)
        b = inputs.gaussian_field(d, k=k)
        with gpu.Context(d, staged=0) as c0:
            c0.links_upload(U)
            x, _ = c0.mscg_solve(masses[k], shifts[k], 1e-10, b)
        c = gpu.Context(d)
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



def test_bounded_stage_wait_times_out_and_context_survives(gpu, orc):
    """Failure detection without a fault: a staged block waits for a stage
    that nothing fills; the bounded wait gives up after 50 ms, the call
    returns LQCD_ETIMEOUT, and the same context then computes D_eo and a
    solve correctly."""
    import time
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims, seed=120)
    x = inputs.gaussian_field(dims, k=120)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for limit in (0.05, 0.2):
            t0 = time.perf_counter()
            with pytest.raises(gpu.LqcdError) as e:
                c.selftest_stage_wait(limit)
            dt = time.perf_counter() - t0
            assert e.value.status == gpu.LQCD_ETIMEOUT
            assert limit <= dt < limit + 5.0
        with pytest.raises(gpu.LqcdError) as e:
            c.selftest_stage_wait(0.0)
        assert e.value.status == gpu.LQCD_EINVAL
        y = c.deo_apply(0, x)
        ref = orc.deo(dims, 0, U, x)
        assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
        xs, info = c.mscg_solve(0.05, [1e-3, 0.1], 1e-10, x)
        assert max(info["true_resid"][:2]) <= 1e-10
