"""The two forms of the reduction kernels of the solver iteration through
the C ABI: K3 (r -= alpha q and ||r||^2, beta / convergence finaliser) in
every precision, and the FP32 / FP16 K2 (q = A p and <p, q>, alpha / zeta
finaliser).

By default these run as persistent kernels: resident blocks walk the tiles,
and each block takes one ticket per job. With LQCD_PERSIST_REDUCTIONS=0
they run one block per tile, with a ticket per tile. The site arithmetic,
the in-tile reductions and the tile-ordered sum are the same, so the bar is
bitwise equality. It is checked on solutions, iteration counts, reliable
updates and true residuals.

The choice is read once per process, so each form runs in its own child
process. Cases:
- the FP64 solve on a ragged lattice and on 24^4, which has more tiles than
  resident blocks;
- the hybrid FP32-12r solve (double-float phase, FP32 segments with
  reliable updates, and the per-shift refinement, which is a packed launch
  of one job per shift);
- the FP16-link solve and FP32 18-real links;
- packed FP64 and FP32 solves over several lattices."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import inputs, lqcd
out = {}
cases = [("fp64_ragged", (6, 6, 10, 8), dict(), 15),
         ("fp64_24", (24, 24, 24, 24), dict(), 15),
         ("hybrid_ragged", (6, 6, 10, 8), dict(prec=1, recon=12, fp64_until=1e-3), 15),
         ("hybrid_24", (24, 24, 24, 24), dict(prec=1, recon=12, fp64_until=3e-4), 15),
         ("fp16_ragged", (4, 6, 8, 10), dict(prec=2, recon=12, fp64_until=0.0), 8),
         ("fp32_18r", (8, 8, 8, 8), dict(prec=1, recon=18, fp64_until=1e-3), 4)]
for name, dims, opts, ns in cases:
    U = inputs.random_links(dims, seed=71)
    b = inputs.gaussian_field(dims, k=3)
    with lqcd.Context(dims, **opts) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.01, inputs.log_shifts(ns), 1e-10, b)
    out[name] = x
    out[name + "_info"] = np.array([info["iters"], info["refine_iters"], info["reliable_updates"]])
    out[name + "_res"] = np.array(info["true_resid"])
sizes = [(4, 4, 4, 4), (8, 8, 8, 8), (6, 6, 6, 6)]
for tag, opts in [("packed64", dict()), ("packed32", dict(prec=1, recon=12, fp64_until=1e-3))]:
    ctxs, bs = [], []
    for k, d in enumerate(sizes):
        c = lqcd.Context(d, **opts)
        c.links_upload(inputs.random_links(d, seed=80 + k))
        ctxs.append(c)
        bs.append(inputs.gaussian_field(d, k=k))
    xs, infos = lqcd.mscg_solve_packed(ctxs, [0.01, 0.02, 0.05], [inputs.log_shifts(6)] * 3, [1e-10] * 3, bs)
    for k, x in enumerate(xs):
        out[f"{tag}_{k}"] = x
        out[f"{tag}_{k}_res"] = np.array(infos[k]["true_resid"])
    for c in ctxs:
        c.close()
np.savez(sys.argv[2], **out)
'''


def test_persistent_reductions_bitwise_equal_to_one_block_per_tile(gpu, tmp_path):
    script = tmp_path / "persist.py"
    script.write_text(SCRIPT)
    res = []
    for flag in ("1", "0"):
        npz = tmp_path / f"persist_{flag}.npz"
        env = dict(os.environ, LQCD_PERSIST_REDUCTIONS=flag)
        r = subprocess.run([sys.executable, str(script), ROOT, str(npz)], env=env, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(np.load(npz))
    a, b = res
    assert sorted(a.files) == sorted(b.files)
    for k in a.files:
        assert np.array_equal(a[k], b[k]), k
        if k.endswith("_res"):
            assert a[k].max() <= 1e-10, k
