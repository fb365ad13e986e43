"""Bounds-checked build (the stand-in for a memory checker, which this
machine does not offer): liblqcd_checked.so compares every neighbour and
link index a kernel computes with its array extent and records any index
out of range.  A child process loads that library and runs every kernel
family on ragged and smallest lattices:
- D_eo in every precision, staged and per-thread;
- FP64, mixed-precision and packed solves;
- multi-RHS in both layouts;
- gauge MD steps and the action;
- the fermion force;
- stout smearing and its force chain.
No index may be out of range.  Its D_eo and solve results must equal the
default library's bit for bit: the checks only add comparisons.  Both
libraries run the same script in a child process, with the stand-alone
D_eo's launch shape fixed through the tuning-cache file (tuned variants may
sum in different orders)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DIMS = [(2, 2, 2, 2), (4, 6, 8, 10), (6, 4, 2, 4), (12, 12, 12, 12)]
SHIFTS = [1e-3, 0.1, 2.0]

CHILD = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import build, inputs, lqcd
checked = sys.argv[5] == "1"
lib = build.build(checked=checked)
lqcd.load(lib)
dims_list = [tuple(d) for d in eval(sys.argv[3])]
shifts = eval(sys.argv[4])
out, errs = {}, {}

def check(tag):
    errs[tag] = lqcd.bounds_errors() if checked else 0

for dims in dims_list:
    V = int(np.prod(dims))
    U = inputs.random_links(dims, seed=140)
    x = inputs.gaussian_field(dims, k=140)
    for staged in (1, 0):
        with lqcd.Context(dims, staged=staged) as c:
            c.links_upload(U)
            for p in (0, 1):
                out[f"deo{dims}{p}s{staged}"] = c.deo_apply(p, x)
            xs, _ = c.mscg_solve(0.05, shifts, 1e-10, x)
            out[f"mscg{dims}s{staged}"] = xs
    check(f"fp64 {dims}")
    with lqcd.Context(dims) as c:
        c.links_upload(U)
        xd = lqcd.to_device_spinor(x, dtype=torch.complex64)
        od = torch.empty_like(xd)
        for prec, recon in ((1, 18), (1, 12), (2, 12)):
            c.deo_apply_ex(0, prec, recon, xd, od)
        xd64 = lqcd.to_device_spinor(x)
        od64 = torch.empty_like(xd64)
        c.deo_apply_ex(1, 3, 18, xd64, od64)
        for layout, shape in ((0, (3, c.Vh, 4)), (1, (3, 4, c.Vh))):
            b = torch.randn(shape, dtype=torch.complex64, device="cuda")
            c.deo_apply_mrhs(0, 4, 12, b, torch.empty_like(b), layout=layout)
        torch.cuda.synchronize()
        c.set_opts(prec=1, recon=12, fp64_until=1e-3)
        c.mscg_solve(0.05, shifts, 1e-10, x)
        c.set_opts(prec=0, recon=18)
        c.mom_upload(inputs.random_momenta(dims, seed=141))
        for prec in (0, 3, 1):
            c.gauge_md_steps(5.5, 0.01, 1, prec)
            c.gauge_action(5.5, prec)
        c.fermion_force_update(0.3, 0.2, [0.3, 0.8], [0.05, 0.5], 1e-10, x, 0.01)
        c.stout_smear(0.15, 2)
        c.stout_force(inputs.random_momenta(dims, seed=142))
        c.fermion_force_update(0.3, 0.2, [0.3, 0.8], [0.05, 0.5], 1e-10, x, 0.01)
        c.stout_restore()
    check(f"other {dims}")
ctxs = []
for k, dims in enumerate(dims_list[1:3]):
    c = lqcd.Context(dims)
    c.links_upload(inputs.random_links(dims, seed=150 + k))
    ctxs.append(c)
lqcd.mscg_solve_packed(ctxs, [0.05, 0.05], [shifts, shifts], [1e-10, 1e-10],
                       [inputs.gaussian_field(d, k=3) for d in dims_list[1:3]])
for c in ctxs:
    c.close()
check("packed")
np.savez(sys.argv[2], **out)
print(repr(errs))
'''


def _run_child(tmp_path, checked: bool):
    script = tmp_path / "child.py"
    script.write_text(CHILD)
    cache = tmp_path / "tune.txt"
    cache.write_text("".join(f"deo2 v0 {d[0]}x{d[1]}x{d[2]}x{d[3]} 256\n" for d in DIMS))
    npz = tmp_path / f"out{int(checked)}.npz"
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, str(script), ROOT, str(npz), repr(DIMS), repr(SHIFTS), str(int(checked))],
                       capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    return eval(r.stdout.strip().splitlines()[-1]), np.load(npz)


def test_checked_build_finds_no_out_of_range_index(gpu, tmp_path):
    errs, got = _run_child(tmp_path, True)
    assert errs and all(v == 0 for v in errs.values()), f"out-of-range indices recorded: {errs}"
    _, ref = _run_child(tmp_path, False)
    assert sorted(got.files) == sorted(ref.files)
    for k in got.files:
        assert np.array_equal(got[k], ref[k]), k


def test_default_build_reports_no_bounds_words(gpu):
    with pytest.raises(gpu.LqcdError) as e:
        gpu.bounds_errors()
    assert e.value.status == gpu.LQCD_ESTATE
