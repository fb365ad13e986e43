"""D_eo / D_oe on the GPU against the FP64 CPU oracle (through the C ABI).

Bar: FP64 within 1e-13 relative, normwise and element-wise against the
largest reference element; FP32 / FP16 within the bounds their rounding
allows (stated at each test)."""
import numpy as np
import pytest
import torch

import pins
from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13


def errs(got, ref):
    d = np.abs(np.asarray(got) - np.asarray(ref))
    return float(np.linalg.norm(d) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max())


def check_fp64(got, ref, tol=FP64_TOL):
    n, m = errs(got, ref)
    assert n <= tol and m <= tol, f"normwise {n:.2e}, elementwise {m:.2e} > {tol}"
    return n, m


DIMS = [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 8, 10), (6, 6, 6, 6), (8, 8, 8, 8), (10, 4, 6, 12), (16, 16, 16, 16)]


@pytest.mark.parametrize("dims", DIMS)
@pytest.mark.parametrize("parity", [0, 1])
def test_deo_fp64_host_call_matches_oracle(gpu, orc, dims, parity):
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=parity)
    ref = orc.deo(dims, parity, U, x)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        got = c.deo_apply(parity, x)
    check_fp64(got, ref)


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (8, 8, 8, 8)])
def test_deo_native_fp64_matches_oracle(gpu, orc, dims):
    U = inputs.random_links(dims)
    for parity in (0, 1):
        x = inputs.gaussian_field(dims, k=5 + parity)
        ref = orc.deo(dims, parity, U, x)
        with gpu.Context(dims) as c:
            c.links_upload(U)
            xin = gpu.to_device_spinor(x)
            out = torch.empty_like(xin)
            c.deo_apply_ex(parity, gpu.PREC_FP64_NATIVE, 18, xin, out)
            torch.cuda.synchronize()
            n, m = errs(gpu.from_device_spinor(out), ref)
        assert n <= 1e-15 and m <= 1e-15


def test_deo_device_call_equals_host_call(gpu):
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=2)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        h = c.deo_apply(0, x)
        xin = gpu.to_device_spinor(x)
        out = torch.empty_like(xin)
        c.deo_apply_dev(0, xin, out)
        torch.cuda.synchronize()
        assert np.array_equal(gpu.from_device_spinor(out), h)


@pytest.mark.parametrize("scale", [1e-80, 1e-25, 1e30, 1e90])
def test_deo_fp64_extreme_magnitudes(gpu, orc, scale):
    """Inputs outside the double-float exponent window take the native path."""
    dims = (4, 4, 4, 6)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=9) * scale
    ref = orc.deo(dims, 0, U, x)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        got = c.deo_apply(0, x)
    check_fp64(got, ref)


def test_deo_fp64_sparse_and_mixed_scale_input(gpu, orc):
    """Point source (exact zeros) and entries spanning 1e-70 .. 1e40."""
    dims = (4, 4, 6, 8)
    U = inputs.random_links(dims)
    Vh = int(np.prod(dims)) // 2
    x = np.zeros((Vh, 3), np.complex128)
    x[17, 1] = 1.0 + 0.5j
    with gpu.Context(dims) as c:
        c.links_upload(U)
        check_fp64(c.deo_apply(1, x), orc.deo(dims, 1, U, x))
        rng = np.random.default_rng(3)
        y = inputs.gaussian_field(dims, k=1) * 10.0 ** rng.uniform(-70, 40, size=(Vh, 1))
        check_fp64(c.deo_apply(1, y), orc.deo(dims, 1, U, y))


def test_deo_gpu_antihermitian(gpu):
    """Eq. (diracblock) on GPU results alone: <y, D_eo x> = -<D_oe y, x>."""
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=1)
    y = inputs.gaussian_field(dims, k=2)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        Dx = c.deo_apply(0, x)
        Dy = c.deo_apply(1, y)
    lhs, rhs = np.vdot(y, Dx), -np.vdot(Dy, x)
    assert abs(lhs - rhs) / (np.linalg.norm(y) * np.linalg.norm(Dx)) < 1e-14


def test_deo_gpu_free_field_plane_wave(gpu):
    dims = (4, 6, 8, 10)
    U = inputs.unit_links(dims)
    chi = np.array([0.3 + 0.1j, -0.7j, 1.1])
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for k in [(1, 2, 3, 4), (3, 1, 5, 9)]:
            psi = pins.plane_wave_even(dims, k, chi)
            lam = pins.free_eigenvalue(dims, k, 0.1)
            t = c.deo_apply(1, psi)
            A = (0.1 ** 2) * psi - c.deo_apply(0, t)
            assert pins.rel(A, lam * psi) < 1e-13


@pytest.mark.parametrize("prec,recon,tol", [(1, 18, 2e-6), (1, 12, 5e-6), (2, 12, 5e-3)])
def test_deo_low_precision_bounds(gpu, orc, prec, recon, tol):
    """FP32: inputs rounded to 2^-24, 48 products -> ~1e-6 relative.
    FP16 links: rounding 2^-11 plus the rebuilt third row -> ~1e-3."""
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=4)
    ref = orc.deo(dims, 0, U, x)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        xin = gpu.to_device_spinor(x, dtype=torch.complex64)
        out = torch.empty_like(xin)
        c.deo_apply_ex(0, prec, recon, xin, out)
        torch.cuda.synchronize()
        n, m = errs(gpu.from_device_spinor(out), ref)
    assert n <= tol, f"normwise {n:.2e}"


def test_links_roundtrip_and_upload_errors(gpu):
    dims = (4, 4, 4, 4)
    U = inputs.random_links(dims)
    with gpu.Context(dims) as c:
        with pytest.raises(gpu.LqcdError):
            c.deo_apply(0, inputs.gaussian_field(dims))  # no links yet
        c.links_upload(U)
        assert np.array_equal(c.links_download(), U)
        bad = U.copy()
        bad[2, 5, 1, 1] = np.nan
        with pytest.raises(gpu.LqcdError):
            c.links_upload(bad)


@pytest.mark.slow
@pytest.mark.parametrize("dims", [(48, 48, 48, 48), (32, 32, 32, 32), (32, 32, 8, 32), (24, 24, 24, 24)])
def test_deo_fp64_full_size_matches_oracle(gpu, orc, dims):
    """Benchmark sizes (the D_eo sweep runs 16^4 to 48^4), same launch
    configuration as bench.py, every output."""
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=0)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        xin = gpu.to_device_spinor(x)
        out = torch.empty_like(xin)
        c.deo_apply_dev(0, xin, out)
        torch.cuda.synchronize()
        got = gpu.from_device_spinor(out)
    check_fp64(got, orc.deo(dims, 0, U, x))


FORCE_SCRIPT = r'''
import sys, json, numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import inputs, lqcd
from oracle import oracle
orc = oracle()
out = {}
for dims in [(4, 6, 8, 10), (8, 8, 8, 8), (2, 2, 2, 2)]:
    U = inputs.random_links(dims)
    with lqcd.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            x = inputs.gaussian_field(dims, k=3 + parity)
            ref = orc.deo(dims, parity, U, x)
            got = c.deo_apply(parity, x)
            d = np.abs(got - ref)
            out[f"{dims}{parity}"] = [float(np.linalg.norm(d) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max())]
print(json.dumps(out))
'''


@pytest.mark.parametrize("code", [64, 128, 256, 1024 + 128, 1024 + 256, 2048 + 128, 2048 + 256, 4096 + 128,
                                  4096 + 256, 3072 + 288])
def test_every_tuned_fp64_variant_matches_oracle(gpu, tmp_path, code):
    """Each candidate of the autotuner, forced through a tuning-cache file."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    lines = [f"deo2 v0 {d[0]}x{d[1]}x{d[2]}x{d[3]} {code}" for d in [(4, 6, 8, 10), (8, 8, 8, 8), (2, 2, 2, 2)]]
    cache.write_text("\n".join(lines) + "\n")
    script = tmp_path / "force.py"
    script.write_text(FORCE_SCRIPT)
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for k, (n, m) in res.items():
        assert n <= FP64_TOL and m <= FP64_TOL, f"variant {code} case {k}: {n:.2e} {m:.2e}"


def deo12(gpu, c, parity, x):
    """FP64 D_eo with 12-real links (first two rows streamed, third rebuilt)."""
    xin = gpu.to_device_spinor(x)
    out = torch.empty_like(xin)
    c.deo_apply_ex(parity, gpu.PREC_FP64, 12, xin, out)
    torch.cuda.synchronize()
    return gpu.from_device_spinor(out)


@pytest.mark.parametrize("dims", DIMS)
def test_deo_fp64_12real_matches_oracle(gpu, orc, dims):
    """Sec. 2.3 third-row reconstruction in double-float arithmetic: the same
    1e-13 bar as the 18-real operator (the links are SU(3) to rounding)."""
    U = inputs.random_links(dims)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            x = inputs.gaussian_field(dims, k=20 + parity)
            check_fp64(deo12(gpu, c, parity, x), orc.deo(dims, parity, U, x))


@pytest.mark.parametrize("scale", [1e-80, 1e90])
def test_deo_fp64_12real_extreme_magnitudes(gpu, orc, scale):
    dims = (4, 4, 4, 6)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=9) * scale
    with gpu.Context(dims) as c:
        c.links_upload(U)
        check_fp64(deo12(gpu, c, 0, x), orc.deo(dims, 0, U, x))


@pytest.mark.slow
@pytest.mark.parametrize("dims", [(32, 32, 32, 32), (24, 24, 24, 24)])
def test_deo_fp64_12real_full_size_matches_oracle(gpu, orc, dims):
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=0)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        got = deo12(gpu, c, 1, x)
    check_fp64(got, orc.deo(dims, 1, U, x))


FORCE12_SCRIPT = r'''
import sys, json, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import inputs, lqcd
from oracle import oracle
orc = oracle()
out = {}
for dims in [(4, 6, 8, 10), (8, 8, 8, 8), (2, 2, 2, 2)]:
    U = inputs.random_links(dims)
    with lqcd.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            x = inputs.gaussian_field(dims, k=3 + parity)
            ref = orc.deo(dims, parity, U, x)
            xin = lqcd.to_device_spinor(x)
            o = torch.empty_like(xin)
            c.deo_apply_ex(parity, lqcd.PREC_FP64, 12, xin, o)
            torch.cuda.synchronize()
            d = np.abs(lqcd.from_device_spinor(o) - ref)
            out[f"{dims}{parity}"] = [float(np.linalg.norm(d) / np.linalg.norm(ref)), float(d.max() / np.abs(ref).max())]
print(json.dumps(out))
'''


@pytest.mark.parametrize("code", [64, 128, 256, 3072 + 288])
def test_every_tuned_fp64_12real_variant_matches_oracle(gpu, tmp_path, code):
    """Per-thread blocks of 64/128/256 and the staged kernel, forced."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    cache = tmp_path / "tune.txt"
    lines = [f"deo2 v5 {d[0]}x{d[1]}x{d[2]}x{d[3]} {code}" for d in [(4, 6, 8, 10), (8, 8, 8, 8), (2, 2, 2, 2)]]
    cache.write_text("\n".join(lines) + "\n")
    script = tmp_path / "force12.py"
    script.write_text(FORCE12_SCRIPT)
    env = dict(os.environ, LQCD_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, str(script), root], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    for k, (n, m) in res.items():
        assert n <= FP64_TOL and m <= FP64_TOL, f"variant {code} case {k}: {n:.2e} {m:.2e}"


def test_injected_allocation_failure_leaves_context_usable(gpu, orc):
    """Host-side fault injection: a device allocation made to fail inside
    lqcd_links_upload returns LQCD_ENOMEM and leaves the context without
    links (LQCD_ESTATE, no kernel runs); the next upload succeeds and D_eo
    matches the oracle.  Covered for the first upload (link storage) and a
    re-upload (the staging buffer)."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims, seed=130)
    x = inputs.gaussian_field(dims, k=130)
    ref = orc.deo(dims, 0, U, x)
    with gpu.Context(dims) as c:
        try:
            for attempt in range(2):
                gpu.inject_alloc_failure(1)
                with pytest.raises(gpu.LqcdError) as e:
                    c.links_upload(U)
                assert e.value.status == gpu.LQCD_ENOMEM and "injected" in str(e.value)
                with pytest.raises(gpu.LqcdError) as e:
                    c.deo_apply(0, x)
                assert e.value.status == gpu.LQCD_ESTATE
                c.links_upload(U)
                y = c.deo_apply(0, x)
                assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
        finally:
            gpu.inject_alloc_failure(0)


@pytest.mark.gpu
def test_calls_from_a_thread_that_never_set_a_device(gpu, orc):
    """Every call switches to the context's device itself: a context made on
    the main thread is driven from a fresh thread whose current device was
    never set, with the same results."""
    import threading
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    x = inputs.gaussian_field(dims, k=5)
    ref = orc.deo(dims, 0, U, x)
    out = {}
    with gpu.Context(dims) as c:
        c.links_upload(U)

        def work():
            try:
                out["deo"] = c.deo_apply(0, x)
                out["noalloc"] = c.deo_apply_host_noalloc(0, x)
            except Exception as exc:  # reported on the main thread
                out["error"] = exc

        t = threading.Thread(target=work)
        t.start()
        t.join()
    assert "error" not in out, out.get("error")
    for k in ("deo", "noalloc"):
        assert np.linalg.norm(out[k] - ref) / np.linalg.norm(ref) <= 1e-13


LOWP_SCRIPT = r'''
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1701_00426_gb300 import inputs, lqcd
out = {}
for dims in [(4, 6, 8, 10), (8, 8, 8, 8)]:
    U = inputs.random_links(dims)
    with lqcd.Context(dims) as c:
        c.links_upload(U)
        x = lqcd.to_device_spinor(inputs.gaussian_field(dims, k=7), dtype=torch.complex64)
        for prec, recon in ((1, 18), (1, 12), (2, 12)):
            o = torch.empty_like(x)
            c.deo_apply_ex(1, prec, recon, x, o)
            torch.cuda.synchronize()
            out[f"{dims}{prec}{recon}"] = o.cpu().numpy()
np.savez(sys.argv[2], **out)
'''


def test_unrolled_low_precision_variants_are_bitwise_equal(gpu, tmp_path):
    """The FP32 / FP16 kernels with the direction loop unrolled (tuner kind 5)
    give the bits of the rolled kernels: same FMAs in the same order."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    script = tmp_path / "lowp.py"
    script.write_text(LOWP_SCRIPT)
    res = []
    for code in (256, 5120 + 128):
        cache = tmp_path / f"tune{code}.txt"
        cache.write_text("".join(f"deo2 v{v} {d[0]}x{d[1]}x{d[2]}x{d[3]} {code}\n"
                                 for v in (2, 3, 4) for d in [(4, 6, 8, 10), (8, 8, 8, 8)]))
        npz = tmp_path / f"o{code}.npz"
        r = subprocess.run([sys.executable, str(script), root, str(npz)], capture_output=True, text=True,
                           timeout=300, env=dict(os.environ, LQCD_TUNE_CACHE=str(cache)))
        assert r.returncode == 0, r.stderr[-2000:]
        res.append(np.load(npz))
    assert sorted(res[0].files) == sorted(res[1].files)
    for k in res[0].files:
        assert np.array_equal(res[0][k], res[1][k]), k


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (8, 8, 8, 8), (10, 4, 6, 12)])
def test_deo_fp16_spinors_with_site_norm(gpu, orc, dims):
    """FP16 links and FP16 spinors with a per-site FP32 norm: against the
    oracle within a few 2^-11 (links, inputs and outputs each rounded to
    FP16), and the output halves lie in [-1, 1] with the site's largest
    component at +-1."""
    U = inputs.random_links(dims)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        for parity in (0, 1):
            x = inputs.gaussian_field(dims, k=30 + parity)
            h, n = gpu.to_device_h16(x)
            ho, no = torch.empty_like(h), torch.empty_like(n)
            c.deo_apply_h16(parity, h, n, ho, no)
            torch.cuda.synchronize()
            got = gpu.from_device_h16(ho, no)
            ref = orc.deo(dims, parity, U, x)
            nrm, _ = errs(got, ref)
            assert nrm <= 3e-3, f"normwise {nrm:.2e}"
            hv = ho.float().abs().amax(dim=(0, 2)).cpu().numpy()
            assert np.all(hv <= 1.0) and np.allclose(hv[no.cpu().numpy() > 0], 1.0)


def test_deo_fp16_spinors_zero_site(gpu):
    """A zero input gives zero output with norm 0 (no division by zero)."""
    dims = (4, 4, 4, 4)
    with gpu.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        x = np.zeros((c.Vh, 3), np.complex128)
        h, n = gpu.to_device_h16(x)
        ho, no = torch.empty_like(h), torch.empty_like(n)
        c.deo_apply_h16(0, h, n, ho, no)
        torch.cuda.synchronize()
        assert not torch.any(no) and not torch.any(ho.float())
