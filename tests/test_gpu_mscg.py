"""Multi-shift CG on the GPU against the FP64 CPU oracle (through the C ABI).

Bar (stated by the method): for every shift the FP64 true residual
||(A + sigma_i) x_i - b|| / ||b|| is at or below tol, recomputed here by the
oracle from the returned x_i; the difference to the oracle's own solution is
bounded by the conditioning, |x - x_ref| / |x_ref| <= 2 kappa_i tol with
kappa_i = (m^2 + sigma_i + 16) / (m^2 + sigma_i) (||D|| <= 2 with the 1/2
normalisation, so A <= m^2 + 4 ... 16 is a safe bound)."""
import numpy as np
import pytest
import torch

from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu


def kappa(m, s):
    return (m * m + s + 16.0) / (m * m + s)


def check_solution(orc, dims, U, mass, shifts, b, x, tol, xref=None):
    for i, s in enumerate(shifts):
        r = orc.true_residual(dims, U, mass, s, b, x[i])
        assert r <= tol, f"shift {s}: oracle-recomputed true residual {r:.3e} > {tol}"
        if xref is not None:
            e = np.linalg.norm(x[i] - xref[i]) / np.linalg.norm(xref[i])
            assert e <= 2 * kappa(mass, s) * tol, f"shift {s}: error vs oracle {e:.2e}"


def test_config1_single_shift_cg_8444(gpu, orc):
    """Plain FP64 CG on 8^4, m = 0.1, sigma = 0, tol 1e-10."""
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims)
    xref, iref = orc.mscg(dims, U, 0.1, [0.0], b, 1e-10)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.1, [0.0], 1e-10, b)
    assert info["true_resid"][0] <= 1e-10
    assert abs(info["iters"] - iref["iters"]) <= max(5, 0.05 * iref["iters"])
    check_solution(orc, dims, U, 0.1, [0.0], b, x, 1e-10, xref)


@pytest.mark.parametrize("dims", [(8, 8, 8, 8), (4, 6, 8, 10)])
def test_15_shifts_fp64(gpu, orc, dims):
    shifts = inputs.log_shifts(15)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=1)
    xref, _ = orc.mscg(dims, U, 0.01, shifts, b, 1e-10)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.01, shifts, 1e-10, b)
    assert max(info["true_resid"]) <= 1e-10
    check_solution(orc, dims, U, 0.01, shifts, b, x, 1e-10, xref)


def test_maximum_shift_count(gpu, orc):
    """32 shifts, the most one call takes: every lane of the warp that runs
    the per-shift recurrences and convergence tests carries a shift, and the
    active-shift mask uses all 32 bits."""
    dims = (4, 4, 4, 8)
    shifts = inputs.log_shifts(32, 1e-4, 1e2)
    U = inputs.random_links(dims, seed=77)
    b = inputs.gaussian_field(dims, k=3)
    xref, _ = orc.mscg(dims, U, 0.05, shifts, b, 1e-10)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.05, shifts, 1e-10, b)
    assert len(info["shift_iters"]) == 32 and min(info["shift_iters"]) > 0
    # larger shifts converge no later than smaller ones
    assert all(a >= b_ for a, b_ in zip(info["shift_iters"], info["shift_iters"][1:]))
    assert max(info["true_resid"]) <= 1e-10
    check_solution(orc, dims, U, 0.05, shifts, b, x, 1e-10, xref)


def test_timed_workload_32_sampled_shifts(gpu, orc):
    """The configuration bench.py times: 32^4 hot links (seed 1701), m = 0.01,
    the 15 log-spaced shifts, tol 1e-10, staged FP64 kernels, through the
    device call that the bench times.  The oracle recomputes the true
    residual of the smallest, a middle and the largest shift from the
    returned solutions.  The iteration count is within 5 % of the oracle's
    own full-solve count (tests/golden/oracle_counts.json): the double-float
    iteration rounds at about 2^-48, so the worst-conditioned shift (kappa
    ~ 1.5e5) takes a few per cent more iterations than in IEEE FP64."""
    import json
    import os
    dims = (32, 32, 32, 32)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=0)
    shifts = inputs.log_shifts(15)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        bd = gpu.to_device_spinor(b)
        xd = torch.empty((15, 3, c.Vh), dtype=torch.complex128, device="cuda")
        info = c.mscg_solve_dev(0.01, shifts, 1e-10, bd, xd)
        x = gpu.from_device_spinor(xd)
    assert max(info["true_resid"][:15]) <= 1e-10
    orc.set_threads(0)
    for i in (0, 7, 14):
        r = orc.true_residual(dims, U, 0.01, shifts[i], b, x[i])
        assert r <= 1e-10, f"shift {shifts[i]}: oracle-recomputed true residual {r:.3e}"
    golden = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "oracle_counts.json")
    with open(golden) as f:
        counts = json.load(f)["mscg_32x32x32x32_m0.01_15shifts_tol1e-10"]
    assert abs(info["iters"] - counts["iters"]) <= 0.05 * counts["iters"]


@pytest.mark.parametrize("prec,recon,fp64_until", [(1, 12, 3e-4), (2, 12, 0.0)])
def test_timed_workload_32_mixed_precision_sampled_shifts(gpu, orc, prec, recon, fp64_until):
    """The mixed-precision solves bench.py times on the same 32^4 workload:
    FP32 12-real links after an FP64 phase to 3e-4 (the hybrid default), and
    FP16 12-real links, with FP64 reliable updates and per-shift refinement.
    At full size the route differs from the small-lattice tests (tens of
    refinement iterations, several reliable updates), so the oracle
    recomputes the true residual of the smallest, a middle and the largest
    shift from the returned solutions, and every shift's solution is within
    2 kappa_i tol of the FP64 GPU solve of the same system."""
    dims = (32, 32, 32, 32)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=0)
    shifts = inputs.log_shifts(15)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        bd = gpu.to_device_spinor(b)
        x64 = torch.empty((15, 3, c.Vh), dtype=torch.complex128, device="cuda")
        c.mscg_solve_dev(0.01, shifts, 1e-10, bd, x64)
        c.set_opts(prec=prec, recon=recon, fp64_until=fp64_until)
        xd = torch.empty_like(x64)
        info = c.mscg_solve_dev(0.01, shifts, 1e-10, bd, xd)
        x, xr = gpu.from_device_spinor(xd), gpu.from_device_spinor(x64)
    assert max(info["true_resid"][:15]) <= 1e-10
    assert info["reliable_updates"] + info["refine_iters"] > 0
    orc.set_threads(0)
    for i in (0, 7, 14):
        r = orc.true_residual(dims, U, 0.01, shifts[i], b, x[i])
        assert r <= 1e-10, f"shift {shifts[i]}: oracle-recomputed true residual {r:.3e}"
    for i, s in enumerate(shifts):
        kappa = (0.01 ** 2 + s + 16) / (0.01 ** 2 + s)
        assert np.linalg.norm(x[i] - xr[i]) / np.linalg.norm(xr[i]) <= 2 * kappa * 1e-10


@pytest.mark.parametrize("prec,recon,fp64_until",
                         [(1, 18, 1e-4), (1, 12, 1e-4), (1, 12, 1e-2), (1, 18, 0.0), (1, 12, 0.0), (2, 12, 0.0)])
def test_15_shifts_mixed_precision(gpu, orc, prec, recon, fp64_until):
    """FP32 / FP16-link iterations with FP64 reliable updates reach 1e-10,
    with the FP32 phase from the start (fp64_until = 0) or after a
    double-float phase down to fp64_until."""
    dims = (8, 8, 8, 8)
    shifts = inputs.log_shifts(15)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=2)
    xref, iref = orc.mscg(dims, U, 0.01, shifts, b, 1e-10)
    with gpu.Context(dims, prec=prec, recon=recon, fp64_until=fp64_until) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.01, shifts, 1e-10, b)
    assert max(info["true_resid"]) <= 1e-10
    assert info["reliable_updates"] > 0
    # the multi-shift iteration is one Krylov run across the switch
    if prec == 1:
        assert abs(info["iters"] - iref["iters"]) <= 0.1 * iref["iters"] + 10
    check_solution(orc, dims, U, 0.01, shifts, b, x, 1e-10, xref)


def test_hybrid_switch_on_ragged_lattice(gpu, orc):
    """Double-float phase, switch and FP32 phase on a lattice whose half
    volume is not a multiple of the tile (ragged last tile)."""
    dims = (6, 6, 10, 8)
    shifts = [1e-4, 1e-2, 0.3, 5.0]
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=5)
    with gpu.Context(dims, prec=1, recon=12, fp64_until=1e-3) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.02, shifts, 1e-10, b)
    assert max(info["true_resid"]) <= 1e-10
    check_solution(orc, dims, U, 0.02, shifts, b, x, 1e-10)


def test_shift_order_and_duplicates(gpu, orc):
    dims = (4, 4, 6, 8)
    shifts = [1.0, 1e-3, 0.1, 1e-3, 30.0]
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=3)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.05, shifts, 1e-11, b)
    check_solution(orc, dims, U, 0.05, shifts, b, x, 1e-11)
    assert np.array_equal(x[1], x[3])


def test_device_call_equals_host_call_and_is_deterministic(gpu):
    dims = (8, 8, 8, 8)
    shifts = [1e-3, 0.1, 1.0]
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=4)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x1, _ = c.mscg_solve(0.05, shifts, 1e-10, b)
        x2, _ = c.mscg_solve(0.05, shifts, 1e-10, b)
        bd = gpu.to_device_spinor(b)
        xd = torch.empty((3, 3, c.Vh), dtype=torch.complex128, device="cuda")
        c.mscg_solve_dev(0.05, shifts, 1e-10, bd, xd)
        x3 = gpu.from_device_spinor(xd)
    assert np.array_equal(x1, x2)
    assert np.array_equal(x1, x3)


def test_host_call_into_caller_buffer(gpu):
    """out= receives the solution in place; host calls with more and then
    fewer shifts reuse the context's device copies; a wrong buffer is refused."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=5)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        ref, _ = c.mscg_solve(0.05, [1e-3, 0.1, 1.0], 1e-10, b)
        out = np.full((3, c.Vh, 3), np.nan + 0j)
        x, _ = c.mscg_solve(0.05, [1e-3, 0.1, 1.0], 1e-10, b, out=out)
        assert x is out and np.array_equal(out, ref)
        bytes_after = c.device_bytes()
        one, _ = c.mscg_solve(0.05, [0.1], 1e-10, b)
        assert c.device_bytes() == bytes_after
        x, _ = c.mscg_solve(0.05, [1e-3, 0.1, 1.0], 1e-10, b, out=out)
        assert np.array_equal(out, ref)
        for bad in (np.zeros((2, c.Vh, 3), complex), np.zeros((3, c.Vh, 3), np.complex64),
                    np.zeros((3, 3, c.Vh), complex).transpose(0, 2, 1)):
            with pytest.raises(ValueError):
                c.mscg_solve(0.05, [1e-3, 0.1, 1.0], 1e-10, b, out=bad)


def test_free_field_closed_form(gpu):
    import pins
    dims = (4, 4, 6, 8)
    U = inputs.unit_links(dims)
    k = (1, 3, 2, 5)
    b = pins.plane_wave_even(dims, k, np.array([1.0, 0.5j, -0.25]))
    lam = pins.free_eigenvalue(dims, k, 0.1)
    shifts = [0.0, 0.3, 7.0]
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, _ = c.mscg_solve(0.1, shifts, 1e-12, b)
    for i, s in enumerate(shifts):
        assert pins.rel(x[i], b / (lam + s)) < 1e-11


def test_edge_cases(gpu):
    dims = (2, 2, 2, 2)
    U = inputs.random_links(dims)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.1, [0.0, 1.0], 1e-10, np.zeros((8, 3)))
        assert not np.any(x) and info["iters"] == 0
        b = inputs.gaussian_field(dims)
        x, info = c.mscg_solve(0.1, [0.0, 1.0], 1e-12, b)
        assert max(info["true_resid"]) <= 1e-12
        bad = b.copy()
        bad[3, 1] = np.nan
        with pytest.raises(gpu.LqcdError) as e:
            c.mscg_solve(0.1, [0.0], 1e-10, bad)
        assert e.value.status == gpu.LQCD_ENAN
        for args in [(0.1, [], 1e-10), (0.1, [-1.0], 1e-10), (0.1, [0.0], 0.0), (0.0, [0.0], 1e-10),
                     (0.1, list(range(33)), 1e-10)]:
            with pytest.raises(gpu.LqcdError) as e:
                c.mscg_solve(args[0], args[1], args[2], b)
            assert e.value.status == gpu.LQCD_EINVAL


def test_max_iter_reports_noconv(gpu):
    dims = (8, 8, 8, 8)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims)
    with gpu.Context(dims, max_iter=10, check_every=4) as c:
        c.links_upload(U)
        x, info = c.mscg_solve(0.01, [1e-5], 1e-10, b, allow_noconv=True)
    assert info["status"] == gpu.LQCD_ENOCONV
    assert 10 <= info["iters"] <= 12
    assert np.all(np.isfinite(x))
