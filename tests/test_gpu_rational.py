"""Rational function of A on the GPU (RHMC, Sec. 2.2; Eqs. rooting, shlineq):
y = a0 b + sum_i a_i (A + sigma_i)^{-1} b and the action Re <b, y>, through
the C ABI, against the FP64 CPU oracle and the dense matrix function.

Bar: every pole's FP64 true residual <= tol, and |y - y_ref| within the bound
the method states, tol ||b|| sum_i |a_i| / (lambda_min + sigma_i) with
lambda_min >= m^2 (twice that between two approximate results).  The device
epilogue alone is checked at 24^4 against the same combination done on the
host from the library's own shifted solutions (rounding order only)."""
import numpy as np
import pytest
import torch

import pins
from paper_1701_00426_gb300 import inputs, rational

pytestmark = pytest.mark.gpu

A0, A, SIGMA = pins.RAT_A0, pins.RAT_A, pins.RAT_SIGMA


def bound(tol, b, mass, a=A, sigma=SIGMA):
    return pins.rational_bound(tol, np.linalg.norm(b), a, sigma, mass * mass)


@pytest.mark.parametrize("dims", [(4, 6, 8, 10), (8, 8, 8, 8)])
def test_rational_matches_oracle(gpu, orc, dims):
    mass, tol = 0.05, 1e-10
    U = inputs.random_links(dims, seed=61)
    b = inputs.gaussian_field(dims, k=8)
    yo, so, st = orc.rational_apply(dims, U, mass, A0, A, SIGMA, b, tol)
    assert st == 0
    with gpu.Context(dims) as c:
        c.links_upload(U)
        y, s, info = c.rational_apply(mass, A0, A, SIGMA, tol, b)
    assert max(info["true_resid"][:len(A)]) <= tol
    bd = bound(tol, b, mass)
    assert np.linalg.norm(y - yo) <= 2 * bd
    assert abs(s - so) <= 2 * np.linalg.norm(b) * bd
    assert abs(s - np.vdot(b, y).real) <= 1e-12 * abs(s)


def test_rational_inverse_sqrt_vs_dense_matrix_function(gpu, orc):
    """Quadrature poles of x^(-1/2): y against A^(-1/2) b from eigh of the
    dense A (built column by column from the oracle's operator)."""
    dims, mass, tol = (4, 4, 4, 4), 0.1, 1e-10
    U = inputs.random_links(dims, seed=62)
    b = inputs.gaussian_field(dims, k=9)
    lam, V = np.linalg.eigh(pins.dense_A(orc, dims, U, mass))
    a0, a, sg = rational.inverse_sqrt_poles(20, lam[0], lam[-1])
    with gpu.Context(dims) as c:
        c.links_upload(U)
        y, s, info = c.rational_apply(mass, a0, a, sg, tol, b)
    ystar = V @ (lam ** -0.5 * (V.conj().T @ b.ravel()))
    approx = float(np.max(np.abs(rational.evaluate(a0, a, sg, lam) - lam ** -0.5)))
    bd = approx * np.linalg.norm(b) + pins.rational_bound(tol, np.linalg.norm(b), a, sg, lam[0])
    assert np.linalg.norm(y.ravel() - ystar) <= 1.01 * bd
    assert abs(s - np.vdot(b.ravel(), ystar).real) <= 1.01 * np.linalg.norm(b) * bd


def test_rational_free_field_closed_form(gpu):
    dims, mass, k = (4, 4, 6, 8), 0.1, (1, 3, 2, 5)
    b = pins.plane_wave_even(dims, k, np.array([1.0, 0.5j, -0.25]))
    lam = pins.free_eigenvalue(dims, k, mass)
    r = A0 + sum(ai / (lam + si) for ai, si in zip(A, SIGMA))
    with gpu.Context(dims) as c:
        c.links_upload(inputs.unit_links(dims))
        y, s, _ = c.rational_apply(mass, A0, A, SIGMA, 1e-12, b)
    assert pins.rel(y, r * b) <= 1e-10
    assert abs(s / (r * np.linalg.norm(b) ** 2) - 1.0) <= 1e-10


def test_rational_epilogue_equals_host_combination_24(gpu):
    """24^4, m = 0.01, 15 poles of x^(-1/2) on [m^2, m^2 + 16]: the device
    epilogue against a0 b + sum_i a_i x_i formed on the host from the
    library's multi-shift solutions of the same systems."""
    dims, mass, tol = (24, 24, 24, 24), 0.01, 1e-10
    a0, a, sg = rational.inverse_sqrt_poles(15, mass * mass, mass * mass + 16.0)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=10)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        y, s, info = c.rational_apply(mass, a0, a, sg, tol, b)
        x, xinfo = c.mscg_solve(mass, sg, tol, b)
    assert max(info["true_resid"][:15]) <= tol
    assert info["iters"] == xinfo["iters"]
    yh = a0 * b + np.tensordot(a, x, axes=1)
    assert pins.rel(y, yh) <= 1e-14
    assert abs(s - np.vdot(b, y).real) <= 1e-12 * abs(s)


def test_rational_device_call_equals_host_call(gpu):
    dims, mass, tol = (8, 8, 8, 8), 0.05, 1e-10
    U = inputs.random_links(dims, seed=63)
    b = inputs.gaussian_field(dims, k=11)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        y, s, _ = c.rational_apply(mass, A0, A, SIGMA, tol, b)
        bd = gpu.to_device_spinor(b)
        yd = torch.empty_like(bd)
        s2, _ = c.rational_apply_dev(mass, A0, A, SIGMA, tol, bd, yd)
        y2 = gpu.from_device_spinor(yd)
    assert np.array_equal(y, y2) and s == s2


def test_rational_edge_cases(gpu):
    dims = (4, 4, 4, 4)
    with gpu.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        b = inputs.gaussian_field(dims)
        with pytest.raises(gpu.LqcdError):
            c.rational_apply(0.1, 0.0, [float("nan")], [0.1], 1e-10, b)
        with pytest.raises(gpu.LqcdError):
            c.rational_apply(0.1, float("inf"), [1.0], [0.1], 1e-10, b)
        with pytest.raises((gpu.LqcdError, ValueError)):
            c.rational_apply(0.1, 0.0, [], [], 1e-10, b)
        y, s, _ = c.rational_apply(0.1, 0.7, [1.0, -0.5], [0.1, 1.0], 1e-10, np.zeros_like(b))
        assert not np.any(y) and s == 0.0
        # a0 only (all a_i = 0): y = a0 b exactly
        y, s, _ = c.rational_apply(0.1, 0.7, [0.0], [0.1], 1e-10, b)
        assert np.array_equal(y, 0.7 * b)
