"""The CPU oracle against what the paper and the mathematics fix (no GPU)."""
import numpy as np
import pytest

import pins
from paper_1701_00426_gb300 import inputs


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 8, 10)])
def test_geometry_matches_bruteforce_rank(orc, dims):
    ok, msg = pins.pin_geometry(orc, dims)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 6, 8, 10)])
def test_phases_anticommute_and_time_is_antiperiodic(orc, dims):
    ok, msg = pins.pin_phase_anticommutation(orc, dims)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (4, 6, 8, 10)])
def test_deo_antihermitian(orc, dims):
    """Eq. (diracblock): D_oe^dag = -D_eo."""
    ok, msg = pins.pin_antihermitian(orc, dims)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 6)])
def test_deo_gauge_covariant(orc, dims):
    ok, msg = pins.pin_gauge_covariance(orc, dims)
    assert ok, msg


def test_free_plane_waves_are_eigenvectors(orc):
    ks = [(0, 0, 0, 0), (1, 2, 3, 4), (3, 1, 5, 9), (2, 5, 7, 2), (1, 0, 0, 0), (0, 0, 0, 3)]
    ok, msg = pins.pin_free_plane_waves(orc, (4, 6, 8, 10), ks)
    assert ok, msg


def test_free_two_site_lattice(orc):
    ok, msg = pins.pin_two_site(orc)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4), (2, 4, 2, 6)])
def test_free_spectrum_closed_form(orc, dims):
    ok, msg = pins.pin_free_spectrum(orc, dims)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_A_hermitian_positive(orc, dims):
    """Eq. (lineqeo): m^2 - D_eo D_oe is Hermitian with spectrum >= m^2."""
    ok, msg = pins.pin_hermitian_positive(orc, dims)
    assert ok, msg


def test_mscg_matches_lapack_2444(orc):
    ok, msg = pins.pin_mscg_vs_lapack(orc, (2, 2, 2, 2), [0.0, 1e-3, 1.0])
    assert ok, msg


def test_mscg_matches_lapack_4444(orc):
    ok, msg = pins.pin_mscg_vs_lapack(orc, (4, 4, 4, 4), [1e-5, 1e-3, 0.05, 1.0, 30.0])
    assert ok, msg


def test_mscg_free_field_closed_form(orc):
    ok, msg = pins.pin_free_solve(orc, (4, 4, 6, 8), [0.0, 0.3, 7.0], (1, 3, 2, 5))
    assert ok, msg


def test_single_shift_mscg_is_plain_cg(orc):
    """With one shift the recurrences collapse to CG (zeta = 1 exactly)."""
    dims = (4, 4, 4, 4)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims)
    x1, info = orc.mscg(dims, U, 0.1, [0.02], b, 1e-10)
    x2, it = orc.cg(dims, U, 0.1, 0.02, b, 1e-10)
    assert info["iters"] == it
    assert np.array_equal(x1[0], x2)


def test_mscg_equals_independent_cgs(orc):
    dims = (4, 4, 4, 6)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=1)
    shifts = inputs.log_shifts(6, 1e-4, 10.0)
    tol = 1e-10
    x, info = orc.mscg(dims, U, 0.05, shifts, b, tol)
    assert info["status"] == 0
    for i, s in enumerate(shifts):
        xc, it = orc.cg(dims, U, 0.05, s, b, tol)
        assert it > 0
        kappa = (0.05 ** 2 + s + 16) / (0.05 ** 2 + s)
        assert pins.rel(x[i], xc) <= 2 * kappa * tol
        assert info["true_resid"][i] <= tol


def test_mscg_shift_order_irrelevant(orc):
    """Shifts may come in any order; each x_i belongs to shifts[i]."""
    dims = (4, 4, 4, 4)
    U = inputs.random_links(dims)
    b = inputs.gaussian_field(dims, k=2)
    sh = [1.0, 1e-3, 0.1]
    x, info = orc.mscg(dims, U, 0.1, sh, b, 1e-11)
    for i, s in enumerate(sh):
        assert orc.true_residual(dims, U, 0.1, s, b, x[i]) <= 1e-11


def test_zero_source_gives_zero(orc):
    dims = (2, 2, 2, 4)
    U = inputs.random_links(dims)
    b = np.zeros((16, 3), np.complex128)
    x, info = orc.mscg(dims, U, 0.1, [0.0, 1.0], b, 1e-10)
    assert info["iters"] == 0 and not np.any(x)


def test_oracle_rejects_bad_shift_count(orc):
    dims = (2, 2, 2, 2)
    U = inputs.unit_links(dims)
    b = np.ones((8, 3), np.complex128)
    _, info = orc.mscg(dims, U, 0.1, np.linspace(0, 1, 65), b, 1e-8)
    assert info["status"] == -2


def test_inputs_are_su3_and_seeded():
    dims = (4, 4, 4, 4)
    U = inputs.random_links(dims)
    U2 = inputs.random_links(dims)
    assert np.array_equal(U, U2)
    m = U.reshape(-1, 3, 3)
    eye = np.einsum("nij,nkj->nik", m, m.conj())
    assert np.max(np.abs(eye - np.eye(3))) < 1e-14
    assert np.max(np.abs(np.linalg.det(m) - 1)) < 1e-14
    b = inputs.gaussian_field(dims, k=0)
    assert b.shape == (128, 3) and abs(np.mean(np.abs(b) ** 2) - 2.0) < 0.3


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_rational_apply_matches_dense_eigendecomposition(orc, dims):
    """RHMC rational function (Sec. 2.2): r(A) b and b^dag r(A) b vs LAPACK."""
    ok, msg = pins.pin_rational_vs_dense(orc, dims)
    assert ok, msg


def test_rational_inverse_sqrt_matches_matrix_function(orc):
    """Quadrature poles of x^(-1/2): r(A) b vs A^(-1/2) b from eigh."""
    ok, msg = pins.pin_rational_inverse_sqrt(orc, (4, 4, 4, 4))
    assert ok, msg


def test_rational_free_field_closed_form(orc):
    ok, msg = pins.pin_rational_free(orc)
    assert ok, msg


def test_inverse_sqrt_poles_converge():
    """The quadrature rule is exact at x = s^2 and its error falls with the
    number of poles on a fixed interval."""
    from paper_1701_00426_gb300 import rational
    errs = [rational.max_rel_error(*rational.inverse_sqrt_poles(n, 0.01, 4.01), 0.01, 4.01) for n in (8, 16, 24)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-10
    a0, a, s = rational.inverse_sqrt_poles(5, 0.01, 4.01)
    x = (0.01 * 4.01) ** 0.5
    assert abs(rational.evaluate(a0, a, s, [x])[0] * x ** 0.5 - 1.0) < 1e-14
    assert np.all(np.asarray(a) > 0) and np.all(np.diff(s) > 0)


def test_gauge_action_of_unit_links(orc):
    """Tree-level Symanzik action (Sec. 2.1): S(U = 1) = -9 beta V."""
    ok, msg = pins.pin_gauge_action_unit(orc)
    assert ok, msg


def test_gauge_action_invariant_and_force_covariant(orc):
    ok, msg = pins.pin_gauge_invariance(orc)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_gauge_force_is_derivative_of_action(orc, dims):
    """The force from the staple sums (Listing lst:rect_staples) against a
    central difference of the action enumerated loop by loop."""
    ok, msg = pins.pin_force_is_derivative(orc, dims)
    assert ok, msg


def test_su3_exponential(orc):
    ok, msg = pins.pin_exp(orc)
    assert ok, msg


def test_md_leapfrog_reversible(orc):
    ok, msg = pins.pin_md_reversible(orc)
    assert ok, msg


def test_md_energy_violation_second_order(orc):
    ok, msg = pins.pin_md_energy(orc)
    assert ok, msg


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 6)])
def test_fermion_force_is_derivative_of_rational_action(orc, dims):
    """Force of phi^dag r(A) phi (Sec. 2.2) against a central difference of
    the oracle's rational application along random algebra directions."""
    ok, msg = pins.pin_fermion_force_is_derivative(orc, dims)
    assert ok, msg


def test_fermion_force_gauge_covariant(orc):
    ok, msg = pins.pin_fermion_force_covariant(orc)
    assert ok, msg


def test_stout_identity_unitarity_covariance(orc):
    ok, msg = pins.pin_stout_basic(orc)
    assert ok, msg


def test_stout_smearing_lowers_wilson_action(orc):
    ok, msg = pins.pin_stout_smooths(orc)
    assert ok, msg


@pytest.mark.parametrize("dims", [(4, 4, 4, 4), (2, 4, 2, 4)])
def test_stout_force_chain_is_derivative(orc, dims):
    ok, msg = pins.pin_stout_force_is_derivative(orc, dims=dims)
    assert ok, msg


def test_stout_fermion_force_is_derivative(orc):
    ok, msg = pins.pin_stout_fermion_force(orc)
    assert ok, msg


@pytest.mark.parametrize("dims", [(4, 4, 2, 6), (2, 2, 2, 2)])
def test_oracle_A_equals_numpy_assembly(orc, dims):
    ok, msg = pins.pin_A_numpy_assembly(orc, dims)
    assert ok, msg


@pytest.mark.parametrize("dims", [(2, 2, 2, 2), (4, 4, 4, 4)])
def test_true_residual_against_numpy_assembled_A(orc, dims):
    """The checker behind every solve test: perturbed solutions, so the
    residual is of order 1e-3, at shifts 0, 0.37 and 25."""
    ok, msg = pins.pin_true_residual(orc, dims)
    assert ok, msg


def test_stout_single_nontrivial_link_by_hand(orc):
    ok, msg = pins.pin_stout_single_link(orc)
    assert ok, msg
