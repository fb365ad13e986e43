"""Fermion force of the rational pseudofermion action on the GPU (Sec. 2.2:
Eq. rooting with the rational function of Eq. shlineq; Algorithm 2's
fermion force steps), through the C ABI, against the FP64 CPU oracle and the
derivative it must be.

Bars: F_f depends on the shifted solutions, each solved to the FP64 true
residual tol = 1e-12; with m = 0.3 and poles >= 0.05 (condition number
<= ~120) the force agrees with the oracle's to 1e-8 relative.  The
derivative identity and the second-order energy violation of a full
(gauge + fermion) leapfrog hold as for the oracle."""
import numpy as np
import pytest

import pins
from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

M, A0, A, SIG = pins.FF_MASS, pins.FF_A0, pins.FF_A, pins.FF_SIGMA


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


def gpu_force(gpu, dims, U, phi, tol=1e-12):
    """F_f read back from one update with H = 0 and eps = 1 (H' = -F_f)."""
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(np.zeros((4, int(np.prod(dims)), 3, 3), np.complex128))
        S, info = c.fermion_force_update(M, A0, A, SIG, tol, phi, 1.0)
        return -c.mom_download(), S, info


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (4, 6, 8, 10)])
def test_fermion_force_matches_oracle(gpu, orc, dims):
    U = inputs.random_links(dims, seed=97)
    phi = inputs.gaussian_field(dims, k=7)
    F, S, info = gpu_force(gpu, dims, U, phi)
    Fo, So, st = orc.fermion_force(dims, U, M, A0, A, SIG, phi, 1e-12)
    assert st == 0 and max(info["true_resid"][:len(A)]) <= 1e-12
    assert rel(F, Fo) <= 1e-8
    assert abs(S - So) <= 1e-9 * abs(So)
    assert np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max() == 0.0


def test_fermion_force_is_derivative_8(gpu):
    """GPU operations only: central difference of the GPU rational action
    along exp(+-i h X) against sum Tr(X F_f)."""
    dims, h = (8, 8, 8, 8), 1e-4
    U = inputs.random_links(dims, seed=98)
    phi = inputs.gaussian_field(dims, k=8)
    X = inputs.random_momenta(dims, seed=99)
    F, _, _ = gpu_force(gpu, dims, U, phi, tol=1e-13)
    S = []
    with gpu.Context(dims) as c:
        for sign in (1.0, -1.0):
            c.links_upload(U)
            c.mom_upload(X)
            c.gauge_link_update(sign * h)
            S.append(c.rational_apply(M, A0, A, SIG, 1e-13, phi)[1])
    num = (S[0] - S[1]) / (2 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    assert abs(num - ana) <= 1e-6 * abs(ana)


def test_hmc_energy_violation_second_order(gpu):
    """Leapfrog of the whole Hamiltonian K + S_g + S_f (momentum updates with
    the gauge and the fermion force, link updates in between): the energy
    violation falls four times per halving of the step."""
    dims, beta, tau = (4, 4, 4, 4), 5.5, 0.1
    U0 = inputs.random_links(dims, seed=100)
    H0 = inputs.random_momenta(dims, seed=101)
    phi = inputs.gaussian_field(dims, k=9)
    tol = 1e-13

    def energy(c):
        return c.mom_energy() + c.gauge_action(beta) + c.rational_apply(M, A0, A, SIG, tol, phi)[1]

    def kick(c, e):
        c.gauge_mom_update(beta, e)
        c.fermion_force_update(M, A0, A, SIG, tol, phi, e)

    dH = []
    with gpu.Context(dims) as c:
        for n in (4, 8, 16):
            c.links_upload(U0)
            c.mom_upload(H0)
            E0 = energy(c)
            e = tau / n
            kick(c, 0.5 * e)
            for k in range(n):
                c.gauge_link_update(e)
                kick(c, e if k < n - 1 else 0.5 * e)
            dH.append(abs(energy(c) - E0))
    assert 3.5 <= dH[0] / dH[1] <= 4.5 and 3.5 <= dH[1] / dH[2] <= 4.5, dH


def test_fermion_force_edge_cases(gpu):
    dims = (4, 4, 4, 4)
    phi = inputs.gaussian_field(dims)
    with gpu.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        with pytest.raises(gpu.LqcdError):
            c.fermion_force_update(M, A0, A, SIG, 1e-10, phi, 0.1)      # no momenta yet
        H = inputs.random_momenta(dims)
        c.mom_upload(H)
        S, _ = c.fermion_force_update(M, A0, A, SIG, 1e-10, phi, 0.0)   # eps = 0: H unchanged
        assert np.abs(c.mom_download() - H).max() <= 1e-14 and S > 0
        with pytest.raises(gpu.LqcdError):
            c.fermion_force_update(M, A0, [float("nan")], [0.1], 1e-10, phi, 0.1)
        S0, _ = c.fermion_force_update(M, A0, A, SIG, 1e-10, np.zeros_like(phi), 0.1)  # phi = 0: no force
        assert S0 == 0.0 and np.abs(c.mom_download() - H).max() <= 1e-14
