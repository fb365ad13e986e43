"""Stout smearing of the fermion links and the force chained through it
(Sec. 2.1 stout-improved staggered action, Ref. Morningstar:2003gk), on the
GPU through the C ABI, against the FP64 oracle and the derivative identity.

Bars: smeared links and the chained force within 1e-13 / 1e-12 relative of
the oracle (native FP64 on both sides; the exponential and its derivative
come from different series, the staple sums from different orders); the
fermion force of the smeared action within 1e-9 (it rests on solves to the
true residual 1e-12); the derivative identity at 8^4 to 1e-6 (central
difference, h = 1e-4)."""
import numpy as np
import pytest

import pins
from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

RHO, LEVELS, BETA = pins.STOUT_RHO, pins.STOUT_LEVELS, pins.BETA


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("levels", [1, LEVELS, 3])
@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (2, 4, 6, 8)])
def test_smeared_links_match_oracle(gpu, orc, dims, levels):
    U = inputs.random_links(dims, seed=110)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.stout_smear(RHO, levels)
        got = c.links_download()
        c.stout_restore()
        back = c.links_download()
    assert rel(got, orc.stout_smear(dims, U, RHO, levels)) <= 1e-13
    assert np.array_equal(back, U)


@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (6, 4, 2, 4)])
def test_chained_force_matches_oracle(gpu, orc, dims):
    U = inputs.random_links(dims, seed=111)
    Us = orc.stout_smear(dims, U, RHO, LEVELS)
    Fs = orc.gauge_force(dims, Us, BETA)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.stout_smear(RHO, LEVELS)
        got = c.stout_force(Fs)
    ref = orc.stout_force(dims, U, RHO, Fs, LEVELS)
    assert rel(got, ref) <= 1e-12
    assert np.abs(got - np.conj(np.swapaxes(got, -1, -2))).max() <= 1e-13 * np.abs(got).max()


def test_deo_and_fermion_force_use_smeared_links(gpu, orc):
    dims = (4, 4, 4, 6)
    U = inputs.random_links(dims, seed=112)
    phi = inputs.gaussian_field(dims, k=112)
    x = inputs.gaussian_field(dims, k=113)
    Us = orc.stout_smear(dims, U, RHO, LEVELS)
    eps = 0.1
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(np.zeros((4, int(np.prod(dims)), 3, 3), complex))
        c.stout_smear(RHO, LEVELS)
        y = c.deo_apply(0, x)
        S, _ = c.fermion_force_update(pins.FF_MASS, pins.FF_A0, pins.FF_A, pins.FF_SIGMA, 1e-12, phi, eps)
        H = c.mom_download()
    assert rel(y, orc.deo(dims, 0, Us, x)) <= 1e-13
    Fs, So, st = orc.fermion_force(dims, Us, pins.FF_MASS, pins.FF_A0, pins.FF_A, pins.FF_SIGMA, phi, 1e-13)
    assert st == 0
    ref = orc.stout_force(dims, U, RHO, Fs, LEVELS)
    assert abs(S - So) <= 1e-10 * abs(So)
    assert rel(-H / eps, ref) <= 1e-9


def test_state_rules(gpu):
    dims = (2, 2, 2, 4)
    U = inputs.random_links(dims, seed=114)
    with gpu.Context(dims) as c:
        with pytest.raises(gpu.LqcdError):
            c.stout_smear(RHO, 1)                      # no links yet
        c.links_upload(U)
        c.mom_upload(inputs.random_momenta(dims, seed=115))
        for bad in ((-0.1, 1), (RHO, 0), (RHO, 9), (float("nan"), 1)):
            with pytest.raises(gpu.LqcdError):
                c.stout_smear(*bad)
        with pytest.raises(gpu.LqcdError):
            c.stout_force(np.zeros((4, int(np.prod(dims)), 3, 3), complex))   # not smeared
        c.stout_smear(RHO, 2)
        with pytest.raises(gpu.LqcdError):
            c.stout_smear(RHO, 1)                      # already smeared
        with pytest.raises(gpu.LqcdError):
            c.gauge_md_steps(BETA, 0.01, 1)            # MD moves thin links only
        with pytest.raises(gpu.LqcdError):
            c.gauge_link_update(0.01)
        c.gauge_action(BETA)                           # of the smeared links: allowed
        c.stout_restore()
        c.stout_restore()                              # no-op
        assert np.array_equal(c.links_download(), U)
        c.gauge_md_steps(BETA, 0.01, 1)
        Ub = c.links_download()
        c.stout_smear(0.0, 1)                          # rho = 0: the identity
        assert np.array_equal(c.links_download(), Ub)
        c.links_upload(U)                              # a new upload ends the smearing
        c.gauge_md_steps(BETA, 0.01, 1)


def test_smeared_fermion_force_is_derivative_8(gpu):
    """At 8^4 with GPU operations only: the central difference of S_f on the
    smeared links along thin-link directions exp(+-i h X) equals
    sum Tr(X F), F read back from one chained fermion force update
    (H = 0, eps = 1 gives H' = -F)."""
    dims, h, tol = (8, 8, 8, 8), 1e-4, 1e-12
    V = int(np.prod(dims))
    U = inputs.random_links(dims, seed=116)
    X = inputs.random_momenta(dims, seed=117)
    phi = inputs.gaussian_field(dims, k=116)
    args = (pins.FF_MASS, pins.FF_A0, pins.FF_A, pins.FF_SIGMA)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(np.zeros((4, V, 3, 3), complex))
        c.stout_smear(RHO, LEVELS)
        c.fermion_force_update(*args, tol, phi, 1.0)
        F = -c.mom_download()
        S = []
        for sign in (1.0, -1.0):
            c.links_upload(U)
            c.mom_upload(X)
            c.gauge_link_update(sign * h)
            c.stout_smear(RHO, LEVELS)
            _, s, _ = c.rational_apply(*args, tol, phi)
            S.append(s)
    num = (S[0] - S[1]) / (2 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    assert abs(num - ana) <= 1e-6 * abs(ana)
