"""Gauge part of the molecular dynamics step on the GPU (Sec. 2.1 tree-level
Symanzik action, Sec. 4.2 / Algorithm 2 gauge cycle, Listing lst:rect_staples
staples), through the C ABI, against the FP64 CPU oracle and the invariants
the mathematics fixes.

Precisions: FP64 (double-float arithmetic on the FP32 pipes, FP64 storage),
native FP64 (DFMA) and FP32.  Bars: FP64 action, momentum and link updates
within 1e-13 (native) and 1e-12 (double-float: 48-bit products) relative of
the oracle (sums of ~70 SU(3) products in a different order);
FP32 within 5e-6 for the action and the force and 2e-6 for the links
(unit roundoff 6e-8 times the products and sums of a staple; measured
<= 3.2e-7).  Reversibility and second-order energy violation as for the
oracle; the derivative identity at 16^4 with GPU operations only."""
import numpy as np
import pytest

import pins
from paper_1701_00426_gb300 import inputs

pytestmark = pytest.mark.gpu

BETA = pins.BETA
FP64, FP32, NAT = 0, 1, 3   # double-float, FP32, native FP64
TOL = {FP64: 1e-12, NAT: 1e-13, FP32: 5e-6}
PRECS = [FP64, NAT, FP32]


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (2, 4, 6, 8)])
def test_action_matches_oracle(gpu, orc, dims, prec):
    U = inputs.random_links(dims, seed=81)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        S = c.gauge_action(BETA, prec)
        c.links_upload(inputs.unit_links(dims))
        S1 = c.gauge_action(BETA, prec)
    So = orc.gauge_action(dims, U, BETA)
    assert abs(S - So) <= TOL[prec] * abs(So)
    V = int(np.prod(dims))
    assert abs(S1 + 9 * BETA * V) <= 1e-12 * 9 * BETA * V


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("dims", [(4, 4, 4, 6), (2, 2, 2, 2), (6, 4, 2, 4)])
def test_mom_update_matches_oracle(gpu, orc, dims, prec):
    U = inputs.random_links(dims, seed=82)
    H = inputs.random_momenta(dims, seed=83)
    eps = 0.03
    ref = orc.mom_update(dims, U, H, BETA, eps)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(H)
        c.gauge_mom_update(BETA, eps, prec)
        got = c.mom_download()
    # compare the change eps F: relative to its own size
    assert rel(got - H, ref - H) <= TOL[prec]
    assert np.abs(got - np.conj(np.swapaxes(got, -1, -2))).max() == 0.0


@pytest.mark.parametrize("prec", PRECS)
def test_link_update_matches_oracle(gpu, orc, prec):
    dims = (4, 4, 4, 6)
    U = inputs.random_links(dims, seed=84)
    H = inputs.random_momenta(dims, seed=85)
    ref = orc.link_update(dims, U, H, 0.07)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(H)
        c.gauge_link_update(0.07, prec)
        got = c.links_download()
    assert rel(got, ref) <= (2e-6 if prec == FP32 else 1e-13)
    uu = np.einsum("mvij,mvkj->mvik", got, np.conj(got))
    assert np.abs(uu - np.eye(3)).max() <= (2e-6 if prec == FP32 else 1e-13)


@pytest.mark.parametrize("prec", PRECS)
def test_md_steps_match_oracle(gpu, orc, prec):
    dims, eps, n = (4, 4, 4, 6), 0.02, 3
    U = inputs.random_links(dims, seed=86)
    H = inputs.random_momenta(dims, seed=87)
    Uo, Ho = U, H
    for _ in range(n):
        Ho = orc.mom_update(dims, Uo, Ho, BETA, eps)
        Uo = orc.link_update(dims, Uo, Ho, eps)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(H)
        c.gauge_md_steps(BETA, eps, n, prec)
        Ug, Hg = c.links_download(), c.mom_download()
    assert rel(Ug, Uo) <= (2e-6 if prec == FP32 else 1e-13)
    assert rel(Hg, Ho) <= (2e-6 if prec == FP32 else 1e-13)


def test_deo_after_md_uses_moved_links(gpu, orc):
    """After FP64 and FP32 steps the fermion side (D_eo, whose df64 link
    formats are rebuilt from the moved links) equals the oracle's D_eo on the
    downloaded links."""
    dims = (4, 6, 8, 10)
    U = inputs.random_links(dims, seed=88)
    H = inputs.random_momenta(dims, seed=89)
    x = inputs.gaussian_field(dims, k=3)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(H)
        for prec in (FP64, NAT, FP32, FP64):
            c.gauge_md_steps(BETA, 0.05, 2, prec)
            Ud = c.links_download()
            assert rel(Ud, U) > 1e-3
            y = c.deo_apply(0, x)
            ref = orc.deo(dims, 0, Ud, x)
            assert rel(y, ref) <= 1e-13


def leapfrog_gpu(c, beta, tau, n, prec):
    e = tau / n
    c.gauge_mom_update(beta, 0.5 * e, prec)
    for k in range(n):
        c.gauge_link_update(e, prec)
        c.gauge_mom_update(beta, e if k < n - 1 else 0.5 * e, prec)


@pytest.mark.parametrize("prec", [FP64, NAT])
def test_md_reversible_and_second_order_fp64(gpu, prec):
    dims = (4, 4, 4, 8)
    U0 = inputs.random_links(dims, seed=90)
    H0 = inputs.random_momenta(dims, seed=91)
    with gpu.Context(dims) as c:
        c.links_upload(U0)
        c.mom_upload(H0)
        E0 = c.mom_energy() + c.gauge_action(BETA)
        leapfrog_gpu(c, BETA, 0.1, 4, prec)
        U1 = c.links_download()
        c.mom_upload(-c.mom_download())
        leapfrog_gpu(c, BETA, 0.1, 4, prec)
        assert rel(c.links_download(), U0) <= 1e-12 and rel(U1, U0) > 1e-3
        assert rel(-c.mom_download(), H0) <= 1e-12
        dH = []
        for n in (4, 8, 16):
            c.links_upload(U0)
            c.mom_upload(H0)
            leapfrog_gpu(c, BETA, 0.2, n, prec)
            dH.append(abs(c.mom_energy() + c.gauge_action(BETA) - E0))
    assert 3.5 <= dH[0] / dH[1] <= 4.5 and 3.5 <= dH[1] / dH[2] <= 4.5


def test_force_is_derivative_16(gpu):
    """At 16^4, GPU operations only: the central difference of the GPU action
    along exp(+-i h X) equals sum Tr(X F), with F read back from one momentum
    update (H = 0, eps = 1 gives H' = -F)."""
    dims, h = (16, 16, 16, 16), 1e-4
    U = inputs.random_links(dims, seed=92)
    X = inputs.random_momenta(dims, seed=93)
    with gpu.Context(dims) as c:
        c.links_upload(U)
        c.mom_upload(np.zeros_like(X))
        c.gauge_mom_update(BETA, 1.0)
        F = -c.mom_download()
        S = []
        for sign in (1.0, -1.0):
            c.links_upload(U)
            c.mom_upload(X)
            c.gauge_link_update(sign * h)
            S.append(c.gauge_action(BETA))
    num = (S[0] - S[1]) / (2 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    assert abs(num - ana) <= 1e-6 * abs(ana)


def test_mom_upload_checks(gpu):
    dims = (2, 2, 2, 2)
    with gpu.Context(dims) as c:
        c.links_upload(inputs.random_links(dims))
        with pytest.raises(gpu.LqcdError):
            c.gauge_md_steps(BETA, 0.1, 1)        # no momenta yet
        H = inputs.random_momenta(dims)
        bad = H.copy()
        bad[0, 0, 0, 1] += 0.5                     # not Hermitian
        with pytest.raises(gpu.LqcdError):
            c.mom_upload(bad)
        bad = H.copy()
        bad[1, 3] += np.eye(3)                     # not traceless
        with pytest.raises(gpu.LqcdError):
            c.mom_upload(bad)
        c.mom_upload(H)
        with pytest.raises(gpu.LqcdError):
            c.gauge_md_steps(BETA, 0.1, 1, 2)     # FP16 is not an MD precision
        c.gauge_md_steps(BETA, 0.1, 0)            # zero steps: nothing moves
        assert np.abs(c.mom_download() - H).max() <= 1e-14
