"""Pins for the CPU oracle: checks against what the paper and the mathematics
fix, written without re-using the oracle's own formulas.

Each check returns (ok: bool, detail: str) so that the same battery can be run
against the default oracle (tests/test_oracle_pins.py) and against builds
with a planted mistake (tests/test_oracle_mutants.py).

Sources of truth:
* Eq. (lexicographic_eo): brute-force rank of a site among the sites of its
  parity in lexicographic order;
* Eq. (diracblock): D_oe^dag = -D_eo (anti-hermiticity);
* gauge covariance of the covariant hops (Sec. 2: links transform as
  U_mu(n) -> Omega(n) U_mu(n) Omega(n+mu)^dag, quark fields as psi -> Omega psi);
* free field U = 1: the even-site plane waves are eigenvectors of
  m^2 - D_eo D_oe with eigenvalue m^2 + sum_mu sin^2 p_mu (antiperiodic
  momenta in time);
* Eq. (lineqeo) / Eq. (shlineq): the shifted systems' solutions from LAPACK
  (numpy.linalg.solve / eigvalsh) on small lattices.
"""
from __future__ import annotations

import itertools

import numpy as np

from paper_1701_00426_gb300 import inputs

MASS = 0.1


def sites(dims):
    """All coordinates in lexicographic order (x0 fastest)."""
    for x3, x2, x1, x0 in itertools.product(*(range(d) for d in dims[::-1])):
        yield (x0, x1, x2, x3)


def inner(a, b) -> complex:
    return complex(np.vdot(a.ravel(), b.ravel()))


def rel(a, b) -> float:
    den = max(np.linalg.norm(b), 1e-300)
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / den)


# --------------------------------------------------------------- geometry
def pin_geometry(orc, dims) -> tuple[bool, str]:
    rank = [0, 0]
    for n, x in enumerate(sites(dims)):
        if orc.lex(dims, x) != n:
            return False, f"lex of {x} is {orc.lex(dims, x)}, expected {n}"
        p = sum(x) % 2
        if orc.parity(x) != p:
            return False, f"parity of {x}"
        if orc.idxh(dims, x) != rank[p]:
            return False, f"idxh of {x} is {orc.idxh(dims, x)}, expected rank {rank[p]}"
        rank[p] += 1
    Vh = int(np.prod(dims)) // 2
    return (rank == [Vh, Vh]), f"parity counts {rank}"


# ------------------------------------------------------------------ phases
def pin_phase_anticommutation(orc, dims) -> tuple[bool, str]:
    """s_mu(x) s_nu(x+mu) = - s_nu(x) s_mu(x+nu) for every x and mu != nu (the
    property that makes the free D^2 diagonal; it survives the periodic wrap
    because every side is even, and the time-boundary sign cancels), and the
    time-link signs multiply to -1 around every time line (antiperiodic)."""
    for x in sites(dims):
        for mu in range(4):
            for nu in range(4):
                if mu == nu:
                    continue
                xm = list(x); xm[mu] = (xm[mu] + 1) % dims[mu]
                xn = list(x); xn[nu] = (xn[nu] + 1) % dims[nu]
                lhs = orc.link_sign(dims, x, mu) * orc.link_sign(dims, xm, nu)
                rhs = orc.link_sign(dims, x, nu) * orc.link_sign(dims, xn, mu)
                if lhs != -rhs:
                    return False, f"signs commute at {x} mu={mu} nu={nu}"
    for x0, x1, x2 in ((0, 0, 0), (1, 0, 0), (1, 1, 1), (0, 1, 0)):
        prod = 1.0
        for t in range(dims[3]):
            prod *= orc.link_sign(dims, (x0, x1, x2, t), 3)
        if prod != -1.0:
            return False, f"time line ({x0},{x1},{x2}) sign product {prod}"
    return True, "ok"


# -------------------------------------------------------- anti-hermiticity
def pin_antihermitian(orc, dims, seed=11) -> tuple[bool, str]:
    U = inputs.random_links(dims, seed=seed)
    Vh = int(np.prod(dims)) // 2
    rng = np.random.default_rng(seed + 1)
    x = rng.standard_normal((Vh, 3)) + 1j * rng.standard_normal((Vh, 3))
    y = rng.standard_normal((Vh, 3)) + 1j * rng.standard_normal((Vh, 3))
    Dx = orc.deo(dims, 0, U, x)   # D_eo x_odd
    Dy = orc.deo(dims, 1, U, y)   # D_oe y_even
    lhs = inner(y, Dx)
    rhs = -inner(Dy, x)
    scale = np.linalg.norm(y) * np.linalg.norm(Dx)
    err = abs(lhs - rhs) / scale
    return err <= 1e-14, f"anti-hermiticity defect {err:.2e}"


# ---------------------------------------------------------- gauge covariance
def pin_gauge_covariance(orc, dims, seed=21) -> tuple[bool, str]:
    U = inputs.random_links(dims, seed=seed)
    V = int(np.prod(dims))
    Vh = V // 2
    Om = inputs.random_gauge_transform(dims, seed=seed + 1)
    # site tables by plain enumeration (independent of the oracle's helpers)
    coords = list(sites(dims))
    lex_of = {x: n for n, x in enumerate(coords)}
    half = {0: [], 1: []}
    for x in coords:
        half[sum(x) % 2].append(x)
    Up = np.empty_like(U)
    for mu in range(4):
        for n, x in enumerate(coords):
            xp = list(x); xp[mu] = (xp[mu] + 1) % dims[mu]
            Up[mu, n] = Om[n] @ U[mu, n] @ Om[lex_of[tuple(xp)]].conj().T
    rng = np.random.default_rng(seed + 2)
    ok = True
    worst = 0.0
    for out_par in (0, 1):
        in_par = 1 - out_par
        psi = rng.standard_normal((Vh, 3)) + 1j * rng.standard_normal((Vh, 3))
        psip = np.stack([Om[lex_of[x]] @ psi[i] for i, x in enumerate(half[in_par])])
        lhs = orc.deo(dims, out_par, Up, psip)
        D = orc.deo(dims, out_par, U, psi)
        rhs = np.stack([Om[lex_of[x]] @ D[i] for i, x in enumerate(half[out_par])])
        e = rel(lhs, rhs)
        worst = max(worst, e)
        ok &= e <= 1e-14
    return ok, f"covariance defect {worst:.2e}"


# ------------------------------------------------------------- free field
def free_eigenvalue(dims, k, mass=MASS) -> float:
    p = [2 * np.pi * k[m] / dims[m] for m in range(3)]
    p.append(2 * np.pi * (k[3] + 0.5) / dims[3])
    return mass * mass + sum(np.sin(q) ** 2 for q in p)


def plane_wave_even(dims, k, chi) -> np.ndarray:
    """e^{i p.x} chi on the even sites, listed by rank in lexicographic order."""
    p = [2 * np.pi * k[m] / dims[m] for m in range(3)]
    p.append(2 * np.pi * (k[3] + 0.5) / dims[3])
    rows = []
    for x in sites(dims):
        if sum(x) % 2 == 0:
            rows.append(np.exp(1j * sum(p[m] * x[m] for m in range(4))) * chi)
    return np.array(rows)


def pin_free_plane_waves(orc, dims, ks, mass=MASS) -> tuple[bool, str]:
    U = inputs.unit_links(dims)
    chi = np.array([0.3 + 0.1j, -0.7j, 1.1])
    worst = 0.0
    for k in ks:
        psi = plane_wave_even(dims, k, chi)
        lam = free_eigenvalue(dims, k, mass)
        out = orc.apply_A(dims, U, mass, 0.0, psi)
        worst = max(worst, rel(out, lam * psi))
    return worst <= 1e-13, f"plane-wave defect {worst:.2e}"


def dense_A(orc, dims, U, mass, sigma=0.0) -> np.ndarray:
    """A + sigma assembled column by column from the oracle's operator."""
    Vh = int(np.prod(dims)) // 2
    n = 3 * Vh
    A = np.empty((n, n), np.complex128)
    e = np.zeros(n, np.complex128)
    for j in range(n):
        e[:] = 0
        e[j] = 1
        A[:, j] = orc.apply_A(dims, U, mass, sigma, e.reshape(Vh, 3)).ravel()
    return A


def pin_free_spectrum(orc, dims, mass=MASS) -> tuple[bool, str]:
    """Whole spectrum of the free even/odd operator vs the closed form."""
    U = inputs.unit_links(dims)
    A = dense_A(orc, dims, U, mass)
    ev = np.linalg.eigvalsh(A)
    lam = []
    for k in itertools.product(*(range(d) for d in dims)):
        lam.append(free_eigenvalue(dims, k, mass))
    lam = np.sort(np.array(lam))
    # each even-site plane wave is shared by p and p + (pi,pi,pi,pi); 3 colours
    expect = np.sort(np.repeat(lam[::2], 3))
    err = float(np.max(np.abs(ev - expect)))
    return err <= 1e-12, f"free spectrum max defect {err:.2e}"


def pin_two_site(orc, mass=MASS) -> tuple[bool, str]:
    """On 2^4 (where n+mu = n-mu) the free operator is (m^2 + 1) I."""
    dims = (2, 2, 2, 2)
    U = inputs.unit_links(dims)
    rng = np.random.default_rng(5)
    v = rng.standard_normal((8, 3)) + 1j * rng.standard_normal((8, 3))
    out = orc.apply_A(dims, U, mass, 0.0, v)
    e = rel(out, (mass * mass + 1.0) * v)
    return e <= 1e-15, f"2^4 free defect {e:.2e}"


def pin_hermitian_positive(orc, dims, mass=MASS) -> tuple[bool, str]:
    U = inputs.random_links(dims, seed=33)
    A = dense_A(orc, dims, U, mass)
    herm = float(np.max(np.abs(A - A.conj().T)))
    ev = np.linalg.eigvalsh(A)
    ok = herm <= 1e-14 and ev[0] >= mass * mass * (1 - 1e-10)
    return ok, f"hermiticity {herm:.2e}, lowest eigenvalue {ev[0]:.3e}"


def numpy_deo_matrix(dims, U, out_parity) -> np.ndarray:
    """D_eo (out_parity 0) or D_oe (out_parity 1) as a dense (3 Vh, 3 Vh)
    matrix, assembled here from Eq. (diracblock) without the oracle: rows are
    the output sites of one parity and columns the input sites of the other,
    both in rank order (Eq. lexicographic_eo), with the staggered sign
    eta_mu(x) = (-1)^(x_0 + ... + x_{mu-1}) and -1 on the time links of the
    last time slice."""
    coords = list(sites(dims))
    lex_of = {x: n for n, x in enumerate(coords)}
    rank = {}
    count = [0, 0]
    for x in coords:
        p = sum(x) % 2
        rank[x] = count[p]
        count[p] += 1
    Vh = len(coords) // 2

    def sign(x, mu):
        s = -1.0 if sum(x[:mu]) % 2 else 1.0
        if mu == 3 and x[3] == dims[3] - 1:
            s = -s
        return s

    D = np.zeros((3 * Vh, 3 * Vh), np.complex128)
    for x in coords:
        if sum(x) % 2 != out_parity:
            continue
        i = rank[x]
        for mu in range(4):
            xf = list(x); xf[mu] = (xf[mu] + 1) % dims[mu]; xf = tuple(xf)
            xb = list(x); xb[mu] = (xb[mu] - 1) % dims[mu]; xb = tuple(xb)
            jf, jb = rank[xf], rank[xb]
            D[3 * i:3 * i + 3, 3 * jf:3 * jf + 3] += 0.5 * sign(x, mu) * U[mu, lex_of[x]]
            D[3 * i:3 * i + 3, 3 * jb:3 * jb + 3] -= 0.5 * sign(xb, mu) * U[mu, lex_of[xb]].conj().T
    return D


def numpy_A(dims, U, mass, sigma=0.0) -> np.ndarray:
    """m^2 + sigma - D_eo D_oe (Eq. lineqeo) from numpy_deo_matrix."""
    Deo, Doe = numpy_deo_matrix(dims, U, 0), numpy_deo_matrix(dims, U, 1)
    return (mass * mass + sigma) * np.eye(Deo.shape[0]) - Deo @ Doe


def pin_A_numpy_assembly(orc, dims, mass=MASS, sigma=0.37, seed=57) -> tuple[bool, str]:
    """The oracle's matrix-free A + sigma, column by column, equals the
    matrix assembled here from Eq. (diracblock) and Eq. (lineqeo)."""
    U = inputs.random_links(dims, seed=seed)
    ref = numpy_A(dims, U, mass, sigma)
    got = dense_A(orc, dims, U, mass, sigma)
    e = float(np.abs(got - ref).max() / np.abs(ref).max())
    return e <= 1e-14, f"max |A_oracle - A_numpy| / max |A| = {e:.2e}"


def pin_true_residual(orc, dims, mass=MASS, seed=58) -> tuple[bool, str]:
    """oracle_true_residual = ||(A + sigma) x - b|| / ||b|| with A assembled in
    numpy and x = the LAPACK solution perturbed by a relative 1e-3, so the
    expected value is of order 1e-3, not zero; shifts 0, 0.37 and 25."""
    U = inputs.random_links(dims, seed=seed)
    Vh = int(np.prod(dims)) // 2
    rng = np.random.default_rng(seed + 1)
    b = (rng.standard_normal((Vh, 3)) + 1j * rng.standard_normal((Vh, 3))) * 3.0
    worst, vals = 0.0, []
    for sigma in (0.0, 0.37, 25.0):
        A = numpy_A(dims, U, mass, sigma)
        xs = np.linalg.solve(A, b.ravel())
        noise = rng.standard_normal(xs.shape) + 1j * rng.standard_normal(xs.shape)
        x = (xs + 1e-3 * np.linalg.norm(xs) / np.linalg.norm(noise) * noise).reshape(Vh, 3)
        expect = np.linalg.norm(A @ x.ravel() - b.ravel()) / np.linalg.norm(b)
        got = orc.true_residual(dims, U, mass, sigma, b, x)
        vals.append(expect)
        worst = max(worst, abs(got - expect) / expect)
    ok = worst <= 1e-12 and min(vals) > 1e-5
    return ok, f"max relative defect {worst:.2e} over residuals {['%.2e' % v for v in vals]}"


# ---------------------------------------------------------------- solvers
def pin_mscg_vs_lapack(orc, dims, shifts, mass=MASS, tol=1e-10) -> tuple[bool, str]:
    U = inputs.random_links(dims, seed=44)
    Vh = int(np.prod(dims)) // 2
    b = inputs.gaussian_field(dims, k=3)
    A = dense_A(orc, dims, U, mass)
    x, info = orc.mscg(dims, U, mass, shifts, b, tol)
    if info["status"] != 0:
        return False, f"mscg status {info['status']}"
    # the shifted recurrences alone must reach tol: the plain-CG clean-up
    # after the true-residual check exists for rounding drift, and at this
    # size and tolerance rounding never needs it
    if info["refine_iters"] != 0:
        return False, f"shifted recurrences needed {info['refine_iters']} refinement iterations"
    ev = np.linalg.eigvalsh(A)
    worst = 0.0
    for i, s in enumerate(shifts):
        xs = np.linalg.solve(A + s * np.eye(3 * Vh), b.ravel())
        kappa = (ev[-1] + s) / (ev[0] + s)
        e = rel(x[i].ravel(), xs) / (kappa * tol)
        worst = max(worst, e)
        r = np.linalg.norm((A + s * np.eye(3 * Vh)) @ x[i].ravel() - b.ravel()) / np.linalg.norm(b)
        if r > tol:
            return False, f"shift {s}: LAPACK-checked residual {r:.2e} > tol"
    return worst <= 1.0, f"max error / (kappa tol) = {worst:.3f}"


def pin_free_solve(orc, dims, shifts, k, mass=MASS, tol=1e-12) -> tuple[bool, str]:
    U = inputs.unit_links(dims)
    chi = np.array([1.0, 0.5j, -0.25])
    b = plane_wave_even(dims, k, chi)
    lam = free_eigenvalue(dims, k, mass)
    x, info = orc.mscg(dims, U, mass, shifts, b, tol)
    worst = 0.0
    for i, s in enumerate(shifts):
        worst = max(worst, rel(x[i], b / (lam + s)))
    return worst <= 1e-10, f"free solve defect {worst:.2e}"


# ------------------------------------------------- rational function (RHMC)
RAT_A0 = 0.25
RAT_A = [0.5, 1.2, 0.05, 3.0]
RAT_SIGMA = [1e-3, 0.1, 2.0, 30.0]


def rational_bound(tol, bnorm, a, sigma, lam_min) -> float:
    """||y - r(A) b|| when every shifted solve meets the true residual tol:
    ||x_i - x_i*|| <= ||(A + sigma_i)^{-1}|| tol ||b||."""
    return tol * bnorm * sum(abs(ai) / (lam_min + si) for ai, si in zip(a, sigma))


def pin_rational_vs_dense(orc, dims, mass=MASS, tol=1e-10) -> tuple[bool, str]:
    """r(A) b = V diag(a0 + sum_i a_i / (lam + sigma_i)) V^dag b from the
    eigendecomposition of the dense A (LAPACK), and the action b^dag r(A) b."""
    U = inputs.random_links(dims, seed=55)
    b = inputs.gaussian_field(dims, k=6)
    y, act, st = orc.rational_apply(dims, U, mass, RAT_A0, RAT_A, RAT_SIGMA, b, tol)
    if st != 0:
        return False, f"status {st}"
    lam, V = np.linalg.eigh(dense_A(orc, dims, U, mass))
    r = RAT_A0 + sum(ai / (lam + si) for ai, si in zip(RAT_A, RAT_SIGMA))
    ystar = V @ (r * (V.conj().T @ b.ravel()))
    bound = rational_bound(tol, np.linalg.norm(b), RAT_A, RAT_SIGMA, lam[0])
    err = float(np.linalg.norm(y.ravel() - ystar))
    act_star = float(np.vdot(b.ravel(), ystar).real)
    aerr = abs(act - act_star)
    ok = err <= bound and aerr <= np.linalg.norm(b) * bound
    return ok, f"|y - y*| = {err:.2e} (bound {bound:.2e}), |S - S*| = {aerr:.2e}"


def pin_rational_inverse_sqrt(orc, dims, mass=MASS, tol=1e-10, n_poles=20) -> tuple[bool, str]:
    """With the quadrature coefficients of x^(-1/2), r(A) b is A^(-1/2) b (dense
    eigendecomposition) up to max_k |r(lam_k) - lam_k^(-1/2)| ||b|| plus the
    solver bound; the action is b^dag A^(-1/2) b to the same order."""
    from paper_1701_00426_gb300 import rational
    U = inputs.random_links(dims, seed=56)
    b = inputs.gaussian_field(dims, k=7)
    lam, V = np.linalg.eigh(dense_A(orc, dims, U, mass))
    a0, a, sig = rational.inverse_sqrt_poles(n_poles, lam[0], lam[-1])
    y, act, st = orc.rational_apply(dims, U, mass, a0, a, sig, b, tol)
    if st != 0:
        return False, f"status {st}"
    ystar = V @ (lam ** -0.5 * (V.conj().T @ b.ravel()))
    approx = float(np.max(np.abs(rational.evaluate(a0, a, sig, lam) - lam ** -0.5)))
    bnorm = np.linalg.norm(b)
    bound = approx * bnorm + rational_bound(tol, bnorm, a, sig, lam[0])
    err = float(np.linalg.norm(y.ravel() - ystar))
    aerr = abs(act - float(np.vdot(b.ravel(), ystar).real))
    ok = err <= 1.01 * bound and aerr <= 1.01 * bnorm * bound and approx < 1e-6
    return ok, f"|y - A^-1/2 b| = {err:.2e} (bound {bound:.2e}, rational error {approx:.1e})"


def pin_rational_free(orc, dims=(4, 4, 6, 8), k=(1, 3, 2, 5), mass=MASS, tol=1e-12) -> tuple[bool, str]:
    """Free field: a plane wave b is an eigenvector, so r(A) b = r(lam_p) b."""
    U = inputs.unit_links(dims)
    b = plane_wave_even(dims, k, np.array([1.0, 0.5j, -0.25]))
    lam = free_eigenvalue(dims, k, mass)
    y, act, st = orc.rational_apply(dims, U, mass, RAT_A0, RAT_A, RAT_SIGMA, b, tol)
    r = RAT_A0 + sum(ai / (lam + si) for ai, si in zip(RAT_A, RAT_SIGMA))
    e = rel(y, r * b)
    ae = abs(act - r * np.linalg.norm(b) ** 2) / (r * np.linalg.norm(b) ** 2)
    return st == 0 and e <= 1e-10 and ae <= 1e-10, f"free rational defect {e:.2e}, action {ae:.2e}"


# ------------------------------------------------------- gauge MD (f2)
BETA = 5.5


def pin_gauge_action_unit(orc, dims=(4, 4, 4, 6), beta=BETA) -> tuple[bool, str]:
    """U = 1: every plaquette and rectangle has trace 3, 6 plaquettes and 12
    rectangles per site: S = -(beta/3) V (6 c0 + 12 c1) 3 = -9 beta V."""
    V = int(np.prod(dims))
    S = orc.gauge_action(dims, inputs.unit_links(dims), beta)
    return abs(S + 9.0 * beta * V) <= 1e-12 * 9.0 * beta * V, f"S(1) = {S}, expected {-9.0 * beta * V}"


def gauge_transform_links(dims, U, Om):
    coords = list(sites(dims))
    lex_of = {x: n for n, x in enumerate(coords)}
    Up = np.empty_like(U)
    for mu in range(4):
        for n, x in enumerate(coords):
            xp = list(x); xp[mu] = (xp[mu] + 1) % dims[mu]
            Up[mu, n] = Om[n] @ U[mu, n] @ Om[lex_of[tuple(xp)]].conj().T
    return Up


def pin_gauge_invariance(orc, dims=(4, 4, 4, 6), beta=BETA, seed=71) -> tuple[bool, str]:
    """S[U^Omega] = S[U] and F[U^Omega]_mu(x) = Omega(x) F[U]_mu(x) Omega(x)^dag."""
    U = inputs.random_links(dims, seed=seed)
    Om = inputs.random_gauge_transform(dims, seed=seed + 1)
    Up = gauge_transform_links(dims, U, Om)
    S, Sp = orc.gauge_action(dims, U, beta), orc.gauge_action(dims, Up, beta)
    F, Fp = orc.gauge_force(dims, U, beta), orc.gauge_force(dims, Up, beta)
    Frot = np.einsum("vij,mvjk,vlk->mvil", Om, F, Om.conj())
    eS = abs(S - Sp) / abs(S)
    eF = rel(Fp, Frot)
    return eS <= 1e-13 and eF <= 1e-13, f"action {eS:.2e}, force covariance {eF:.2e}"


def pin_force_is_derivative(orc, dims=(4, 4, 4, 4), beta=BETA, h=1e-4, seed=72) -> tuple[bool, str]:
    """d/de S(exp(i e X) U) at e = 0 equals sum Tr(X F) for a random Hermitian
    traceless X on every link (central difference, S enumerated loop by loop),
    and F is Hermitian and traceless."""
    U = inputs.random_links(dims, seed=seed)
    X = inputs.random_momenta(dims, seed=seed + 1)
    F = orc.gauge_force(dims, U, beta)
    num = (orc.gauge_action(dims, orc.link_update(dims, U, X, h), beta)
           - orc.gauge_action(dims, orc.link_update(dims, U, X, -h), beta)) / (2.0 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    herm = float(np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max())
    trace = float(np.abs(np.trace(F, axis1=-2, axis2=-1)).max())
    e = abs(num - ana) / abs(ana)
    ok = e <= 1e-6 and herm <= 1e-13 * np.abs(F).max() and trace <= 1e-13 * np.abs(F).max()
    return ok, f"derivative defect {e:.2e}, hermiticity {herm:.1e}, trace {trace:.1e}"


def pin_exp(orc, seed=73) -> tuple[bool, str]:
    """exp(i t H) against scipy.linalg.expm; unitary with determinant 1."""
    import scipy.linalg
    H = inputs.random_momenta((2, 2, 2, 2), seed=seed)[0, :6]
    worst = 0.0
    for t in (1e-3, 0.3, 5.0):
        for h in H:
            E = orc.exp_iH(h, t)
            ref = scipy.linalg.expm(1j * t * h)
            worst = max(worst, float(np.abs(E - ref).max()),
                        float(np.abs(E @ E.conj().T - np.eye(3)).max()), abs(np.linalg.det(E) - 1.0))
    return worst <= 1e-13, f"exp defect {worst:.2e}"


def leapfrog(orc, dims, U, H, beta, tau, n):
    """tau split in n leapfrog steps from the two updates (H half, U, H half)."""
    e = tau / n
    H = orc.mom_update(dims, U, H, beta, 0.5 * e)
    for k in range(n):
        U = orc.link_update(dims, U, H, e)
        H = orc.mom_update(dims, U, H, beta, e if k < n - 1 else 0.5 * e)
    return U, H


def pin_md_reversible(orc, dims=(4, 4, 4, 4), beta=BETA, seed=74) -> tuple[bool, str]:
    """Leapfrog forward, momenta flipped, leapfrog again: back to the start."""
    U0 = inputs.random_links(dims, seed=seed)
    H0 = inputs.random_momenta(dims, seed=seed + 1)
    U1, H1 = leapfrog(orc, dims, U0, H0, beta, 0.1, 4)
    U2, H2 = leapfrog(orc, dims, U1, -H1, beta, 0.1, 4)
    eU, eH = rel(U2, U0), rel(-H2, H0)
    moved = rel(U1, U0)
    return eU <= 1e-12 and eH <= 1e-12 and moved > 1e-3, f"return defect U {eU:.1e}, H {eH:.1e} (moved {moved:.1e})"


def pin_md_energy(orc, dims=(4, 4, 4, 4), beta=BETA, seed=75) -> tuple[bool, str]:
    """dH = dK + dS of a leapfrog trajectory shrinks as the squared step: four
    times less per halving of the step (second-order integrator)."""
    U0 = inputs.random_links(dims, seed=seed)
    H0 = inputs.random_momenta(dims, seed=seed + 1)
    E0 = orc.mom_energy(dims, H0) + orc.gauge_action(dims, U0, beta)
    dH = []
    for n in (4, 8, 16):
        U, H = leapfrog(orc, dims, U0, H0, beta, 0.2, n)
        dH.append(abs(orc.mom_energy(dims, H) + orc.gauge_action(dims, U, beta) - E0))
    r1, r2 = dH[0] / dH[1], dH[1] / dH[2]
    ok = 3.5 <= r1 <= 4.5 and 3.5 <= r2 <= 4.5
    return ok, f"|dH| {dH[0]:.2e} {dH[1]:.2e} {dH[2]:.2e}, ratios {r1:.2f} {r2:.2f}"


# --------------------------------------------------- fermion force (f4)
FF_MASS, FF_A0 = 0.3, 0.2
FF_A, FF_SIGMA = [0.3, 0.8, 1.5], [0.05, 0.5, 3.0]


def pin_fermion_force_is_derivative(orc, dims=(4, 4, 4, 4), h=1e-4, tol=1e-13, seed=95) -> tuple[bool, str]:
    """d/de S_f(exp(i e X) U) at e = 0, S_f = phi^dag r(A) phi evaluated by the
    oracle's rational application (central difference), equals sum Tr(X F_f);
    F_f Hermitian and traceless."""
    U = inputs.random_links(dims, seed=seed)
    phi = inputs.gaussian_field(dims, k=seed)
    X = inputs.random_momenta(dims, seed=seed + 1)
    F, S, st = orc.fermion_force(dims, U, FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)
    if st != 0:
        return False, f"status {st}"
    Sp = orc.rational_apply(dims, orc.link_update(dims, U, X, h), FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)[1]
    Sm = orc.rational_apply(dims, orc.link_update(dims, U, X, -h), FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)[1]
    num = (Sp - Sm) / (2.0 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    e = abs(num - ana) / abs(ana)
    herm = float(np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max())
    trace = float(np.abs(np.trace(F, axis1=-2, axis2=-1)).max())
    ok = e <= 1e-6 and herm <= 1e-13 * np.abs(F).max() and trace <= 1e-13 * np.abs(F).max()
    return ok, f"derivative defect {e:.2e}, hermiticity {herm:.1e}, trace {trace:.1e}"


def pin_fermion_force_covariant(orc, dims=(4, 4, 4, 6), tol=1e-13, seed=96) -> tuple[bool, str]:
    """U -> U^Omega, phi -> Omega phi on the even sites: F_f_mu(x) -> Omega(x) F_f_mu(x) Omega(x)^dag
    and S_f unchanged."""
    U = inputs.random_links(dims, seed=seed)
    Om = inputs.random_gauge_transform(dims, seed=seed + 1)
    phi = inputs.gaussian_field(dims, k=seed)
    evens = [n for n, x in enumerate(sites(dims)) if sum(x) % 2 == 0]
    phip = np.stack([Om[n] @ phi[i] for i, n in enumerate(evens)])
    F, S, _ = orc.fermion_force(dims, U, FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)
    Fp, Sp, _ = orc.fermion_force(dims, gauge_transform_links(dims, U, Om), FF_MASS, FF_A0, FF_A, FF_SIGMA, phip, tol)
    Frot = np.einsum("vij,mvjk,vlk->mvil", Om, F, Om.conj())
    eF, eS = rel(Fp, Frot), abs(Sp - S) / abs(S)
    return eF <= 1e-10 and eS <= 1e-12, f"force covariance {eF:.2e}, action {eS:.2e}"


# Stout smearing (isotropic weight per level; Sec. 2.1 stout-improved action)
STOUT_RHO = 0.15
STOUT_LEVELS = 2


def pin_stout_basic(orc, dims=(4, 4, 4, 6), seed=97) -> tuple[bool, str]:
    """rho = 0 leaves the links unchanged (bit for bit); smeared links stay in
    SU(3); smearing commutes with gauge transformations, U^Omega ->
    smear(U)^Omega."""
    U = inputs.random_links(dims, seed=seed)
    same = np.array_equal(orc.stout_smear(dims, U, 0.0, 1), U)
    Us = orc.stout_smear(dims, U, STOUT_RHO, STOUT_LEVELS)
    unit = float(np.abs(np.einsum("mvij,mvkj->mvik", Us, Us.conj()) - np.eye(3)).max())
    det = float(np.abs(np.linalg.det(Us) - 1.0).max())
    Om = inputs.random_gauge_transform(dims, seed=seed + 1)
    lhs = orc.stout_smear(dims, gauge_transform_links(dims, U, Om), STOUT_RHO, STOUT_LEVELS)
    cov = rel(lhs, gauge_transform_links(dims, Us, Om))
    ok = same and unit <= 1e-13 and det <= 1e-13 and cov <= 1e-13
    return ok, f"rho=0 identity {same}, unitarity {unit:.1e}, det {det:.1e}, covariance {cov:.1e}"


def pin_stout_smooths(orc, dims=(4, 4, 4, 4), seed=98) -> tuple[bool, str]:
    """A stout step with small rho moves the links along the descent direction
    of the plaquette action (the staple sum C U^dag is the negative gradient
    of the Wilson action), so the Wilson action of the smeared links is lower
    than that of the thin links and falls further as rho grows."""
    U = inputs.random_links(dims, seed=seed)

    def wilson(Ut):
        return sum(-float(np.trace(plaq(dims, Ut, mu, nu), axis1=1, axis2=2).real.sum())
                   for mu in range(4) for nu in range(mu + 1, 4))

    s = [wilson(orc.stout_smear(dims, U, r, 1)) for r in (0.0, 0.01, 0.02)]
    return s[0] > s[1] > s[2], f"Wilson action at rho = 0, 0.01, 0.02: {s}"


def pin_stout_single_link(orc, dims=(4, 4, 4, 4), rho=0.11, nu0=1, y=(1, 2, 0, 3), seed=101) -> tuple[bool, str]:
    """One stout level of a field that is the identity on every link but one,
    U_nu0(y) = W in SU(3), worked out by hand from the definition of C, Omega
    and Q (each staple product is the identity unless it passes through W):
      link (y, nu0):                   C = 6 rho 1 (six staples, none holds W);
      links (y, mu), mu != nu0:        the upper staple in nu0 is W;
      links (y - mu, mu):              the upper staple in nu0 ends in W^dag;
      links (y + nu0, mu):             the lower staple in nu0 starts with W^dag;
      links (y + nu0 - mu, mu):        the lower staple in nu0 ends in W;
      links (y - mu, nu0):             the upper staple in mu has W in the middle;
      links (y + mu, nu0):             the lower staple in mu has W in the middle;
    then C = rho (S + 5 1) with S that staple, Omega = C U^dag, and every other
    link has C = 6 rho 1, so Q = 0 and the link stays the identity: 19 links
    move.
    Expected U' = expm(iQ) U with scipy; compared link by link."""
    import scipy.linalg
    V = int(np.prod(dims))
    coords = list(sites(dims))
    lex_of = {x: n for n, x in enumerate(coords)}
    W = inputs.random_links((2, 2, 2, 2), seed=seed)[0, 0]
    U = inputs.unit_links(dims).copy()
    U[nu0, lex_of[y]] = W

    def step(x, mu, d):
        z = list(x); z[mu] = (z[mu] + d) % dims[mu]; return tuple(z)

    eye = np.eye(3)
    C = np.empty((4, V, 3, 3), complex)
    C[:] = 6.0 * rho * eye
    C[nu0, lex_of[y]] = 6.0 * rho * eye
    for mu in range(4):
        if mu == nu0:
            continue
        for x, S in ((y, W), (step(y, mu, -1), W.conj().T), (step(y, nu0, 1), W.conj().T),
                     (step(step(y, nu0, 1), mu, -1), W)):
            C[mu, lex_of[x]] = rho * (S + 5.0 * eye)
        for x in (step(y, mu, -1), step(y, mu, 1)):
            C[nu0, lex_of[x]] = rho * (W + 5.0 * eye)
    expect = np.empty_like(U)
    for mu in range(4):
        for n in range(V):
            Om = C[mu, n] @ U[mu, n].conj().T
            T = Om.conj().T - Om
            Q = 0.5j * T - (1j / 6.0) * np.trace(T) * eye
            expect[mu, n] = scipy.linalg.expm(1j * Q) @ U[mu, n]
    got = orc.stout_smear(dims, U, rho, 1)
    e = float(np.abs(got - expect).max())
    moved = int(np.sum(np.abs(expect - U).reshape(4 * V, 9).max(axis=1) > 1e-12))
    return e <= 1e-13 and moved == 19, f"max defect {e:.2e}, links moved {moved} (expected 19)"


def plaq(dims, U, mu, nu):
    """P_{mu nu}(x) for every site by plain enumeration."""
    coords = list(sites(dims))
    lex_of = {x: n for n, x in enumerate(coords)}
    out = np.empty((len(coords), 3, 3), complex)
    for n, x in enumerate(coords):
        xm = list(x); xm[mu] = (xm[mu] + 1) % dims[mu]
        xn = list(x); xn[nu] = (xn[nu] + 1) % dims[nu]
        out[n] = U[mu, n] @ U[nu, lex_of[tuple(xm)]] @ U[mu, lex_of[tuple(xn)]].conj().T @ U[nu, n].conj().T
    return out


def pin_stout_force_is_derivative(orc, dims=(4, 4, 4, 4), beta=BETA, h=1e-4, seed=99) -> tuple[bool, str]:
    """For S(U) = S_g(smear^2(U)) (Symanzik action of twice-smeared links):
    d/de S(exp(i e X) U) at e = 0 equals sum Tr(X F) with F the force on the
    smeared links chained back to the thin ones (central difference)."""
    U = inputs.random_links(dims, seed=seed)
    X = inputs.random_momenta(dims, seed=seed + 1)
    Us = orc.stout_smear(dims, U, STOUT_RHO, STOUT_LEVELS)
    F = orc.stout_force(dims, U, STOUT_RHO, orc.gauge_force(dims, Us, beta), STOUT_LEVELS)

    def S(Ut):
        return orc.gauge_action(dims, orc.stout_smear(dims, Ut, STOUT_RHO, STOUT_LEVELS), beta)

    num = (S(orc.link_update(dims, U, X, h)) - S(orc.link_update(dims, U, X, -h))) / (2.0 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    e = abs(num - ana) / abs(ana)
    herm = float(np.abs(F - np.conj(np.swapaxes(F, -1, -2))).max())
    trace = float(np.abs(np.trace(F, axis1=-2, axis2=-1)).max())
    ok = e <= 1e-6 and herm <= 1e-13 * np.abs(F).max() and trace <= 1e-13 * np.abs(F).max()
    return ok, f"derivative defect {e:.2e}, hermiticity {herm:.1e}, trace {trace:.1e}"


def pin_stout_fermion_force(orc, dims=(4, 4, 4, 4), h=1e-4, tol=1e-13, seed=100) -> tuple[bool, str]:
    """The rational pseudofermion action on smeared links, S_f(smear^2(U)):
    its central difference along thin-link directions equals sum Tr(X F)
    with F = the fermion force on the smeared links chained back."""
    U = inputs.random_links(dims, seed=seed)
    phi = inputs.gaussian_field(dims, k=seed)
    X = inputs.random_momenta(dims, seed=seed + 1)
    Us = orc.stout_smear(dims, U, STOUT_RHO, STOUT_LEVELS)
    Fs, _, st = orc.fermion_force(dims, Us, FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)
    if st != 0:
        return False, f"status {st}"
    F = orc.stout_force(dims, U, STOUT_RHO, Fs, STOUT_LEVELS)

    def S(Ut):
        Ust = orc.stout_smear(dims, Ut, STOUT_RHO, STOUT_LEVELS)
        return orc.rational_apply(dims, Ust, FF_MASS, FF_A0, FF_A, FF_SIGMA, phi, tol)[1]

    num = (S(orc.link_update(dims, U, X, h)) - S(orc.link_update(dims, U, X, -h))) / (2.0 * h)
    ana = float(np.einsum("mvij,mvji->", X, F).real)
    e = abs(num - ana) / abs(ana)
    return e <= 1e-6, f"derivative defect {e:.2e}"


BATTERY = [
    ("geometry 4x6x8x10", lambda o: pin_geometry(o, (4, 6, 8, 10))),
    ("phase anticommutation 4x6x8x10", lambda o: pin_phase_anticommutation(o, (4, 6, 8, 10))),
    ("anti-hermiticity 4x6x8x10", lambda o: pin_antihermitian(o, (4, 6, 8, 10))),
    ("gauge covariance 4x4x4x6", lambda o: pin_gauge_covariance(o, (4, 4, 4, 6))),
    ("free plane waves 4x6x8x10", lambda o: pin_free_plane_waves(
        o, (4, 6, 8, 10), [(0, 0, 0, 0), (1, 2, 3, 4), (3, 1, 5, 9), (2, 5, 7, 2)])),
    ("free 2^4", pin_two_site),
    ("mscg vs LAPACK 4^4", lambda o: pin_mscg_vs_lapack(o, (4, 4, 4, 4), [1e-3, 0.05, 1.0, 30.0])),
    ("free solve 4x4x6x8", lambda o: pin_free_solve(o, (4, 4, 6, 8), [0.0, 0.3, 7.0], (1, 3, 2, 5))),
    ("rational vs dense 4^4", lambda o: pin_rational_vs_dense(o, (4, 4, 4, 4))),
    ("rational free 4x4x6x8", pin_rational_free),
    ("gauge action U=1", pin_gauge_action_unit),
    ("gauge force = derivative of the action 4^4", pin_force_is_derivative),
    ("MD energy conservation O(dt^2) 4^4", pin_md_energy),
    ("fermion force = derivative of the rational action 4^4", pin_fermion_force_is_derivative),
    ("A vs numpy assembly 4x4x2x6", lambda o: pin_A_numpy_assembly(o, (4, 4, 2, 6))),
    ("true residual vs numpy A 2^4", lambda o: pin_true_residual(o, (2, 2, 2, 2))),
    ("true residual vs numpy A 4^4", lambda o: pin_true_residual(o, (4, 4, 4, 4))),
    ("stout: one non-trivial link by hand 4^4", pin_stout_single_link),
    ("stout: rho=0, SU(3), gauge covariance 4x4x4x6", pin_stout_basic),
    ("stout smearing lowers the Wilson action 4^4", pin_stout_smooths),
    ("stout force chain = derivative 4^4", pin_stout_force_is_derivative),
]
