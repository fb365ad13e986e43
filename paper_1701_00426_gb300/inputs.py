"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This module draws random numbers and lays them out in the canonical host
formats; it contains none of the method's arithmetic (no Dirac operator, no
phases, no solver, no link compression).  Both sides receive identical bytes.

The paper's workloads are thermalised gauge configurations that are not
available here; "hot" random SU(3) fields of the same lattice shapes stand in
for them.  Recipe:

* links: for every (mu, site) a 3x3 matrix with i.i.d. N(0,1) real and
  imaginary parts, orthonormalised row by row (two-pass Gram-Schmidt), then the last
  row multiplied by the conjugate determinant so that det U = 1 to rounding;
  numpy PCG64 seeded with 1701, drawn in mu-major, lexicographic order;
* sources: i.i.d. N(0,1) real and imaginary parts on the sites of one parity,
  seed 426 + k for the k-th source;
* shifts: log-spaced between 1e-5 and 1e2 (15 values for the 15-shift runs).

Canonical layouts: links ``[4][V][3][3]`` complex128 (U_mu(x)[row][col] at
lexicographic index ``x0 + N0 (x1 + N1 (x2 + N2 x3))``); half-lattice fields
``[Vh][3]`` complex128 in the paper's half index order (Eq. lexicographic_eo).
"""
from __future__ import annotations

import numpy as np

LINK_SEED = 1701
SOURCE_SEED = 426
ARRIVAL_SEED = 7
_CHUNK = 1 << 18  # matrices drawn per block (fixed so streams never depend on it)


def volume(dims) -> int:
    return int(np.prod([int(d) for d in dims]))


def check_dims(dims) -> tuple[int, int, int, int]:
    d = tuple(int(v) for v in dims)
    if len(d) != 4 or any(v < 2 or v % 2 for v in d):
        raise ValueError(f"lattice sides must be 4 even integers >= 2, got {dims}")
    return d


def _orthonormal_su3(g: np.ndarray) -> np.ndarray:
    """Gram-Schmidt (two passes, for orthogonality at rounding level) on the
    rows of each 3x3 block, then the last row rescaled so that det U = 1."""
    def proj(u, v):
        return np.sum(np.conj(u) * v, axis=1, keepdims=True) * u

    def unit(v):
        return v / np.linalg.norm(v, axis=1, keepdims=True)

    r0 = unit(g[:, 0, :])
    r1 = g[:, 1, :]
    for _ in range(2):
        r1 = r1 - proj(r0, r1)
    r1 = unit(r1)
    r2 = g[:, 2, :]
    for _ in range(2):
        r2 = r2 - proj(r0, r2) - proj(r1, r2)
    r2 = unit(r2)
    u = np.stack([r0, r1, r2], axis=1)
    det = np.linalg.det(u)
    u[:, 2, :] *= np.conj(det / np.abs(det))[:, None]
    return u


def random_su3(n: int, rng: np.random.Generator) -> np.ndarray:
    """n random SU(3) matrices, complex128 (n, 3, 3)."""
    out = np.empty((n, 3, 3), np.complex128)
    for s in range(0, n, _CHUNK):
        e = min(n, s + _CHUNK)
        g = rng.standard_normal((e - s, 3, 3, 2))
        out[s:e] = _orthonormal_su3(g[..., 0] + 1j * g[..., 1])
    return out


def random_links(dims, seed: int = LINK_SEED) -> np.ndarray:
    """Hot SU(3) gauge field, canonical layout [4][V][3][3] complex128."""
    V = volume(check_dims(dims))
    rng = np.random.default_rng(seed)
    return random_su3(4 * V, rng).reshape(4, V, 3, 3)


def unit_links(dims) -> np.ndarray:
    """Free field U = 1."""
    V = volume(check_dims(dims))
    u = np.zeros((4, V, 3, 3), np.complex128)
    u[..., 0, 0] = u[..., 1, 1] = u[..., 2, 2] = 1.0
    return u


def gaussian_field(dims, k: int = 0, n: int | None = None) -> np.ndarray:
    """Gaussian complex field on the sites of one parity, [Vh][3] complex128.

    ``k`` selects the source seed 426 + k.  ``n`` overrides the number of
    sites (used for multi-right-hand-side batches)."""
    Vh = volume(check_dims(dims)) // 2 if n is None else int(n)
    rng = np.random.default_rng(SOURCE_SEED + int(k))
    g = rng.standard_normal((Vh, 3, 2))
    return np.ascontiguousarray(g[..., 0] + 1j * g[..., 1])


def random_gauge_transform(dims, seed: int) -> np.ndarray:
    """One random SU(3) matrix per site, [V][3][3] complex128."""
    V = volume(check_dims(dims))
    return random_su3(V, np.random.default_rng(seed))


MOM_SEED = 2017


def random_momenta(dims, seed: int = MOM_SEED) -> np.ndarray:
    """Hermitian traceless 3x3 matrices, one per link, [4][V][3][3] complex128,
    with density proportional to exp(-(1/2) Tr H^2): real Gaussian diagonal
    pairs and complex off-diagonal entries of variance 1/2 per part, the
    diagonal made traceless."""
    V = volume(check_dims(dims))
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((4, V, 3, 3)) + 1j * rng.standard_normal((4, V, 3, 3))) / np.sqrt(2.0)
    h = 0.5 * (a + np.conj(np.swapaxes(a, -1, -2)))
    tr = np.trace(h, axis1=-2, axis2=-1) / 3.0
    return h - tr[..., None, None] * np.eye(3)


def log_shifts(n: int = 15, lo: float = 1e-5, hi: float = 1e2) -> np.ndarray:
    """n shifts log-spaced from lo to hi, ascending."""
    if n == 1:
        return np.array([lo], np.float64)
    return np.logspace(np.log10(lo), np.log10(hi), n)


def poisson_arrivals(rate_hz: float, n: int, seed: int = ARRIVAL_SEED) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_hz, size=n))
