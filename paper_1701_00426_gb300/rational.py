"""Partial-fraction coefficients for the rational function of the RHMC.

The RHMC replaces a root of the fermion matrix (Eq. rooting) by a rational
function r(x) = a0 + sum_i a_i / (x + sigma_i) with real poles sigma_i
(Sec. 2.2, Eq. shlineq); ``lqcd_rational_apply`` evaluates r(A) b on the
device.  Production runs bring coefficients from an offline Remez
computation; this module gives a closed-form set for the inverse square root
that tests and benchmarks use, from the integral representation

    x^(-1/2) = (2 / pi) * integral_0^inf dt / (t^2 + x)

with t = s tan(theta) and Gauss-Legendre quadrature in theta on [0, pi/2):
a node theta_k with weight w_k (on [-1, 1]) gives the pole
sigma_k = s^2 tan^2(theta_k) and the residue a_k = (w_k / 2) s sec^2(theta_k).
The rule is exact at x = s^2; s = (lam_min lam_max)^(1/4) centres it on the
spectrum in the logarithmic sense.  Host-side helper, not part of the device
path.
"""
from __future__ import annotations

import numpy as np


def inverse_sqrt_poles(n: int, lam_min: float, lam_max: float):
    """(a0, a[n], sigma[n]) with a0 + sum a_i / (x + sigma_i) ~ x^(-1/2) on [lam_min, lam_max]."""
    if n < 1 or not (0.0 < lam_min <= lam_max):
        raise ValueError("need n >= 1 and 0 < lam_min <= lam_max")
    s = (lam_min * lam_max) ** 0.25
    xi, w = np.polynomial.legendre.leggauss(n)
    theta = 0.25 * np.pi * (xi + 1.0)
    sigma = (s * np.tan(theta)) ** 2
    a = 0.5 * w * s / np.cos(theta) ** 2
    order = np.argsort(sigma)
    return 0.0, a[order], sigma[order]


def evaluate(a0: float, a, sigma, x):
    """r(x) = a0 + sum_i a_i / (x + sigma_i) for an array of x."""
    x = np.asarray(x, dtype=np.float64)[..., None]
    return a0 + np.sum(np.asarray(a) / (x + np.asarray(sigma)), axis=-1)


def max_rel_error(a0: float, a, sigma, lam_min: float, lam_max: float, power: float = -0.5, points: int = 4001):
    """max over a logarithmic grid of |r(x) - x^power| / x^power on [lam_min, lam_max]."""
    x = np.geomspace(lam_min, lam_max, points)
    return float(np.max(np.abs(evaluate(a0, a, sigma, x) / x ** power - 1.0)))
