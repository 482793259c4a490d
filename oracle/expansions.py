"""Reaction-component multipole expansion in the paper's own normalisation.

TEST INFRASTRUCTURE ONLY (part of the oracle).  Used to reproduce the ME
convergence example of Section 3.3 (after eq. lecoeffimage):

    u~^{ab}(r, r'_ab) = sum_{n<=p} sum_{|m|<=n} M_nm F~^{ab}_nm(r, r_c)

with M_nm = c_n^{-2} r_c^n conj(Y_n^m(theta_c, phi_c))  (eq. melayerupgoingimage)
and F~ in terms of I_nm (eq. coefintable):
    F~^{1b}_nm = c_n e^{i m phi_s} I^{1b}_nm(rho_s, z - z_c) / (4 pi)
    F~^{2b}_nm = (-1)^{n+m} c_n e^{i m phi_s} I^{2b}_nm(rho_s, z_c - z) / (4 pi)
Y_n^m is the paper's spherical harmonic (eq. sphericalharmonics), built here
from scipy's associated Legendre function.
"""
from __future__ import annotations

from math import factorial, pi, sqrt

import numpy as np
from scipy.special import lpmv

from . import sommerfeld_K


def c_n(n: int) -> float:
    return sqrt((2 * n + 1) / (4 * pi))


def Phat(n: int, m: int, x: float) -> float:
    """Normalised associated Legendre function of eq. sphericalharmonics."""
    if m < 0:
        return (-1) ** (-m) * Phat(n, -m, x)
    return (-1) ** m * sqrt((2 * n + 1) / (4 * pi) * factorial(n - m) / factorial(n + m)) * lpmv(m, n, x)


def Y(n: int, m: int, theta: float, phi: float) -> complex:
    return Phat(n, m, np.cos(theta)) * np.exp(1j * m * phi)


def _sph(v):
    r = float(np.linalg.norm(v))
    return r, float(np.arccos(v[2] / r)) if r > 0 else 0.0, float(np.arctan2(v[1], v[0]))


def I_nm(d, eps, l, lp, a, b, n, m, rho, z, sigma_one=False):
    """I_nm of eq. uniformintegral (normalised by sqrt((n+m)!(n-m)!))."""
    mm = abs(m)
    K = sommerfeld_K(d, eps, l, lp, a, b, n, mm, rho, z, sigma_one=sigma_one, tol=1e-14)
    val = K / sqrt(factorial(n + mm) * factorial(n - mm))
    return val * ((-1) ** mm if m < 0 else 1)


def reaction_me(d, eps, l, lp, a, b, r, rp_ab, rc, p):
    """Truncated ME of u~^{ab}_{l lp}(r, r'_ab) about the centre rc, order p."""
    rcv = np.asarray(rp_ab, float) - np.asarray(rc, float)
    rcr, thc, phc = _sph(rcv)
    dv = np.asarray(r, float) - np.asarray(rc, float)
    rho_s = float(np.hypot(dv[0], dv[1]))
    phi_s = float(np.arctan2(dv[1], dv[0]))
    zz = dv[2] if a == 1 else -dv[2]
    total = 0.0 + 0.0j
    for n in range(p + 1):
        for m in range(-n, n + 1):
            M = rcr ** n * np.conj(Y(n, m, thc, phc)) / c_n(n) ** 2
            F = c_n(n) * np.exp(1j * m * phi_s) * I_nm(d, eps, l, lp, a, b, n, m, rho_s, zz) / (4 * pi)
            if a == 2:
                F *= (-1) ** (n + m)
            total += M * F
    return total


def reaction_exact(d, eps, l, lp, a, b, r, rp_ab):
    """u~^{ab}(r, r'_ab) = I_00(rho, |z - z'_ab|) / (4 pi) (eq. reactfieldpolarization)."""
    dv = np.asarray(r, float) - np.asarray(rp_ab, float)
    rho = float(np.hypot(dv[0], dv[1]))
    return sommerfeld_K(d, eps, l, lp, a, b, 0, 0, rho, abs(dv[2]), tol=1e-14) / (4 * pi)
