"""Zeroth-order prolate spheroidal wave function psi_0(c, x) on [-1, 1] (oracle, FP64).

Tab. AWP-CFSETUP (Sec. 6) names the anti-aliasing Prolate Spheroidal term of the
convolution function.  The paper gives no formula; the function used is the
angular prolate spheroidal function of order 0, the ground state of

    d/dx[(1 - x^2) dpsi/dx] - c^2 x^2 psi = -chi psi,   x in [-1, 1].

Expanding psi = sum_n b_n Pbar_n(x) in orthonormal Legendre functions
Pbar_n = sqrt((2n+1)/2) P_n, and using -d/dx[(1-x^2) P_n'] = n(n+1) P_n together
with the three-term form of x^2 P_n, gives a symmetric tridiagonal eigenproblem
in the even coefficients b_0, b_2, b_4, ...:

    B[n, n]   = n(n+1) + c^2 (2n(n+1) - 1) / ((2n+3)(2n-1))
    B[n, n+2] = c^2 (n+1)(n+2) / ((2n+3) sqrt((2n+1)(2n+5)))

psi_0 is the eigenvector of the smallest eigenvalue chi_0.  A library routine
(LAPACK via scipy) does the eigen-decomposition.  The tests pin the result with the
integral equation that psi_0 also satisfies, int_{-1}^{1} exp(i c x t) psi_0(t) dt
= mu psi_0(x), evaluated by Gauss-Legendre quadrature.
"""
from __future__ import annotations

import functools
import math

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy.linalg import eigh_tridiagonal


def bouwkamp_matrix(c: float, n_terms: int):
    """Diagonal and off-diagonal of the even-order Legendre matrix B (see module docstring)."""
    n = 2 * np.arange(n_terms, dtype=np.float64)
    c2 = c * c
    diag = n * (n + 1.0) + c2 * (2.0 * n * (n + 1.0) - 1.0) / ((2.0 * n + 3.0) * (2.0 * n - 1.0))
    nn = n[:-1]
    off = c2 * (nn + 1.0) * (nn + 2.0) / ((2.0 * nn + 3.0) * np.sqrt((2.0 * nn + 1.0) * (2.0 * nn + 5.0)))
    return diag, off


@functools.lru_cache(maxsize=64)
def legendre_coeffs(c: float, n_terms: int = 60):
    """(chi_0, coefficients a_n of psi_0 = sum a_n P_n) with psi_0(0) > 0 and unit L2 norm."""
    diag, off = bouwkamp_matrix(c, n_terms)
    w, v = eigh_tridiagonal(diag, off, select="i", select_range=(0, 0))
    b = v[:, 0]
    n = 2 * np.arange(n_terms)
    a = np.zeros(2 * n_terms - 1)
    a[n] = b * np.sqrt((2.0 * n + 1.0) / 2.0)      # Pbar_n -> P_n
    if npleg.legval(0.0, a) < 0:
        a = -a
    return float(w[0]), a


def psi0(c: float, x) -> np.ndarray:
    """psi_0(c, x) for |x| <= 1 (unit L2 norm on [-1, 1], positive at 0)."""
    _, a = legendre_coeffs(float(c))
    return npleg.legval(np.asarray(x, dtype=np.float64), a)


def pswf_c(ps_support: int) -> float:
    """Bandwidth parameter for a kernel of width W pixels: c = pi W / 2.

    With c = pi W / 2 the uv kernel psi_0(2u/W), |u| <= W/2, and the image-plane
    taper psi_0(2x/N) over the N-pixel field are a Fourier pair (Sec. 6 PS term).
    """
    return math.pi * ps_support / 2.0


def taper(ps_support: int, x_over_half_fov) -> np.ndarray:
    """Image-plane taper T = psi_0(c, x) / psi_0(c, 0), x in units of the half field of view."""
    c = pswf_c(ps_support)
    return psi0(c, x_over_half_fov) / psi0(c, 0.0)
