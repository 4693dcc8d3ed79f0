"""Prolate spheroidal gridding kernel, its oversampled table and the grid correction.

Sec. 3.2.3 selects the truncated spheroidal function of Schwab (1984) as the gridding
convolution function.  Schwab's coefficient tables are not reproduced here; the kernel
is built from its definition instead:

  * psi0(c, eta) is the zeroth prolate spheroidal angular function (alpha = 0), the
    eigenfunction with the smallest eigenvalue of the prolate differential operator
    (1 - eta^2) psi'' - 2 eta psi' - c^2 eta^2 psi = -lambda psi on [-1, 1].
  * In the normalised even Legendre basis Pbar_k = sqrt((2k+1)/2) P_k (k = 0, 2, 4, ...)
    the operator is a symmetric tridiagonal matrix (DLMF 30.8):
        diag_k     = k(k+1) + c^2 (2k(k+1) - 1) / ((2k+3)(2k-1))
        off_{k,k+2} = c^2 (k+1)(k+2) / ((2k+3) sqrt((2k+1)(2k+5)))
    and psi0 = sum_k d_k Pbar_k with d the eigenvector of the smallest eigenvalue.
  * Kernel, support W cells, c = pi W / 2:  C(d) = psi0(c, 2d/W) / psi0(c, 0) for |d| <= W/2.
  * Because psi0 is an eigenfunction of the finite Fourier transform, the transform of
    C is proportional to psi0(c, 2 xi): the grid correction is
        gc(xi) = psi0(c, 2 xi) / psi0(c, 0),   xi = (x - G/2) / G.
  * Both paths use C through a table of OS samples per cell with linear interpolation.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import eigh_tridiagonal
from scipy.special import eval_legendre

N_TERMS = 40


def spheroidal_c(W: int) -> float:
    """Bandwidth parameter c = pi W / 2 (reading A7: alpha = 0, c from the support)."""
    return math.pi * W / 2.0


def legendre_coefficients(c: float, n_terms: int = N_TERMS):
    """Eigenvalue and coefficients d_k (normalised-Legendre basis, even k) of psi0."""
    k = 2.0 * np.arange(n_terms)
    diag = k * (k + 1) + c * c * (2 * k * (k + 1) - 1) / ((2 * k + 3) * (2 * k - 1))
    kk = k[:-1]
    off = c * c * (kk + 1) * (kk + 2) / ((2 * kk + 3) * np.sqrt((2 * kk + 1) * (2 * kk + 5)))
    vals, vecs = eigh_tridiagonal(diag, off)
    d = vecs[:, 0]
    if psi0_from(d, 0.0) < 0:
        d = -d
    return vals[0], d


def psi0_from(d, eta):
    """psi0(eta) = sum_k d_k sqrt((2k+1)/2) P_k(eta) over even k."""
    eta = np.asarray(eta, float)
    out = np.zeros_like(eta)
    for i, dk in enumerate(d):
        k = 2 * i
        out = out + dk * math.sqrt((2 * k + 1) / 2.0) * eval_legendre(k, eta)
    return out


class Spheroidal:
    """The W-cell spheroidal kernel with OS samples per cell (Sec. 3.2.3)."""

    def __init__(self, W: int = 7, OS: int = 1024):
        self.W, self.OS = W, OS
        self.c = spheroidal_c(W)
        self.eigenvalue, self.d = legendre_coefficients(self.c)
        self.psi00 = float(psi0_from(self.d, 0.0))
        n = int(math.floor(W / 2 * OS)) + 2
        j = np.arange(n)
        dist = j / OS
        tab = self.psi(2 * dist / W)
        tab[dist > W / 2] = 0.0
        self.table = tab                         # C(j / OS), j = 0 .. W/2*OS + 1

    def psi(self, eta):
        """psi0(c, eta) / psi0(c, 0)."""
        return psi0_from(self.d, eta) / self.psi00

    def kernel_exact(self, dist):
        """Untabulated C(d) (zero outside |d| <= W/2)."""
        dist = np.asarray(dist, float)
        return np.where(np.abs(dist) <= self.W / 2, self.psi(2 * dist / self.W), 0.0)

    def kernel(self, dist):
        """Tabulated C(d): linear interpolation between table samples at |d| * OS."""
        pos = np.abs(np.asarray(dist, float)) * self.OS
        i = np.floor(pos).astype(np.int64)
        t = pos - i
        inside = i <= len(self.table) - 2
        i = np.minimum(i, len(self.table) - 2)
        return np.where(inside, self.table[i] * (1 - t) + self.table[i + 1] * t, 0.0)

    def grid_correction(self, G: int):
        """gc(x) for x = 0 .. G-1: psi0(c, 2 (x - G/2) / G) / psi0(c, 0)."""
        x = np.arange(G)
        return self.psi(2.0 * (x - G / 2) / G)

    def integral(self):
        """K = integral of C over its support (Gauss-Legendre quadrature, 200 nodes)."""
        t, wq = np.polynomial.legendre.leggauss(200)
        half = self.W / 2
        return float(np.sum(wq * self.kernel_exact(t * half)) * half)
