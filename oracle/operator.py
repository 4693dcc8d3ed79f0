"""Degridding measurement operator, its adjoint and the chi-square gradient (FP64).

The paper grids measured visibilities onto a uv grid and inverts the FFT
(Sec. 3.2.3, Alg. 1 dirty_image).  The measurement operator here is the transpose of
that pipeline, for gradient-based imaging of a real sky image x [N, N]:

  A x = (1/K^2) Interp( F( Pad_G( x / (gc gc) ) ) )
    Pad_G  -- place the N x N image at the centre of a G x G array (G = 2N, sigma = 2);
    F      -- centred forward DFT, X[k] = sum_p x[p] exp(-2 pi i (k - G/2).(p - G/2) / G);
    Interp -- V_k = sum_taps C(tu + fu) C(tv + fv) X[kv + tv, ku + tu]  (same kernel, W taps);
    gc     -- the grid correction of the same kernel;  K = integral of C, so the
              separable 2-D kernel C(du) C(dv) integrates to K^2.
  A approximates the direct transform V(u, v) = sum_p x[p] exp(-2 pi i (u l_p + v m_p)).

  A^H y = (1/K^2) (1 / (gc gc)) Crop_N( F^H( Grid(y) ) ), F^H the centred inverse DFT
  (unnormalised), Grid the transpose of Interp.

  chi2(x) = sum_k w_k |(A x)_k - V_k|^2 / sigma^2,  grad = 2 Re A^H (w (A x - V)) / sigma^2.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .pswf import Spheroidal


def _taps(ker):
    h = (ker.W - 1) // 2
    return np.arange(-h, h + 1), h


def _pad_slice(N, G):
    lo = G // 2 - N // 2
    return slice(lo, lo + N)


def apodisation(N, G, ker):
    gc = ker.grid_correction(G)[_pad_slice(N, G)]
    return np.outer(gc, gc)


def forward(x, rec, N, G, ker: Spheroidal, K=None):
    """A x for every record (zero for records with w = 0)."""
    K = ker.integral() if K is None else K
    xp = np.zeros((G, G), np.complex128)
    s = _pad_slice(N, G)
    xp[s, s] = np.asarray(x, float) / apodisation(N, G, ker)
    X = np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(xp)))
    taps, h = _taps(ker)
    out = np.zeros(len(rec["w"]), np.complex128)
    for i in np.nonzero(rec["w"] > 0)[0]:
        cu = ker.kernel(taps + rec["fu"][i])
        cv = ker.kernel(taps + rec["fv"][i])
        ku, kv = rec["ku"][i], rec["kv"][i]
        out[i] = (np.outer(cv, cu) * X[kv - h:kv + h + 1, ku - h:ku + h + 1]).sum() / K ** 2
    return out


def adjoint(y, rec, N, G, ker: Spheroidal, K=None):
    """A^H y (complex N x N)."""
    K = ker.integral() if K is None else K
    taps, h = _taps(ker)
    Z = np.zeros((G, G), np.complex128)
    for i in np.nonzero(rec["w"] > 0)[0]:
        cu = ker.kernel(taps + rec["fu"][i])
        cv = ker.kernel(taps + rec["fv"][i])
        ku, kv = rec["ku"][i], rec["kv"][i]
        Z[kv - h:kv + h + 1, ku - h:ku + h + 1] += np.outer(cv, cu) * y[i]
    I = G * G * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(Z)))
    s = _pad_slice(N, G)
    return I[s, s] / apodisation(N, G, ker) / K ** 2


def direct(x, rec, N, cell):
    """Direct transform V(u, v) = sum_p x[p] exp(-2 pi i (u l + v m)) (tiny cases)."""
    l = (np.arange(N) - N // 2) * cell
    out = np.zeros(len(rec["w"]), np.complex128)
    keep = np.nonzero(rec["w"] > 0)[0]
    u = rec["uvw"][keep, 0]
    v = rec["uvw"][keep, 1]
    for j, (uu, vv) in enumerate(zip(u, v)):
        ph = np.exp(-2j * math.pi * (vv * l[:, None] + uu * l[None, :]))
        out[keep[j]] = (x * ph).sum()
    return out


def chi2_grad(x, rec, V, sigma, N, G, ker, K=None):
    """(chi2, grad) of chi2(x) = sum_k w_k |A x - V|^2 / sigma^2."""
    w = rec["w"]
    d = forward(x, rec, N, G, ker, K) - V
    chi2 = float((w * np.abs(d) ** 2).sum() / sigma ** 2)
    grad = 2.0 * adjoint(w * d, rec, N, G, ker, K).real / sigma ** 2
    return chi2, grad


def lipschitz(rec, N, G, ker, sigma, iters=20, seed=0, K=None):
    """Largest eigenvalue of the chi2 Hessian 2 Re(A^H W A)/sigma^2 by power iteration."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((N, N))
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = 2.0 * adjoint(forward(x, rec, N, G, ker, K) * rec["w"], rec, N, G, ker, K).real / sigma ** 2
        lam = float(np.linalg.norm(y))
        x = y / lam
    return lam


def gradient_descent(rec, V, sigma, N, G, ker, steps=100, K=None, L=None):
    """x_{t+1} = x_t - grad chi2(x_t) / L from x_0 = 0.  Returns (x, chi2 history)."""
    K = ker.integral() if K is None else K
    L = lipschitz(rec, N, G, ker, sigma, K=K) if L is None else L
    x = np.zeros((N, N))
    hist = []
    for _ in range(steps):
        c, g = chi2_grad(x, rec, V, sigma, N, G, ker, K)
        hist.append(c)
        x = x - g / L
    return x, np.asarray(hist)
