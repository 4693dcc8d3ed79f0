"""W-projection: the w-term correction of dirty_image (Alg. 1; Sec. 3.2 and Sec. 6.1 give the
phase-error criterion |pi (l^2 + m^2) w| << 1 and cite the GPU w-projection of Muscat 2014;
the method is Cornwell, Golap & Bhatnagar 2008), FP64.

Definition followed (the direct transform with the w-term, which w-projection approximates):
    D_w(l, m)  = sum_k wt_k Re[V_k exp(+2 pi i (u_k l + v_k m + w_k (n - 1)))] / sum_k wt_k,
    Bm_w(l, m) = sum_k wt_k cos(2 pi (u_k l + v_k m + w_k (n - 1))) / sum_k wt_k,
    n = sqrt(1 - l^2 - m^2).

Reading (the paper gives no kernel construction):
  * Paraxial w-term: 2 pi w (n - 1) ~ -pi w (l^2 + m^2).  For a solar field (|l|, |m| <= 1 deg)
    and |w| <= 3000 wavelengths the neglected 2 pi |w| (l^2 + m^2)^2 / 8 stays below 3e-4 rad.
    The image-plane screen then factors, s(l, m) = exp(-i pi w l^2) exp(-i pi w m^2), and so
    does the kernel.
  * Grid units: with xi = l / (G cell) in [-1/2, 1/2) the screen is exp(-i pi wg xi^2) with
    wg = w (G cell)^2, so one set of kernels serves every channel whatever its pixel size.
  * Kernel of plane p (wg_p = p wg_max / (P - 1), p = 0 .. P - 1), tap offset d in cells:
        k_p(d) = int gc(xi) exp(-i pi wg_p xi^2) exp(-2 pi i d xi) dxi / int gc(xi) dxi
    over xi in [-1/2, 1/2] (Gauss-Legendre, 256 nodes), gc the spheroidal grid correction.
    Its image-plane transform is gc times the screen; k_0 is the spheroidal kernel C up to the
    spheroidal's aliasing (pinned).  Even in d; tabulated at OS samples per cell for
    |d| <= Ww / 2 and read with linear interpolation, like C.
  * A sample (u, v, w) takes plane p = min(P - 1, round(|wg| / dwg)) and kernel
    K = k_p(tu + fu) k_p(tv + fv), conjugated when w < 0 (a mirrored w);
        Z[kv + tv, ku + tu]         += wt K (V + i)
        Z[G - kv - tv, G - ku - tu] += wt conj(K) (conj(V) + i)
    for tu, tv in -hw .. hw, hw = (Ww - 1) / 2.  Both parts of Z stay Hermitian, so the dirty map
    and beam follow from the transform exactly as without w (imaging.dirty_and_beam).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .pswf import Spheroidal

GL_NODES = 256


def kernel_tables(wg_max: float, P: int, Ww: int, OS: int, ker: Spheroidal):
    """[P, n] complex128 tables k_p(j / OS), j = 0 .. n - 1, n = floor(Ww / 2 OS) + 2."""
    t, wq = np.polynomial.legendre.leggauss(GL_NODES)
    xi = 0.5 * t
    g = 0.5 * wq * ker.psi(2.0 * xi)              # quadrature weight times gc(xi)
    n = int(math.floor(Ww / 2 * OS)) + 2
    d = np.arange(n) / OS
    dwg = wg_max / (P - 1) if P > 1 else 0.0
    E = np.exp(-2j * math.pi * np.outer(xi, d))                        # [nodes, n]
    screens = g[None, :] * np.exp(-1j * math.pi * (np.arange(P) * dwg)[:, None] * (xi * xi)[None, :])
    tabs = screens @ E / g.sum()
    tabs[:, d > Ww / 2] = 0.0
    return tabs


def lookup(tab, OS: int, dist):
    """Linear interpolation in a table of OS samples per cell, |dist| (even kernel)."""
    pos = np.abs(np.asarray(dist, float)) * OS
    i = np.floor(pos).astype(np.int64)
    t = pos - i
    inside = i <= len(tab) - 2
    i = np.minimum(i, len(tab) - 2)
    return np.where(inside, tab[i] * (1 - t) + tab[i + 1] * t, 0.0)


def plane_of(wg, wg_max: float, P: int):
    dwg = wg_max / (P - 1) if P > 1 else 1.0
    return np.minimum(P - 1, np.floor(np.abs(wg) / dwg + 0.5)).astype(np.int64)


def grid(rec, G: int, tabs, wg_max: float, Ww: int, OS: int):
    """The w-projected uv grid Z [G, G] complex128 (record fields as geometry.grid_records,
    plus "wg")."""
    P = tabs.shape[0]
    h = (Ww - 1) // 2
    taps = np.arange(-h, h + 1)
    Z = np.zeros((G, G), np.complex128)
    for i in np.nonzero(rec["w"] > 0)[0]:
        p = int(plane_of(rec["wg"][i], wg_max, P))
        tab = tabs[p] if rec["wg"][i] >= 0 else np.conj(tabs[p])
        K = rec["w"][i] * np.outer(lookup(tab, OS, taps + rec["fv"][i]), lookup(tab, OS, taps + rec["fu"][i]))
        ku, kv, V = rec["ku"][i], rec["kv"][i], rec["vis"][i]
        Z[kv - h:kv + h + 1, ku - h:ku + h + 1] += K * (V + 1j)
        Z[np.ix_(G - kv - taps, G - ku - taps)] += np.conj(K) * (np.conj(V) + 1j)
    return Z


def direct_dirty_w(rec, N: int, cell: float):
    """D_w over N x N and Bm_w over 2N x 2N by direct sums (exact n): tiny cases only."""
    keep = rec["w"] > 0
    u, v, w = rec["uvw"][keep, 0], rec["uvw"][keep, 1], rec["uvw"][keep, 2]
    V = rec["vis"][keep]
    wt = rec["w"][keep]
    sw = wt.sum()
    l = (np.arange(N) - N // 2) * cell
    D = np.empty((N, N))
    for y in range(N):
        n = np.sqrt(1 - l * l - l[y] ** 2)
        ph = np.exp(2j * math.pi * (np.outer(l, u) + (l[y] * v)[None, :] + np.outer(n - 1, w)))
        D[y] = (ph * (wt * V)[None, :]).real.sum(1) / sw
    lb = (np.arange(2 * N) - N) * cell
    Bm = np.empty((2 * N, 2 * N))
    for y in range(2 * N):
        n = np.sqrt(1 - lb * lb - lb[y] ** 2)
        Bm[y] = (np.cos(2 * math.pi * (np.outer(lb, u) + (lb[y] * v)[None, :] + np.outer(n - 1, w)))
                 * wt[None, :]).sum(1) / sw
    return D, Bm
