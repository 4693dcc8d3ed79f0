"""Solar-disk centring correction (Sec. 4.2, Alg. 1 pre_clean / improved_clean).

Steps, in the paper's order:
 1. deconvolve the dirty image until its peak is at most the disk brightness mu_b
    (Hogbom, cap 1000), so only the disk and the sky background remain;
 2. pick the bright points (h_dirty).  Reading A12: after step 1 no pixel exceeds mu_b,
    so the literal selection R > mu_b is empty; the points kept are those with
    R > (mu_a + mu_b) / 2, halfway between the sky and the disk brightness, with their
    brightness (a binary mask correlates to a flat-topped peak that hides the offset);
 3. correlate them with a simulated uniform disk (radius 16', centred) over integer
    shifts |s| <= N/4; the best shift (ties: smallest |s|, then lowest row-major index),
    refined per axis by a 3-point parabola (reading A13), is the disk offset;
 4. the offset (dl, dm) = s * pixel gives RA offset dl / cos(dec) and DEC offset dm; the
    visibilities are phase-corrected by exp(+2 pi i (u dl + v dm)) and re-imaged.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .clean import hogbom


def disk_model(N, radius_px):
    """Uniform disk of the given radius (pixels) centred on (N/2, N/2)."""
    yy, xx = np.mgrid[0:N, 0:N]
    return ((xx - N // 2) ** 2 + (yy - N // 2) ** 2 <= radius_px ** 2).astype(float)


def correlation(M, S, smax):
    """Cc(s) = sum_p M(p) S(p - s) for integer shifts |s_x|, |s_y| <= smax.

    Computed with zero-padded FFTs; ``correlation_bruteforce`` is the plain sum.
    Returned as [2 smax + 1, 2 smax + 1] indexed by (s_y + smax, s_x + smax).
    """
    N = M.shape[0]
    P = 2 * N
    FM = np.fft.fft2(M, (P, P))
    FS = np.fft.fft2(S, (P, P))
    c = np.fft.ifft2(FM * np.conj(FS)).real        # c[s] = sum_p M(p) S(p - s), s mod P
    idx = np.arange(-smax, smax + 1) % P
    return c[np.ix_(idx, idx)]


def correlation_bruteforce(M, S, smax):
    N = M.shape[0]
    out = np.zeros((2 * smax + 1, 2 * smax + 1))
    for sy in range(-smax, smax + 1):
        for sx in range(-smax, smax + 1):
            Ss = np.zeros_like(S)
            ys = slice(max(0, sy), min(N, N + sy))
            xs = slice(max(0, sx), min(N, N + sx))
            yd = slice(max(0, -sy), min(N, N - sy))
            xd = slice(max(0, -sx), min(N, N - sx))
            Ss[ys, xs] = S[yd, xd]                  # Ss(p) = S(p - s)
            out[sy + smax, sx + smax] = (M * Ss).sum()
    return out


def best_shift(Cc, smax):
    """argmax with ties to the smallest |s|, then the lowest row-major index; plus a
    3-point parabolic refinement per axis.  Returns (sx, sy) in pixels (float)."""
    best = Cc.max()
    cand = np.argwhere(Cc == best)
    d2 = ((cand - smax) ** 2).sum(1)
    cand = cand[d2 == d2.min()]
    iy, ix = cand[0]

    def parabola(cm, c0, cp):
        den = cm - 2 * c0 + cp
        if den >= 0:
            return 0.0
        return float(np.clip(0.5 * (cm - cp) / den, -0.5, 0.5))

    n = Cc.shape[0]
    dx = parabola(Cc[iy, ix - 1], Cc[iy, ix], Cc[iy, ix + 1]) if 0 < ix < n - 1 else 0.0
    dy = parabola(Cc[iy - 1, ix], Cc[iy, ix], Cc[iy + 1, ix]) if 0 < iy < n - 1 else 0.0
    return ix - smax + dx, iy - smax + dy


def disk_offset(D, Bm, mu_a, mu_b, cell, dec, gain=0.1, cap=1000, sun_radius=16 * math.pi / 180 / 60):
    """(dl, dm, ra_offset, dec_offset, mask) for one dirty image (Sec. 4.2 steps 1-3)."""
    N = D.shape[0]
    R, _, _ = hogbom(D, Bm, gain, mu_b, cap)
    M = np.where(R > 0.5 * (mu_a + mu_b), R, 0.0)
    S = disk_model(N, sun_radius / cell)
    smax = N // 4
    sx, sy = best_shift(correlation(M, S, smax), smax)
    dl, dm = sx * cell, sy * cell
    return dl, dm, dl / math.cos(dec), dm, M
