"""Clean beam and restored image (Alg. 1: dirty_image returns the clean beam too).

Reading C9: the clean beam is the elliptical Gaussian whose half-maximum ellipse has
the second moments of the dirty beam's main lobe.  The main lobe is the 4-connected
region of beam pixels >= 1/2 that contains the beam centre.  Each lobe pixel counts as
a unit square, so the moment matrix is the mean of (dx^2, dx dy, dy^2) over the lobe
pixels (offsets from the beam centre, pixels) plus 1/12 on the diagonal.  A uniform
ellipse {q' A q <= 1} has second moment A^-1 / 4 and a Gaussian's half-maximum ellipse
is q' Sigma^-1 q <= 2 ln 2, hence Sigma = (2 / ln 2) M.  The restored image is the
residual plus every component convolved with exp(-q' Sigma^-1 q / 2).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math
from collections import deque

import numpy as np


def main_lobe(Bm):
    """Boolean mask of the 4-connected region with Bm >= 0.5 containing the centre."""
    M2 = Bm.shape[0]
    c = M2 // 2
    mask = np.zeros(Bm.shape, bool)
    if not Bm[c, c] >= 0.5:
        return mask
    q = deque([(c, c)])
    mask[c, c] = True
    while q:
        y, x = q.popleft()
        for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            yy, xx = y + dy, x + dx
            if 0 <= yy < M2 and 0 <= xx < M2 and not mask[yy, xx] and Bm[yy, xx] >= 0.5:
                mask[yy, xx] = True
                q.append((yy, xx))
    return mask


def clean_beam(Bm):
    """Covariance (Sxx, Sxy, Syy) in pixel^2 of the clean beam fitted to Bm."""
    mask = main_lobe(Bm)
    c = Bm.shape[0] // 2
    ys, xs = np.nonzero(mask)
    dx, dy = xs - c, ys - c
    n = len(xs)
    mxx = (dx * dx).sum() / n + 1.0 / 12.0
    mxy = (dx * dy).sum() / n
    myy = (dy * dy).sum() / n + 1.0 / 12.0
    k = 2.0 / math.log(2.0)
    return k * mxx, k * mxy, k * myy


def gaussian(S, dx, dy):
    """exp(-q' S^-1 q / 2) at offsets (dx, dy)."""
    sxx, sxy, syy = S
    det = sxx * syy - sxy * sxy
    ixx, ixy, iyy = syy / det, -sxy / det, sxx / det
    return np.exp(-0.5 * (ixx * dx * dx + 2 * ixy * dx * dy + iyy * dy * dy))


def restore(R, pos, flux, S):
    """Restored image R + sum_c f_c CB(q - p_c) with the untruncated Gaussian."""
    N = R.shape[0]
    out = np.array(R, dtype=np.float64, copy=True)
    yy, xx = np.mgrid[0:N, 0:N]
    agg = {}
    for p, f in zip(pos, flux):
        agg[int(p)] = agg.get(int(p), 0.0) + float(f)
    for p, f in agg.items():
        py, px = divmod(p, N)
        out += f * gaussian(S, xx - px, yy - py)
    return out
