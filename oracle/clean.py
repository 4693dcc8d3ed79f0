"""Hogbom CLEAN with the sky-brightness stopping rule (FP64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def peak(R, peak_mode: int = 0):
    """Strength and position of the peak (Alg. 1 "find the strength and position").

    peak_mode 0: the largest signed value; 1: the largest absolute value (reading A2).
    Ties go to the lowest row-major index (reading A3).
    """
    flat = R.ravel()
    p = int(np.argmax(flat if peak_mode == 0 else np.abs(flat)))
    return flat[p], p


def hogbom(D, Bm, gain: float, thr: float, cap: int, peak_mode: int = 0):
    """Hogbom (1974) CLEAN as used in the loop of Alg. 1 (improved_clean).

    it = 0; find the peak p of R = D.  While R[p] > thr (|R[p]| for peak_mode 1) and
    it < cap: record the component (p, f = gain * R[p]); subtract f times the dirty beam
    centred on p, R[q] -= f Bm[q - p + (N, N)] for every q of the N x N image; it += 1;
    find the peak again.  Sec. 4.3: gain 0.1, thr = the GMM sky brightness mu_a (or a
    fixed threshold with an iteration cap).  Returns (R, pos[n], flux[n]).
    """
    R = np.array(D, dtype=np.float64, copy=True)
    N = R.shape[0]
    pos, flux = [], []
    val, p = peak(R, peak_mode)
    while (val if peak_mode == 0 else abs(val)) > thr and len(pos) < cap:
        f = gain * val
        py, px = divmod(p, N)
        R -= f * Bm[N - py:2 * N - py, N - px:2 * N - px]
        pos.append(p)
        flux.append(f)
        val, p = peak(R, peak_mode)
    return R, np.asarray(pos, np.int64), np.asarray(flux, float)


def replay(D, Bm, pos, flux):
    """Apply a given component list to D (no peak search): R after each subtraction.

    Used by the lockstep comparison: yields (R before the step, p, f) per component.
    """
    R = np.array(D, dtype=np.float64, copy=True)
    N = R.shape[0]
    for p, f in zip(pos, flux):
        yield R, int(p), float(f)
        py, px = divmod(int(p), N)
        R = R - f * Bm[N - py:2 * N - py, N - px:2 * N - px]
