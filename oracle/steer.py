"""Steer CLEAN (Steer, Dewdney & Ito 1984), major cycle by major cycle (FP64).

The paper's production deconvolution is the Steer clean (Sec. 3.2 and Alg. 1, "Steer clean";
Table 3 times one of its iterations); it states neither the selection level nor the scaling.
Reading (written out for both sides), per major cycle:

    m  = max R (the signed peak); stop when m <= thr, m <= 0 or after cap cycles;
    S  = {p : R(p) >= clip m}, the component map C = R on S and 0 elsewhere;
    Y  = the dirty beam convolved with C over the image, Y(q) = sum_p C(p) Bm(q - p + (N, N));
    a  = gain m / max_q Y(q)  (so that the largest value subtracted is gain times the peak);
    R -= a Y,  model += a C.

With clip = 1 the map holds the peak alone, Y = m Bm(q - p + (N, N)) peaks at m (the beam is 1
at its centre) and a = gain: the cycle is one Hogbom step.  D = R + Bm * model holds after
every cycle (the subtraction is linear in the map).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np


def convolve_beam(C, Bm):
    """Y(q) = sum_p C(p) Bm(q - p + (N, N)) for q in the N x N image (Bm is 2N x 2N).

    The circular convolution of side 2N of C (placed at the origin) with Bm equals Y shifted
    by (N, N): q - p + N stays within [1, 2N - 1], so nothing wraps.
    """
    N = C.shape[0]
    P = 2 * N
    Z = np.fft.ifft2(np.fft.fft2(C, (P, P)) * np.fft.fft2(Bm, (P, P))).real
    return Z[N:2 * N, N:2 * N]


def convolve_beam_bruteforce(C, Bm):
    N = C.shape[0]
    Y = np.zeros((N, N))
    for py, px in zip(*np.nonzero(C)):
        Y += C[py, px] * Bm[N - py:2 * N - py, N - px:2 * N - px]
    return Y


def steer(D, Bm, gain: float, thr: float, cap: int, clip: float = 0.9):
    """Returns (R, model, cycles)."""
    R = np.array(D, dtype=np.float64, copy=True)
    model = np.zeros_like(R)
    cycles = 0
    while cycles < cap:
        m = R.max()
        if m <= thr or m <= 0:
            break
        C = np.where(R >= clip * m, R, 0.0)
        Y = convolve_beam(C, Bm)
        ymax = Y.max()
        if ymax <= 0:
            break
        a = gain * m / ymax
        R -= a * Y
        model += a * C
        cycles += 1
    return R, model, cycles
