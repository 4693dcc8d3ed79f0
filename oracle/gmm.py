"""Solar-disk and sky-brightness detection by a Gaussian mixture on the histogram.

Sec. 4.1: the dirty image is divided into 2000 brightness ranges; a Gaussian mixture
is fitted to the histogram; the mean of curve (a) is the sky brightness mu_a and the
mean of curve (b) the solar-disk brightness mu_b (Alg. 1 pre_clean, first step).

Readings (A11): K = 3 components (sky, disk, active region); bins equal on
[min D, max D] with the last bin closed; EM weighted by the bin counts, started from
the count-CDF quantiles {0.25, 0.85, 0.995}, variances var/3 (var of the histogram),
equal weights; variance floor (bin width)^2; stop when |dlogL| < 1e-12 |logL| or after
1000 iterations; components sorted by mean: mu_a the lowest, mu_b the second.  A
component with weight < 1e-4 marks the fit as degenerate.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

QUANTILES = (0.25, 0.85, 0.995)


def histogram(D, bins: int = 2000):
    """Counts h_b and bin centres x_b of ``bins`` equal ranges on [min, max].

    Bin index = floor((v - min) * (bins / (max - min))), the maximum falling in the
    last bin.  Returns (h, x, lo, width).
    """
    D = np.asarray(D, float).ravel()
    lo, hi = D.min(), D.max()
    width = (hi - lo) / bins
    if width == 0:
        h = np.zeros(bins)
        h[0] = D.size
        return h, lo + (np.arange(bins) + 0.5) * width, lo, width
    idx = np.floor((D - lo) * (bins / (hi - lo))).astype(np.int64)
    idx = np.clip(idx, 0, bins - 1)
    h = np.bincount(idx, minlength=bins).astype(float)
    x = lo + (np.arange(bins) + 0.5) * width
    return h, x, lo, width


def em(h, x, width, K: int = 3, max_iter: int = 1000, tol: float = 1e-12):
    """Weighted EM for a K-component 1-D Gaussian mixture on histogram (x_b, h_b).

    E step: r_bk = pi_k N(x_b | mu_k, var_k) / sum_j pi_j N(x_b | mu_j, var_j), evaluated
            from log densities relative to the largest one so that bins far from every
            component keep their responsibilities instead of underflowing to 0/0;
            logL = sum_b h_b log sum_k pi_k N(x_b | mu_k, var_k) for the current parameters.
    M step: n_k = sum_b h_b r_bk; mu_k = sum_b h_b r_bk x_b / n_k;
            var_k = max(sum_b h_b r_bk (x_b - mu_k)^2 / n_k, width^2) with the new mu_k;
            pi_k = n_k / sum h.
    Returns (mu, var, pi, n_iter, logL), components in ascending order of mean.
    """
    total = h.sum()
    cdf = np.cumsum(h) / total
    mu = np.array([x[np.searchsorted(cdf, q)] for q in QUANTILES[:K]], float)
    mean = (h * x).sum() / total
    var0 = (h * (x - mean) ** 2).sum() / total
    var = np.full(K, max(var0 / 3.0, width ** 2))
    pi = np.full(K, 1.0 / K)
    floor = width ** 2
    logL_old = None
    it = 0
    logL = 0.0
    for it in range(1, max_iter + 1):
        with np.errstate(divide="ignore"):
            lp = np.log(pi)[None, :] - 0.5 * (x[:, None] - mu[None, :]) ** 2 / var[None, :] \
                - 0.5 * np.log(2 * math.pi * var)[None, :]
        m = lp.max(1)
        e = np.exp(lp - m[:, None])
        s = e.sum(1)
        logL = float((h * (m + np.log(s))).sum())
        r = e / s[:, None]
        nk = (h[:, None] * r).sum(0)
        nk_safe = np.where(nk > 0, nk, 1.0)
        mu = np.where(nk > 0, (h[:, None] * r * x[:, None]).sum(0) / nk_safe, mu)
        var = np.where(nk > 0, (h[:, None] * r * (x[:, None] - mu[None, :]) ** 2).sum(0) / nk_safe, var)
        var = np.maximum(var, floor)
        pi = nk / total
        if logL_old is not None and abs(logL - logL_old) < tol * abs(logL):
            break
        logL_old = logL
    order = np.argsort(mu, kind="stable")
    return mu[order], var[order], pi[order], it, logL


def sky_and_disk(D, bins: int = 2000):
    """(mu_a, mu_b, degenerate) for one dirty image (Sec. 4.1, Alg. 1 pre_clean)."""
    h, x, lo, width = histogram(D, bins)
    if width == 0:
        return lo, lo, True
    mu, var, pi, _, _ = em(h, x, width)
    return float(mu[0]), float(mu[1]), bool((pi < 1e-4).any())
