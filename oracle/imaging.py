"""Gridding, inverse FFT, dirty map and dirty beam; direct-DFT definition (FP64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

from .pswf import Spheroidal


def uniform_weights(rec, G: int, N: int):
    """Uniform weights 1 / cnt for one instance's records (Alg. 1 weighting mode 1).

    Reading A4: cnt is the number of samples (each kept visibility and its mirror)
    that fall in the same cell of the unpadded N x N grid, cell size G/N uv cells.
    The N-grid cell of a sample is decided in FP32, in this order:
      t = float32(k - G/2) - f;  g_N = t / (G/N) + N/2;  cell = floor(g_N + 1/2)
    with f the FP32 offset, and the mirror sample's cell is N - cell.
    """
    keep = rec["w"] > 0
    r = np.float32(G // N)

    def cell(k, f):
        t = np.float32(k - G // 2).astype(np.float32) - np.asarray(f, np.float32)
        gN = (t / r).astype(np.float32) + np.float32(N // 2)
        return np.floor(gN.astype(np.float32) + np.float32(0.5)).astype(np.int64)

    cu = cell(rec["ku"][keep], rec["fu"][keep])
    cv = cell(rec["kv"][keep], rec["fv"][keep])
    keys = np.concatenate([cv * N + cu, (N - cv) * N + (N - cu)])
    uniq, counts = np.unique(keys, return_counts=True)
    cnt = dict(zip(uniq.tolist(), counts.tolist()))
    w = np.zeros(len(rec["w"]))
    w[np.nonzero(keep)[0]] = [1.0 / cnt[int(k)] for k in (cv * N + cu)]
    return w


def grid(rec, G: int, ker: Spheroidal, weights=None):
    """uv grid Z [G, G] complex128 (row = v cell, column = u cell).

    Sec. 3.2.3 / Alg. 1 ("calculating the weight and gridding"): each visibility,
    multiplied by its weight w, is convolved with the kernel C and accumulated:
        Z[kv+tv, ku+tu]         += w C(tu+fu) C(tv+fv) (V + i)
        Z[G-kv-tv, G-ku-tu]     += w C(tu+fu) C(tv+fv) (conj(V) + i)
    for tu, tv in -h..h.  The real part carries the Hermitian-symmetric visibility
    grid (its transform is the dirty map) and the imaginary part the Hermitian
    sampling grid (its transform is the dirty beam): one complex transform yields both.
    """
    h = (ker.W - 1) // 2
    w = rec["w"] if weights is None else weights
    keep = np.nonzero(rec["w"] > 0)[0]
    Z = np.zeros((G, G), np.complex128)
    taps = np.arange(-h, h + 1)
    for i in keep:
        cu = ker.kernel(taps + rec["fu"][i])
        cv = ker.kernel(taps + rec["fv"][i])
        wk = w[i] * np.outer(cv, cu)
        ku, kv, V = rec["ku"][i], rec["kv"][i], rec["vis"][i]
        Z[kv - h:kv + h + 1, ku - h:ku + h + 1] += wk * (V + 1j)
        rows = G - kv - taps
        cols = G - ku - taps
        Z[np.ix_(rows, cols)] += wk * (np.conj(V) + 1j)
    return Z


def centred_inverse_dft2(Z):
    """I(y, x) = sum_k Z[kv, ku] exp(+2 pi i ((ku - G/2)(x - G/2) + (kv - G/2)(y - G/2)) / G).

    Alg. 1 "invert fast Fourier transform ... with the sun disk at the center":
    the unnormalised inverse DFT with both origins at the grid centre.
    """
    G = Z.shape[0]
    return G * G * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(Z)))


def dirty_and_beam(Z, N: int, ker: Spheroidal):
    """Dirty map D [N, N] and dirty beam Bm [2N, 2N] from the grid (Alg. 1 dirty_image).

    D  = Re I / (gc(x) gc(y)) over the central N x N,
    Bm = Im I / (gc(x) gc(y)) over the central 2N x 2N (Sec. 3.2.1: the beam must be
    twice the image so a point can be subtracted anywhere), both divided by the beam
    centre value so that Bm(N, N) = 1 (reading A8).  Returns (D, Bm, norm) with norm the
    raw beam centre (0 when nothing was gridded; D and Bm are then zero).
    """
    G = Z.shape[0]
    I = centred_inverse_dft2(Z)
    gc = ker.grid_correction(G)
    corr = np.outer(gc, gc)
    lo_d, lo_b = G // 2 - N // 2, G // 2 - N
    D = (I.real / corr)[lo_d:lo_d + N, lo_d:lo_d + N]
    Bm = (I.imag / corr)[lo_b:lo_b + 2 * N, lo_b:lo_b + 2 * N]
    norm = Bm[N, N]
    if norm == 0:
        return np.zeros_like(D), np.zeros_like(Bm), 0.0
    return D / norm, Bm / norm, norm


def direct_dirty(rec, N: int, cell: float, weights=None):
    """The result gridding approximates: direct Fourier sums over the visibilities.

    D_dft(l, m)  = sum_k w_k Re[V_k exp(+2 pi i (u_k l + v_k m))] / sum_k w_k,
    Bm_dft(l, m) = sum_k w_k cos(2 pi (u_k l + v_k m)) / sum_k w_k,
    with l = (x - N/2) cell, m = (y - N/2) cell; the beam over 2N x 2N around (N, N).
    Plain loops over pixels: for tiny cases only.
    """
    w = rec["w"] if weights is None else weights
    keep = rec["w"] > 0
    u = rec["uvw"][keep, 0]
    v = rec["uvw"][keep, 1]
    V = rec["vis"][keep]
    wk = w[keep]
    sw = wk.sum()
    l = (np.arange(N) - N // 2) * cell
    D = np.empty((N, N))
    for y in range(N):
        ph = np.exp(2j * math.pi * (np.outer(l, u) + (l[y] * v)[None, :]))
        D[y] = (ph * (wk * V)[None, :]).real.sum(1) / sw
    lb = (np.arange(2 * N) - N) * cell
    Bm = np.empty((2 * N, 2 * N))
    for y in range(2 * N):
        Bm[y] = (np.cos(2 * math.pi * (np.outer(lb, u) + (lb[y] * v)[None, :])) * wk[None, :]).sum(1) / sw
    return D, Bm


def grid_cells(rec, G: int, ker: Spheroidal, weights=None):
    """The non-zero cells of `grid` as (kv, ku, value) arrays: the same taps and values, kept
    sparse so that grids too large to hold densely (G up to 20480) can be evaluated."""
    h = (ker.W - 1) // 2
    w = rec["w"] if weights is None else weights
    keep = np.nonzero(rec["w"] > 0)[0]
    taps = np.arange(-h, h + 1)
    kvs, kus, vals = [], [], []
    for i in keep:
        wk = w[i] * np.outer(ker.kernel(taps + rec["fv"][i]), ker.kernel(taps + rec["fu"][i]))
        ku, kv, V = rec["ku"][i], rec["kv"][i], rec["vis"][i]
        rr, cc = np.meshgrid(kv + taps, ku + taps, indexing="ij")
        kvs += [rr.ravel(), (G - rr).ravel()]
        kus += [cc.ravel(), (G - cc).ravel()]
        vals += [(wk * (V + 1j)).ravel(), (wk * (np.conj(V) + 1j)).ravel()]
    if not kvs:
        return np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0, np.complex128)
    kv, ku, val = np.concatenate(kvs), np.concatenate(kus), np.concatenate(vals)
    key, inv = np.unique(kv * G + ku, return_inverse=True)
    acc = np.zeros(len(key), np.complex128)
    np.add.at(acc, inv, val)
    return key // G, key % G, acc


def dirty_and_beam_at(rec, G: int, N: int, ker: Spheroidal, dirty_px, beam_px):
    """Selected pixels of `dirty_and_beam`, each the centred inverse DFT of the sparse grid at
    one point: dirty_px [n, 2] (y, x) of the N x N map, beam_px [m, 2] of the 2N x 2N beam.
    Returns (D values, Bm values, norm)."""
    kv, ku, val = grid_cells(rec, G, ker)
    gc = ker.grid_correction(G)
    norm = val.imag.sum() / gc[G // 2] ** 2     # Im I at the grid centre: every phase factor is 1

    def at(y, x):
        ph = np.exp(2j * math.pi * ((ku - G // 2) * (x - G // 2) + (kv - G // 2) * (y - G // 2)) / G)
        return (val * ph).sum() / (gc[x] * gc[y])

    lo_d, lo_b = G // 2 - N // 2, G // 2 - N
    D = np.array([at(lo_d + y, lo_d + x).real for y, x in np.asarray(dirty_px).reshape(-1, 2)])
    Bm = np.array([at(lo_b + y, lo_b + x).imag for y, x in np.asarray(beam_px).reshape(-1, 2)])
    if norm == 0:
        return np.zeros_like(D), np.zeros_like(Bm), 0.0
    return D / norm, Bm / norm, norm
