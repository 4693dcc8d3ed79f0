"""Baseline geometry, pixel-size rule and per-visibility grid records (FP64).

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299_792_458.0


def local_xyz(ant_enu: np.ndarray, lat: float) -> np.ndarray:
    """Antenna positions in the local equatorial frame.

    Sec. 3.2.2 converts surveyed antenna positions to a terrestrial frame before the
    baseline vectors are formed.  With local east/north/up coordinates at latitude
    ``lat`` the textbook frame (Thompson, Moran & Swenson, Sec. 4.1) has X in the
    meridian plane on the celestial equator, Y to the east and Z to the pole:
    X = -sin(lat) N + cos(lat) U,  Y = E,  Z = cos(lat) N + sin(lat) U.
    """
    e, n, u = ant_enu[:, 0], ant_enu[:, 1], ant_enu[:, 2]
    sl, cl = math.sin(lat), math.cos(lat)
    return np.stack([-sl * n + cl * u, e, cl * n + sl * u], axis=-1)


def uvw(ant_enu, pairs, lat, ha, dec, freq) -> np.ndarray:
    """(u, v, w) in wavelengths for every (frame, channel, baseline): [F, C, n_bl, 3].

    Sec. 3.2.2 ("UVW calculation"): baseline b = X_j - X_i (i < j), rotated to the
    (u, v, w) frame of a phase centre at hour angle H and declination d
    (Thompson, Moran & Swenson, eq. 4.1):
        u = ( sin H bx + cos H by) / lambda
        v = (-sin d cos H bx + sin d sin H by + cos d bz) / lambda
        w = ( cos d cos H bx - cos d sin H by + sin d bz) / lambda
    with lambda = c / nu.
    """
    xyz = local_xyz(np.asarray(ant_enu, float), lat)
    pairs = np.asarray(pairs)
    b = xyz[pairs[:, 1]] - xyz[pairs[:, 0]]
    bx, by, bz = b[:, 0], b[:, 1], b[:, 2]
    F, C = len(ha), len(freq)
    out = np.empty((F, C, len(pairs), 3))
    for f in range(F):
        sH, cH = math.sin(ha[f]), math.cos(ha[f])
        sd, cd = math.sin(dec[f]), math.cos(dec[f])
        um = sH * bx + cH * by
        vm = -sd * cH * bx + sd * sH * by + cd * bz
        wm = cd * cH * bx - cd * sH * by + sd * bz
        for c in range(C):
            k = freq[c] / C_LIGHT
            out[f, c, :, 0] = um * k
            out[f, c, :, 1] = vm * k
            out[f, c, :, 2] = wm * k
    return out


def resolution(freq, bmax):
    """Spatial resolution lambda / B_max in radians (Table 1 and Table 2 first column)."""
    return C_LIGHT / np.asarray(freq, float) / bmax


def pixel_size(freq, bmax, N, fov_min):
    """Pixel size in radians for an N x N image.

    Sec. 3.2.1 / Table 2: three pixels per resolution element, pixel = (lambda/B_max)/3.
    Reading for fixed N (the rule alone would put the 16' solar disk outside a 256^2
    image at 1.7 GHz): the pixel is never smaller than fov_min / N, so the image always
    spans at least ``fov_min``.
    """
    return np.maximum(resolution(freq, bmax) / 3.0, fov_min / N)


def grid_records(uvw_fcb, vis, flags, cell, G, W, dlm=None):
    """Per-visibility grid records (Sec. 3.2.3 gridding set-up, Alg. 1 input).

    uvw_fcb: [F, C, nb, 3] wavelengths; vis: [F, C, nb] complex; flags: [F, C, nb];
    cell: [C] pixel size (rad); dlm: optional [F*C, 2] phase-centre shift (rad).

    The uv cell is du = 1 / (G * cell); a visibility falls at grid coordinate
    g = u / du + G / 2 (and likewise for v), nearest cell k = floor(g + 0.5) and
    offset f = k - g in [-1/2, 1/2].  The kernel taps are k - h .. k + h with
    h = (W - 1) / 2; the mirrored sample (-u, -v) uses the mirrored cells G - k.
    A visibility is kept only if every tap of both samples lies inside [0, G), i.e.
    h + 1 <= k <= G - h - 1 on both axes, it is not flagged and it is finite.
    The phase correction of Sec. 4.2 step 3 / Alg. 1 multiplies the visibility by
    exp(+2 pi i (u dl + v dm)), moving a source at (dl, dm) to the phase centre.

    Returns dict of arrays flattened over (frame, channel, baseline):
    ku, kv (int64, -1 when dropped), fu, fv, w (1 kept / 0 dropped), vis (complex128),
    g (the two grid coordinates, for near-tie checks), uvw, and wg = w (G cell)^2 (the w
    coordinate in grid units, which selects the w-projection plane; 0 when dropped).
    With w-projection W is the w-kernel support, so that its footprint stays on the grid.
    """
    F, C, nb, _ = uvw_fcb.shape
    h = (W - 1) // 2
    u = uvw_fcb[..., 0]
    v = uvw_fcb[..., 1]
    scale = G * np.asarray(cell, float)[None, :, None]
    gu = u * scale + G / 2
    gv = v * scale + G / 2
    ku = np.floor(gu + 0.5)
    kv = np.floor(gv + 0.5)
    V = vis.astype(np.complex128)
    if dlm is not None:
        d = np.asarray(dlm, float).reshape(F, C, 2)
        V = V * np.exp(2j * math.pi * (u * d[:, :, None, 0] + v * d[:, :, None, 1]))
    inside = (ku >= h + 1) & (ku <= G - h - 1) & (kv >= h + 1) & (kv <= G - h - 1)
    keep = inside & (np.asarray(flags) == 0) & np.isfinite(V)
    rec = {
        "ku": np.where(keep, ku, -1).astype(np.int64).ravel(),
        "kv": np.where(keep, kv, -1).astype(np.int64).ravel(),
        "fu": np.where(keep, ku - gu, 0.0).ravel(),
        "fv": np.where(keep, kv - gv, 0.0).ravel(),
        "w": keep.astype(np.float64).ravel(),
        "vis": np.where(keep, V, 0).ravel(),
        "gu": gu.ravel(), "gv": gv.ravel(),
        "uvw": uvw_fcb.reshape(-1, 3),
        "wg": np.where(keep, uvw_fcb[..., 2] * scale * np.asarray(cell, float)[None, :, None] * G, 0.0).ravel(),
    }
    return rec


def instance_slice(rec, i, nb):
    """Records of instance i (= frame * n_chan + chan) from ``grid_records`` output."""
    s = slice(i * nb, (i + 1) * nb)
    return {k: val[s] for k, val in rec.items()}
