"""One instance of the imaging hot path end to end (Alg. 1 improved_clean without the
w-term step): records -> grid -> dirty map/beam -> [GMM threshold] -> Hogbom -> restore.

Test infrastructure only (see the package docstring).
"""
from __future__ import annotations

import numpy as np

from . import clean, geometry, gmm, imaging, restore
from .pswf import Spheroidal

_KERNELS = {}


def spheroidal(W=7, OS=1024):
    key = (W, OS)
    if key not in _KERNELS:
        _KERNELS[key] = Spheroidal(W, OS)
    return _KERNELS[key]


def cell_sizes(wl):
    return geometry.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)


def records(wl, dlm=None, frames=None):
    """Grid records of every instance of a workload (optionally a subset of frames)."""
    fr = slice(None) if frames is None else frames
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha[fr], wl.dec[fr], wl.freq)
    return geometry.grid_records(uvw, wl.vis[fr], wl.flags[fr], cell_sizes(wl), wl.G, wl.W, dlm)


def dirty(rec_i, N, G, ker, weight_mode=0):
    w = imaging.uniform_weights(rec_i, G, N) if weight_mode == 1 else None
    Z = imaging.grid(rec_i, G, ker, w)
    D, Bm, norm = imaging.dirty_and_beam(Z, N, ker)
    return Z, D, Bm, norm


def image_instance(rec_i, N, G, *, gain=0.1, cap=200, thr=-np.inf, thr_mode=0,
                   weight_mode=0, peak_mode=0, W=7, OS=1024):
    """Everything the GPU's muser_image computes for one instance, as a dict."""
    ker = spheroidal(W, OS)
    Z, D, Bm, norm = dirty(rec_i, N, G, ker, weight_mode)
    out = {"Z": Z, "D": D, "Bm": Bm, "norm": norm}
    if norm == 0:
        out.update(R=D.copy(), pos=np.zeros(0, np.int64), flux=np.zeros(0), S=(0.0, 0.0, 0.0),
                   clean=D.copy(), thr=thr, all_flagged=True)
        return out
    if thr_mode == 1:
        mu_a, mu_b, degenerate = gmm.sky_and_disk(D)
        thr = mu_a
        out.update(mu_a=mu_a, mu_b=mu_b, gmm_degenerate=degenerate)
    R, pos, flux = clean.hogbom(D, Bm, gain, thr, cap, peak_mode)
    S = restore.clean_beam(Bm)
    out.update(R=R, pos=pos, flux=flux, S=S, thr=thr, all_flagged=False,
               clean=restore.restore(R, pos, flux, S))
    return out
