"""Shared helpers of the GPU parity tests: run both sides on one seeded workload.

The oracle side only ever sees synth inputs; the GPU side only the same synth inputs.
"""
from __future__ import annotations

import math

import numpy as np

import synth
from oracle import clean as oclean
from oracle import geometry, pipeline

KER = pipeline.spheroidal(7, 1024)


def cfg_for(m, wl, max_iter=None, thr_mode=None, batch_chunk=0):
    return m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=wl.max_iter if max_iter is None else max_iter,
                    gain=wl.gain, thr_mode=wl.thr_mode if thr_mode is None else thr_mode, lat_rad=wl.lat,
                    batch_chunk=batch_chunk)


def gpu_records(m, wl, cfg, want_uvw=True, dlm=None):
    import torch
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    rec, uvw, st = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags, dlm=dlm,
                         want_uvw=want_uvw)
    off = torch.arange(wl.n_inst + 1, dtype=torch.int64, device="cuda") * wl.n_bl
    return rec, uvw, st, off, cell


def oracle_records(wl, dlm=None):
    return pipeline.records(wl, dlm=dlm)


def assert_no_ties(rec_o, G, W, eps=1e-9):
    """The GPU and the oracle decide cells in FP64 with different operation orders; no kept
    sample of the oracle may sit within eps of a rounding or grid-edge decision."""
    for g in (rec_o["gu"], rec_o["gv"]):
        frac = (g + 0.5) - np.floor(g + 0.5)
        near = np.minimum(frac, 1 - frac) < eps
        assert not near.any(), "seeded input has a near-tie cell decision"


def lockstep(D_o, Bm_o, pos_g, flux_g, gain, peak_mode=0, tol_pos=1e-5, tol_flux=1e-4):
    """Replay the GPU component list on the oracle residual (FP64).

    At each step the GPU's position must be an exact or near-tie argmax of the oracle
    residual (within tol_pos * peak0) and its flux within tol_flux * peak0 of gain * R[p].
    Returns the number of steps whose position differs from the oracle's own argmax.
    """
    N = D_o.shape[0]
    R = np.array(D_o, dtype=np.float64, copy=True)
    peak0 = np.abs(R).max()
    diffs = 0
    for p, f in zip(pos_g, flux_g):
        key = R if peak_mode == 0 else np.abs(R)
        best = key.max()
        p = int(p)
        assert key.ravel()[p] >= best - tol_pos * peak0, ("not a near-argmax", p, key.ravel()[p], best)
        fo = gain * R.ravel()[p]
        assert abs(f - fo) <= tol_flux * peak0, ("flux", f, fo)
        if int(np.argmax(key)) != p:
            diffs += 1
        py, px = divmod(p, N)
        R -= fo * Bm_o[N - py:2 * N - py, N - px:2 * N - px]
    return diffs


def identical_positions_unless_near_tie(D_o, Bm_o, pos_g, gain, cap, thr=-np.inf, peak_mode=0, tie=1e-5):
    """The GPU list equals the oracle's free-running list up to the first step where the
    oracle's top-2 gap is within tie * peak0 (a genuine near-tie)."""
    R_o, pos_o, _ = oclean.hogbom(D_o, Bm_o, gain, thr, cap, peak_mode)
    peak0 = np.abs(D_o).max()
    R = np.array(D_o, dtype=np.float64, copy=True)
    N = D_o.shape[0]
    for j, (pg, po) in enumerate(zip(pos_g, pos_o)):
        if int(pg) != int(po):
            key = (R if peak_mode == 0 else np.abs(R)).ravel()
            top = np.sort(key)[-2:]
            assert top[1] - top[0] <= tie * peak0, ("positions differ without a near tie", j, pg, po)
            return j
        py, px = divmod(int(po), N)
        R -= gain * R.ravel()[int(po)] * Bm_o[N - py:2 * N - py, N - px:2 * N - px]
    return len(pos_o)
