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


def follow_oracle(D_o, Bm_o, pos_g, flux_g, n_g, gain, cap, thr=-np.inf, peak_mode=0, tol_pos=1e-5, tol_flux=1e-4,
                  tie=1e-5):
    """All CLEAN checks of a GPU component list against the FP64 oracle in one pass.

    Replays the GPU's n_g components on the oracle residual (lockstep).  At every step the GPU
    position must be an exact or near-tie argmax (within tol_pos * peak0) and its flux within
    tol_flux * peak0 of gain * R[p]; until the first step where the oracle's own argmax differs,
    the two lists are identical, and that step must be a genuine near tie (oracle top-2 gap
    within tie * peak0) -- from there on only the lockstep checks apply.  Stopping: the GPU may
    only continue while the oracle's peak is above thr - tol_flux * peak0, and it may stop before
    the cap only once the oracle's peak is at or below thr + tol_flux * peak0 (so the counts differ
    only when the oracle's final peak sits within that band of thr).

    Returns (first step whose position differs from the oracle's own, or n_g; R after the replay;
    the oracle's fluxes gain * R[p] of the replayed steps).
    """
    N = D_o.shape[0]
    R = np.array(D_o, dtype=np.float64, copy=True)
    flat = R.ravel()
    peak0 = np.abs(R).max()
    diverged = None
    flux_o = np.zeros(int(n_g))
    for j in range(int(n_g)):
        key = flat if peak_mode == 0 else np.abs(flat)
        po = int(np.argmax(key))
        best = key[po]
        p = int(pos_g[j])
        assert 0 <= p < N * N, ("position out of range", j, p)
        assert key[p] >= best - tol_pos * peak0, ("not a near-argmax", j, p, key[p], best)
        assert best > thr - tol_flux * peak0, ("continued below the threshold", j, best, thr)
        fo = gain * flat[p]
        flux_o[j] = fo
        assert abs(float(flux_g[j]) - fo) <= tol_flux * peak0, ("flux", j, float(flux_g[j]), fo)
        if diverged is None and p != po:
            top = np.partition(key, -2)[-2:]
            assert top[1] - top[0] <= tie * peak0, ("positions differ without a near tie", j, p, po)
            diverged = j
        py, px = divmod(p, N)
        R -= fo * Bm_o[N - py:2 * N - py, N - px:2 * N - px]
    if int(n_g) < cap:
        key = flat if peak_mode == 0 else np.abs(flat)
        assert key.max() <= thr + tol_flux * peak0, ("stopped above the threshold", int(n_g), key.max(), thr)
    return (int(n_g) if diverged is None else diverged), R, flux_o
