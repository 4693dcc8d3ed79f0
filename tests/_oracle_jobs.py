"""Oracle checks of one imaged instance, run in worker processes (spawned, so that they never
inherit a CUDA context) by the full-size parity tests.  Each job gets the oracle's records of
one instance and the GPU's outputs for it, recomputes the instance with the FP64 oracle and
asserts the parity tolerances; an AssertionError travels back to the test."""
from __future__ import annotations

import numpy as np

from oracle import gmm as ogmm
from oracle import pipeline, restore as orestore

from _parity import follow_oracle


def check_image_instance(job):
    """job: dict with rec (oracle records of the instance), N, G, gain, cap, thr_mode, and the
    GPU's pos, flux, n_comp, residual, clean (or None), beam_params (or None) and thr (the GPU's
    threshold).  The residual and the restored image are compared with the oracle's for the same
    component list (lockstep fluxes), which is defined whether or not a near tie made the lists
    part.  Returns a summary dict."""
    N, G, gain, cap = job["N"], job["G"], job["gain"], job["cap"]
    ker = pipeline.spheroidal(7, 1024)
    Z, D, Bm, norm = pipeline.dirty(job["rec"], N, G, ker)
    assert norm > 0
    out = {"inst": job.get("inst"), "peak0": float(np.abs(D).max())}
    thr = -np.inf
    if job["thr_mode"] == 1:
        mu_a, mu_b, _ = ogmm.sky_and_disk(D)
        rng = D.max() - D.min()
        assert abs(job["thr"] - mu_a) <= 1e-4 * rng, ("GMM sky level", job["thr"], mu_a)
        thr = float(job["thr"])          # the stop decision is checked against the level the GPU used
        out["mu_a"] = mu_a
    n = int(job["n_comp"])
    same, R, flux_o = follow_oracle(D, Bm, job["pos"], job["flux"], n, gain, cap, thr=thr)
    out["identical_steps"] = same
    out["n_comp"] = n
    peak0 = out["peak0"]
    # the GPU residual against the oracle residual of the same component list
    err = np.abs(job["residual"] - R).max()
    assert err <= 1e-4 * peak0, ("residual", err / peak0)
    out["residual_err"] = float(err / peak0)
    if job.get("beam_params") is not None:
        S = orestore.clean_beam(Bm)
        np.testing.assert_allclose(job["beam_params"], S, rtol=1e-5)
        if job.get("clean") is not None:
            # the oracle's restored image of the GPU's components with the lockstep fluxes
            I_o = orestore.restore(R, np.asarray(job["pos"][:n]), flux_o, S)
            err = np.abs(job["clean"] - I_o).max()
            assert err <= 1e-4 * np.abs(I_o).max(), ("restored image", err / np.abs(I_o).max())
            out["clean_err"] = float(err / np.abs(I_o).max())
    return out
