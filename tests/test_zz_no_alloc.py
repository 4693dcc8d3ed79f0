"""muser_dirty_noalloc (no workspace, library-owned static scratch) against muser_dirty.

The no-allocation entry point exists for callers that cannot allocate device memory
(memory owned by another allocator or a fixed budget, or code that must not call
cudaMalloc/cudaFree because they synchronise the device).  It must give the same dirty
maps and beams as the workspace version, also on a second call that reuses the scratch
left over from the first.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _noalloc(m, Z, cfg):
    import torch
    lib = m._lib.load()
    B = Z.shape[0]
    D = torch.empty((B, cfg.N, cfg.N), dtype=torch.float32, device="cuda")
    Bm = torch.empty((B, 2 * cfg.N, 2 * cfg.N), dtype=torch.float32, device="cuda")
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    c = cfg.c()
    rc = lib.muser_dirty_noalloc(ctypes.c_void_p(Z.data_ptr()), B, ctypes.byref(c), ctypes.c_void_p(D.data_ptr()),
                                 ctypes.c_void_p(Bm.data_ptr()), ctypes.c_void_p(st.data_ptr()),
                                 ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, D, Bm, st


def test_noalloc_matches_workspace_version_on_two_calls():
    import torch
    import paper_1712_06913_b300 as m
    results = []
    for cfg_id in (401, 402):            # two different batches, back to back
        wl = synth.small_workload(n_ant=10, N=128, n_frame=2, config_id=cfg_id, bmax=500.0)
        cfg = m.Config(N=wl.N, G=wl.G, lat_rad=wl.lat)
        cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
        rec, _, st = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
        off = torch.arange(wl.n_inst + 1, dtype=torch.int64, device="cuda") * wl.n_bl
        Z, st = m.grid(rec, off, cfg, status=st)
        D_ref, B_ref, _ = m.dirty(Z, cfg)
        rc, D, Bm, st2 = _noalloc(m, Z, cfg)
        assert rc == m._lib.MUSER_OK, m._lib.load().muser_last_error()
        results.append((D_ref, B_ref, D, Bm, st2))
    torch.cuda.synchronize()
    for D_ref, B_ref, D, Bm, st2 in results:
        peak = float(D_ref.abs().max())
        assert float((D - D_ref).abs().max()) <= 1e-6 * peak
        assert float((Bm - B_ref).abs().max()) <= 1e-6
        assert int(st2.max()) == 0


def test_noalloc_rejects_batches_beyond_the_static_scratch():
    import torch
    import paper_1712_06913_b300 as m
    cfg = m.Config(N=1024, G=4096)
    Z = torch.zeros((1, 8, 8), dtype=torch.complex64, device="cuda")   # never read: rejected first
    lib = m._lib.load()
    c = cfg.c()
    dummy = torch.zeros(4, device="cuda")
    rc = lib.muser_dirty_noalloc(ctypes.c_void_p(Z.data_ptr()), 1, ctypes.byref(c), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == m._lib.MUSER_ERR_ARG
    assert b"scratch" in lib.muser_last_error()
