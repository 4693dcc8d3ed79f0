"""muser_dirty_noalloc (no workspace, library-owned static scratch) against muser_dirty.

The no-allocation entry point exists for callers that cannot allocate device memory
(memory owned by another allocator or a fixed budget, or code that must not call
cudaMalloc/cudaFree because they synchronise the device).  It must give the same dirty
maps and beams as the workspace version, also on a second call that reuses the scratch
left over from the first, up to the largest batch its static scratch holds; one instance
more is refused.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

SCRATCH = (16 << 20) + (64 << 10)        # MUSER_NOALLOC_SCRATCH_BYTES


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


def _grids(m, N, n_frame, cfg_id):
    import torch
    wl = synth.small_workload(n_ant=10, N=N, n_frame=n_frame, config_id=cfg_id, bmax=500.0)
    cfg = m.Config(N=wl.N, G=wl.G, lat_rad=wl.lat)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    rec, _, st = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    off = torch.arange(wl.n_inst + 1, dtype=torch.int64, device="cuda") * wl.n_bl
    Z, st = m.grid(rec, off, cfg, status=st)
    return cfg, Z


def _largest_batch(m, cfg):
    B = 0
    while m.workspace_size(m.CALL_DIRTY, B + 1, 0, cfg) <= SCRATCH:
        B += 1
    return B


def test_noalloc_matches_workspace_version_on_two_calls():
    import torch
    import paper_1712_06913_b300 as m
    results = []
    for cfg_id in (401, 402):            # two different batches, back to back
        cfg, Z = _grids(m, 128, 2, cfg_id)
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


@pytest.mark.parametrize("N,expect", [(256, 4), (320, 2), (512, 1)])
def test_noalloc_largest_batch_accepted_and_one_more_refused(N, expect):
    """At the capacity boundary: the largest batch whose muser_dirty workspace fits the static
    scratch (four 256^2, two 320^2, one 512^2 instances) gives muser_dirty's maps and beams on two
    calls in a row; one instance more is refused with MUSER_ERR_ARG before any device work."""
    import torch
    import paper_1712_06913_b300 as m
    cfg0 = m.Config(N=N, G=4 * N)
    Bmax = _largest_batch(m, cfg0)
    assert Bmax == expect
    cfg, Z = _grids(m, N, Bmax + 1, 410 + N)
    D_ref, B_ref, _ = m.dirty(Z[:Bmax].contiguous(), cfg)
    for _ in range(2):
        rc, D, Bm, st = _noalloc(m, Z[:Bmax].contiguous(), cfg)
        assert rc == m._lib.MUSER_OK, m._lib.load().muser_last_error()
        torch.cuda.synchronize()
        assert float((D - D_ref).abs().max()) <= 1e-6 * float(D_ref.abs().max())
        assert float((Bm - B_ref).abs().max()) <= 1e-6
        assert int(st.max()) == 0
    rc, _, _, _ = _noalloc(m, Z, cfg)
    assert rc == m._lib.MUSER_ERR_ARG
    assert b"scratch" in m._lib.load().muser_last_error()


def test_noalloc_refuses_what_muser_dirty_refuses():
    """The configuration checks are muser_dirty's: a non-zero reserved field, a bad peak mode or an
    image side muser_dirty rejects are refused; N = 1024 needs more scratch than the array holds."""
    import torch
    import paper_1712_06913_b300 as m
    lib = m._lib.load()
    Z = torch.zeros((1, 8, 8), dtype=torch.complex64, device="cuda")   # never read: refused first
    dummy = torch.zeros(4, device="cuda")
    for cfg in (m.Config(N=1024, G=4096), m.Config(N=128, G=512, peak_mode=3), m.Config(N=100, G=400)):
        c = cfg.c()
        rc = lib.muser_dirty_noalloc(ctypes.c_void_p(Z.data_ptr()), 1, ctypes.byref(c),
                                     ctypes.c_void_p(dummy.data_ptr()), ctypes.c_void_p(dummy.data_ptr()), None, None)
        assert rc == m._lib.MUSER_ERR_ARG
    c = m.Config(N=128, G=512).c()
    c.reserved[0] = 1
    rc = lib.muser_dirty_noalloc(ctypes.c_void_p(Z.data_ptr()), 1, ctypes.byref(c), ctypes.c_void_p(dummy.data_ptr()),
                                 ctypes.c_void_p(dummy.data_ptr()), None, None)
    assert rc == m._lib.MUSER_ERR_ARG and b"reserved" in lib.muser_last_error()
