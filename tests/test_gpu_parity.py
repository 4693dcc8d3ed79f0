"""GPU (libmuser, sm_103a) versus the FP64 oracle, element by element, through the C ABI.

Tolerances (the FP32 path against FP64): records bit-exact in cell and weight,
offsets within 1e-6 cell; uv grid within 1e-5 of its peak; dirty map within 1e-4 of its
peak and dirty beam within 1e-4 over the full 2N x 2N; CLEAN positions identical unless
the oracle itself has a near-tie (top-2 gap <= 1e-5 peak), every position a near-argmax
of the oracle residual replayed in lockstep, fluxes within 1e-4 of the peak; GMM levels
within 1e-4 of the image range; restored image within 1e-4 of its peak; degridding and
gradient within 1e-4 relative L2.
"""
import math

import numpy as np
import pytest

import synth
from oracle import clean as oclean
from oracle import geometry, gmm as ogmm, imaging, operator as oop, pipeline, restore as orestore

from _parity import (KER, assert_no_ties, cfg_for, gpu_records, identical_positions_unless_near_tie, lockstep,
                     oracle_records)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def m():
    import torch
    import paper_1712_06913_b300 as mod
    torch.cuda.init()
    return mod


def _np(t):
    return t.detach().cpu().numpy()


WORKLOADS = {
    "small-N64": lambda: synth.small_workload(n_ant=10, N=64, config_id=201, bmax=300.0),
    "small-N32-3frames": lambda: synth.small_workload(n_ant=9, N=32, n_frame=3, freq=(1.2e9, 1.7e9),
                                                      config_id=202, bmax=150.0, flag_max=0.3),
    "plain-N256": synth.config1_plain_frame,
}


# ------------------------------------------------------------------------------ uvw
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_uvw_records(m, name):
    wl = WORKLOADS[name]()
    cfg = cfg_for(m, wl)
    rec, uvw, st, off, cell = gpu_records(m, wl, cfg)
    np.testing.assert_allclose(cell, pipeline.cell_sizes(wl), rtol=1e-15)
    ro = oracle_records(wl)
    assert_no_ties(ro, wl.G, wl.W)
    np.testing.assert_allclose(_np(uvw), ro["uvw"], rtol=1e-12, atol=1e-9)
    vis, fu, fv, ku, kv, w, wg = (_np(x) for x in m.record_fields(rec))
    np.testing.assert_array_equal(w, ro["w"])
    np.testing.assert_allclose(wg, ro["wg"], rtol=1e-6, atol=1e-6 * np.abs(ro["wg"]).max())
    np.testing.assert_array_equal(ku, ro["ku"])
    np.testing.assert_array_equal(kv, ro["kv"])
    keep = ro["w"] > 0
    assert np.abs(fu - ro["fu"])[keep].max() <= 1e-6
    assert np.abs(fv - ro["fv"])[keep].max() <= 1e-6
    np.testing.assert_allclose(vis[keep], ro["vis"][keep], rtol=0, atol=2e-6 * np.abs(ro["vis"]).max())


def test_uvw_phase_rotation(m):
    wl = synth.small_workload(n_ant=10, N=64, config_id=203, bmax=300.0)
    cfg = cfg_for(m, wl)
    dlm = np.array([[3.1e-4, -1.7e-4]])
    rec, _, _, _, _ = gpu_records(m, wl, cfg, dlm=dlm)
    ro = oracle_records(wl, dlm=dlm)
    vis = _np(m.record_fields(rec)[0])
    keep = ro["w"] > 0
    np.testing.assert_allclose(vis[keep], ro["vis"][keep], rtol=0, atol=2e-6 * np.abs(ro["vis"]).max())


# ------------------------------------------------------------------------------ grid + dirty
def _dirty_both(m, wl):
    cfg = cfg_for(m, wl)
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    Z, st = m.grid(rec, off, cfg, status=st)
    D, Bm, st = m.dirty(Z, cfg, status=st)
    ro = oracle_records(wl)
    out = []
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Zo = imaging.grid(ri, wl.G, KER)
        Do, Bo, norm = imaging.dirty_and_beam(Zo, wl.N, KER)
        out.append((Zo, Do, Bo, norm))
    return cfg, Z, D, Bm, st, out


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_grid_and_dirty(m, name):
    wl = WORKLOADS[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    Zg, Dg, Bg, stg = _np(Z), _np(D), _np(Bm), _np(st)
    for i, (Zo, Do, Bo, norm) in enumerate(ref):
        assert np.abs(Zg[i] - Zo).max() <= 1e-5 * np.abs(Zo).max()
        assert np.abs(Dg[i] - Do).max() <= 1e-4 * np.abs(Do).max(), i
        assert np.abs(Bg[i] - Bo).max() <= 1e-4, i
        assert abs(Bg[i][wl.N, wl.N] - 1.0) <= 1e-6
        assert (stg[i] & m.ST_ALL_FLAGGED) == 0


def test_grid_and_dirty_into_caller_buffers(m):
    """grid / dirty writing into caller tensors (a view of a larger buffer, poisoned first)
    give the same grids, maps and beams as freshly allocated outputs; bad buffers are refused."""
    import torch
    wl = WORKLOADS["small-N64"]()
    cfg = cfg_for(m, wl)
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    Z, st1 = m.grid(rec, off, cfg, status=st.clone())
    D, Bm, _ = m.dirty(Z, cfg, status=st1)
    B, N, G = wl.n_inst, wl.N, wl.G
    Zb = torch.full((B + 1, G, G), float("nan"), dtype=torch.complex64, device="cuda")
    Db = torch.full((B + 1, N, N), float("nan"), device="cuda")
    Bb = torch.full((B + 1, 2 * N, 2 * N), float("nan"), device="cuda")
    Z2, st2 = m.grid(rec, off, cfg, status=st.clone(), out=Zb[:B], n_vis=int(_np(off)[-1]))
    D2, B2, _ = m.dirty(Z2, cfg, status=st2, out=(Db[:B], Bb[:B]))
    assert Z2.data_ptr() == Zb.data_ptr() and D2.data_ptr() == Db.data_ptr()
    # shared-memory accumulation order may differ between calls: last-bit differences only
    for a, b in ((Z2, Z), (D2, D), (B2, Bm)):
        assert float((a - b).abs().max()) <= 1e-6 * float(b.abs().max())
    assert torch.isnan(Db[B]).all()                     # nothing written past the batch
    with pytest.raises(ValueError):
        m.grid(rec, off, cfg, out=Zb[:B, :, : G // 2])
    with pytest.raises(ValueError):
        m.dirty(Z, cfg, out=(Db[:B], Bb[:B, :N]))


@pytest.mark.parametrize("name", ["small-N64", "small-N32-3frames", "plain-N256"])
def test_uniform_weighting_grid_and_dirty(m, name):
    """weight_mode 1 (Alg. 1's uniform weighting): grids, maps and beams of muser_grid /
    muser_dirty against the oracle's 1 / (samples per N-grid cell) weights; the caller's
    records keep their weights (muser_grid weights a copy)."""
    import dataclasses
    wl = WORKLOADS[name]()
    cfg = dataclasses.replace(cfg_for(m, wl), weight_mode=1)
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    w_before = m.record_fields(rec)[5].clone()
    Z, st = m.grid(rec, off, cfg, status=st)
    D, Bm, st = m.dirty(Z, cfg, status=st)
    assert bool((m.record_fields(rec)[5] == w_before).all())
    ro = oracle_records(wl)
    Zg, Dg, Bg = _np(Z), _np(D), _np(Bm)
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Zo, Do, Bo, norm = pipeline.dirty(ri, wl.N, wl.G, KER, weight_mode=1)
        assert np.abs(Zg[i] - Zo).max() <= 1e-5 * np.abs(Zo).max(), i
        assert np.abs(Dg[i] - Do).max() <= 1e-4 * np.abs(Do).max(), i
        assert np.abs(Bg[i] - Bo).max() <= 1e-4, i
    # natural and uniform weighting give different beams (the weights did change)
    Zn, _ = m.grid(rec, off, dataclasses.replace(cfg, weight_mode=0))
    assert float((Zn - Z).abs().max()) > 1e-3 * float(Z.abs().max())


def test_uniform_weighting_image_end_to_end(m):
    """muser_image with weight_mode 1 on the plain frame: the CLEAN components in lockstep with
    the oracle's uniformly weighted dirty map and beam."""
    import dataclasses
    wl = synth.config1_plain_frame()
    cfg = dataclasses.replace(cfg_for(m, wl), weight_mode=1)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ro = oracle_records(wl)
    o = pipeline.image_instance(geometry.instance_slice(ro, 0, wl.n_bl), wl.N, wl.G, gain=wl.gain, cap=wl.max_iter,
                                weight_mode=1)
    assert int(_np(out.n_comp)[0]) == wl.max_iter
    lockstep(o["D"], o["Bm"], _np(out.comp_pos)[0], _np(out.comp_flux)[0], wl.gain)
    np.testing.assert_allclose(_np(out.beam_params)[0], o["S"], rtol=1e-4)


def test_dirty_full_size_instance(m):
    """One MUSER-II instance at the largest workload size (N = 1024, G = 4096)."""
    wl = synth.config3_muser2_uneven(n_frame=1, chans=[5, 300])
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    Dg, Bg = _np(D), _np(Bm)
    for i, (Zo, Do, Bo, norm) in enumerate(ref):
        assert np.abs(Dg[i] - Do).max() <= 1e-4 * np.abs(Do).max()
        assert np.abs(Bg[i] - Bo).max() <= 1e-4
        # the beam is even about (N, N) (both uv signs gridded): each side within 1e-4 of the
        # oracle's, whose mirror pairs agree to 1e-12
        A = Bg[i][1:, 1:]
        assert np.abs(A - A[::-1, ::-1]).max() <= 2e-4
        N = cfg.N
        assert np.unravel_index(np.argmax(Bg[i]), Bg[i].shape) == (N, N)


# ------------------------------------------------------------------------------ CLEAN
@pytest.mark.parametrize("name,cap", [("small-N64", 60), ("plain-N256", 200)])
def test_clean_lockstep(m, name, cap):
    wl = WORKLOADS[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    cfg.max_iter = cap
    R, pos, flux, nc, st = m.clean(D, Bm, cfg, status=st)
    Rg, pg, fg, ncg = _np(R), _np(pos), _np(flux), _np(nc)
    for i, (Zo, Do, Bo, _) in enumerate(ref):
        assert ncg[i] == cap
        lockstep(Do, Bo, pg[i], fg[i], cfg.gain)
        identical_positions_unless_near_tie(Do, Bo, pg[i], cfg.gain, cap)
        Ro, po, fo = oclean.hogbom(Do, Bo, cfg.gain, -np.inf, cap)
        if np.array_equal(po, pg[i]):
            assert np.abs(Rg[i] - Ro).max() <= 1e-4 * np.abs(Do).max()
            assert np.abs(fg[i] - fo).max() <= 1e-4 * np.abs(Do).max()


ONCHIP_CASES = {
    # 6 instances: clusters of 4 blocks with 16384-pixel bands; 40: one block per instance
    "N256x6": lambda: synth.small_workload(n_ant=31, N=256, n_frame=6, config_id=230, bmax=2000.0),
    "N256x40": lambda: synth.small_workload(n_ant=31, N=256, n_frame=40, config_id=231, bmax=2000.0),
    # 2 instances: clusters of 16 blocks with 16384-pixel bands; 12: clusters of 4
    "N512x2": lambda: synth.config2_muser1_band(n_frame=1, chans=[10, 50]),
    "N512x12": lambda: synth.config2_muser1_band(n_frame=1, chans=list(range(4, 64, 5))),
    "N1024x2": lambda: synth.config3_muser2_uneven(n_frame=1, chans=[7, 400]),
    # four beam copies up to B N^2 = 2^21 (the cases above), two beyond: 3 instances at 1024^2
    "N1024x3": lambda: synth.config3_muser2_uneven(n_frame=1, chans=[7, 200, 400]),
}


@pytest.mark.parametrize("name", list(ONCHIP_CASES))
def test_clean_onchip_equals_streaming_and_oracle(m, name):
    """The on-chip-residual kernel (clusters of 1/4/16 blocks) performs the same FP32
    operations as the streaming kernel: identical components; and both follow the oracle."""
    import torch
    wl = ONCHIP_CASES[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    cfg.max_iter, cfg.thr_mode = 150, 0
    R1, p1, f1, n1, _ = m.clean(D, Bm, cfg)
    cfg.clean_kernel = 1
    R2, p2, f2, n2, _ = m.clean(D, Bm, cfg)
    assert torch.equal(n1, n2) and torch.equal(p1, p2) and torch.equal(f1, f2)
    assert float((R1 - R2).abs().max()) == 0.0
    pg, fg = _np(p1), _np(f1)
    for i, (Zo, Do, Bo, _) in enumerate(ref):
        lockstep(Do, Bo, pg[i], fg[i], cfg.gain)
        identical_positions_unless_near_tie(Do, Bo, pg[i], cfg.gain, cfg.max_iter)


def test_clean_threshold_and_abs_mode(m):
    wl = WORKLOADS["small-N64"]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    Do, Bo = ref[0][1], ref[0][2]
    thr = 0.3 * np.abs(Do).max()
    cfg.max_iter = 500
    R, pos, flux, nc, _ = m.clean(D, Bm, cfg, thr=np.array([thr], np.float32))
    Ro, po, fo = oclean.hogbom(Do, Bo, cfg.gain, thr, 500)
    assert abs(int(_np(nc)[0]) - len(po)) <= 1
    cfg.peak_mode = 1
    R, pos, flux, nc, _ = m.clean(D, Bm, cfg)
    lockstep(Do, Bo, _np(pos)[0], _np(flux)[0], cfg.gain, peak_mode=1)


@pytest.mark.parametrize("name", ["N256x6", "N256x40", "N512x2", "N512x12", "N1024x2", "N1024x3"])
def test_clean_onchip_abs_peaks_equal_streaming_and_oracle(m, name):
    """The same on-chip shapes with the peak of |R| (peak_mode 1: keys |v|, the sign carried with
    the index): components identical to the streaming kernel's, both following the oracle."""
    import torch
    wl = ONCHIP_CASES[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    cfg.max_iter, cfg.thr_mode, cfg.peak_mode = 150, 0, 1
    R1, p1, f1, n1, _ = m.clean(D, Bm, cfg)
    cfg.clean_kernel = 1
    R2, p2, f2, n2, _ = m.clean(D, Bm, cfg)
    assert torch.equal(n1, n2) and torch.equal(p1, p2) and torch.equal(f1, f2)
    assert float((R1 - R2).abs().max()) == 0.0
    pg, fg = _np(p1), _np(f1)
    for i, (Zo, Do, Bo, _) in enumerate(ref):
        lockstep(Do, Bo, pg[i], fg[i], cfg.gain, peak_mode=1)
        identical_positions_unless_near_tie(Do, Bo, pg[i], cfg.gain, cfg.max_iter, peak_mode=1)


# ------------------------------------------------------------------------------ GMM
@pytest.mark.parametrize("name", ["small-N64", "plain-N256"])
def test_gmm(m, name):
    wl = WORKLOADS[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    mu_a, mu_b, _ = m.gmm(D, cfg)
    for i, (_, Do, _, _) in enumerate(ref):
        a, b, _ = ogmm.sky_and_disk(Do)
        rng = Do.max() - Do.min()
        assert abs(float(_np(mu_a)[i]) - a) <= 1e-4 * rng
        assert abs(float(_np(mu_b)[i]) - b) <= 1e-4 * rng


def test_gmm_degenerate_and_few_valued_maps(m):
    """A constant map has no histogram range: both levels are its value and the instance is marked
    GMM_DEGENERATE; a zero map with three bright pixels collapses the three components onto one
    level (no weight below 1e-4, so not marked); a two-valued noisy map splits cleanly.  Levels
    and marks as in the oracle on the same FP32 maps."""
    import torch
    N = 64
    rng = np.random.default_rng(5)
    maps = [np.full((N, N), 0.25), np.zeros((N, N)),
            np.where(rng.uniform(size=(N, N)) < 0.5, 0.0, 1.0) + 1e-3 * rng.normal(size=(N, N))]
    maps[1][5, 7], maps[1][9, 9], maps[1][30, 2] = 1.0, 0.5, -0.2
    maps = [d.astype(np.float32) for d in maps]
    D = torch.tensor(np.stack(maps), device="cuda")
    mu_a, mu_b, st = m.gmm(D, m.Config(N=N, G=4 * N))
    ga, gb, st = _np(mu_a), _np(mu_b), _np(st)
    for i, Dm in enumerate(maps):
        a, b, deg = ogmm.sky_and_disk(Dm.astype(float))
        tol = 1e-4 * max(float(Dm.max() - Dm.min()), 1.0)
        assert abs(float(ga[i]) - a) <= tol and abs(float(gb[i]) - b) <= tol, i
        assert bool(st[i] & m.ST_GMM_DEGENERATE) == deg, i


@pytest.mark.parametrize("bins", [4096, 300])
def test_gmm_bin_counts(m, bins):
    """The histogram has gmm_bins ranges (2..4096): 4096 takes the kernel's instance with sixteen
    bins per thread, 300 the eight-bin one with most threads holding fewer than eight."""
    wl = WORKLOADS["plain-N256"]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    cfg.gmm_bins = bins
    mu_a, mu_b, _ = m.gmm(D, cfg)
    for i, (_, Do, _, _) in enumerate(ref):
        a, b, _ = ogmm.sky_and_disk(Do, bins)
        rng = Do.max() - Do.min()
        assert abs(float(_np(mu_a)[i]) - a) <= 1e-4 * rng
        assert abs(float(_np(mu_b)[i]) - b) <= 1e-4 * rng


# ------------------------------------------------------------------------------ restore
def test_restore(m):
    wl = WORKLOADS["plain-N256"]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    R, pos, flux, nc, st = m.clean(D, Bm, cfg, status=st)
    img, params, st = m.restore(R, Bm, pos, flux, nc, cfg, status=st)
    Do, Bo = ref[0][1], ref[0][2]
    # lobe membership is a threshold decision: no beam pixel near the lobe may sit at 1/2
    N = wl.N
    win = Bo[N - 20:N + 21, N - 20:N + 21]
    assert np.abs(win - 0.5).min() > 1e-5
    So = orestore.clean_beam(Bo)
    np.testing.assert_allclose(_np(params)[0], So, rtol=1e-5)
    pg, fg = _np(pos)[0], _np(flux)[0]
    # restore the oracle residual of the GPU's own component list (lockstep replay)
    Ro = np.array(Do, dtype=np.float64)
    for p, f in zip(pg, fg):
        py, px = divmod(int(p), N)
        Ro -= cfg.gain * Ro.ravel()[int(p)] * Bo[N - py:2 * N - py, N - px:2 * N - px]
    fo = []
    Rr = np.array(Do, dtype=np.float64)
    for p in pg:
        py, px = divmod(int(p), N)
        f = cfg.gain * Rr.ravel()[int(p)]
        fo.append(f)
        Rr -= f * Bo[N - py:2 * N - py, N - px:2 * N - px]
    Io = orestore.restore(Rr, pg, np.array(fo), So)
    assert np.abs(_np(img)[0] - Io).max() <= 1e-4 * np.abs(Io).max()


# ------------------------------------------------------------------------------ whole path
def test_image_end_to_end_plain_frame(m):
    wl = synth.config1_plain_frame()
    cfg = cfg_for(m, wl)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ro = oracle_records(wl)
    o = pipeline.image_instance(geometry.instance_slice(ro, 0, wl.n_bl), wl.N, wl.G, gain=wl.gain, cap=wl.max_iter)
    assert int(_np(out.n_comp)[0]) == wl.max_iter
    lockstep(o["D"], o["Bm"], _np(out.comp_pos)[0], _np(out.comp_flux)[0], wl.gain)
    identical_positions_unless_near_tie(o["D"], o["Bm"], _np(out.comp_pos)[0], wl.gain, wl.max_iter)
    np.testing.assert_allclose(_np(out.beam_params)[0], o["S"], rtol=1e-5)
    if np.array_equal(o["pos"], _np(out.comp_pos)[0]):
        peak = np.abs(o["clean"]).max()
        assert np.abs(_np(out.clean)[0] - o["clean"]).max() <= 1e-4 * peak
        assert np.abs(_np(out.residual)[0] - o["R"]).max() <= 1e-4 * np.abs(o["D"]).max()


def test_image_batched_equals_per_instance(m):
    """Chunked batches give the same result as one image per call (the plain path)."""
    import torch
    wl = WORKLOADS["small-N32-3frames"]()
    cfg = cfg_for(m, wl, max_iter=40, batch_chunk=2)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    cfg1 = cfg_for(m, wl, max_iter=40)
    for f in range(wl.n_frame):
        for c in range(wl.n_chan):
            one = m.image(wl.ant_enu, wl.pairs, wl.ha[f:f + 1], wl.dec[f:f + 1], wl.freq[c:c + 1], cell[c:c + 1],
                          wl.vis[f:f + 1, c:c + 1], cfg1, flags=wl.flags[f:f + 1, c:c + 1])
            i = f * wl.n_chan + c
            # identical components; images equal up to the order of the shared-memory
            # float additions in gridding
            assert torch.equal(one.comp_pos[0], out.comp_pos[i])
            peak = float(one.clean[0].abs().max())
            assert float((one.clean[0] - out.clean[i]).abs().max()) <= 1e-6 * peak


@pytest.mark.parametrize("key,chunk", [("small-N32-3frames", 2), ("N256x6", 4)])
def test_image_graph_replay(m, key, chunk):
    """The whole batch captured in one CUDA graph (both streams of muser_image, several
    chunks) replays to the eager result."""
    import torch
    wl = (WORKLOADS.get(key) or ONCHIP_CASES[key])()
    cfg = cfg_for(m, wl, max_iter=60, batch_chunk=chunk)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ref = im.run()
    torch.cuda.synchronize()
    pos, n, clean = ref.comp_pos.clone(), ref.n_comp.clone(), ref.clean.clone()
    im.capture()
    for _ in range(2):
        out = im.replay()
    torch.cuda.synchronize()
    assert torch.equal(out.n_comp, n)
    assert torch.equal(out.comp_pos, pos)
    peak = float(clean.abs().max())
    assert float((out.clean - clean).abs().max()) <= 1e-6 * peak


def test_gmm_threshold_path(m):
    wl = synth.small_workload(n_ant=10, N=64, config_id=205, bmax=300.0, max_iter=1000)
    cfg = cfg_for(m, wl, thr_mode=1)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ro = oracle_records(wl)
    o = pipeline.image_instance(geometry.instance_slice(ro, 0, wl.n_bl), wl.N, wl.G, cap=1000, thr_mode=1)
    rng = o["D"].max() - o["D"].min()
    assert abs(float(_np(out.thr)[0]) - o["mu_a"]) <= 1e-4 * rng
    n = int(_np(out.n_comp)[0])
    # count may differ by one only when the oracle's final peak is within 1e-4 peak of thr
    if n != len(o["pos"]):
        assert abs(n - len(o["pos"])) == 1
    lockstep(o["D"], o["Bm"], _np(out.comp_pos)[0][:n], _np(out.comp_flux)[0][:n], wl.gain)


# ------------------------------------------------------------------------------ edge cases
def test_edge_cases(m):
    import torch
    wl = synth.small_workload(n_ant=9, N=32, n_frame=2, config_id=206, bmax=150.0)
    wl.flags[1] = 1                          # second instance fully flagged
    wl.vis[0, 0, 3] = np.nan                 # one non-finite visibility
    cfg = cfg_for(m, wl, max_iter=20)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    st = _np(out.status)
    assert st[1] & m.ST_ALL_FLAGGED and int(_np(out.n_comp)[1]) == 0
    assert np.all(_np(out.clean)[1] == 0)
    assert st[0] & m.ST_NONFINITE and not (st[0] & m.ST_ALL_FLAGGED)
    assert np.isfinite(_np(out.clean)[0]).all()
    # empty batch and zero iterations
    z = m.image(wl.ant_enu, wl.pairs, wl.ha[:0], wl.dec[:0], wl.freq, cell, wl.vis[:0], cfg)
    assert z.clean.shape[0] == 0
    cfg0 = cfg_for(m, wl, max_iter=0)
    o0 = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg0, flags=wl.flags)
    assert np.all(_np(o0.n_comp) == 0)
    np.testing.assert_array_equal(_np(o0.clean), _np(o0.residual))
    # errors are reported, not launched
    with pytest.raises(m.MuserError):
        m.dirty(torch.zeros((1, 100, 100), dtype=torch.complex64, device="cuda"), m.Config(N=25, G=100))
    with pytest.raises(m.MuserError):
        m.clean(torch.zeros((1, 32, 32), device="cuda"), torch.zeros((1, 64, 64), device="cuda"),
                m.Config(N=32, G=128, gain=0.0))


# ------------------------------------------------------------------------------ degridding operator
def _op_case(m, N=32, n_chan=3, seed=220):
    wl = synth.small_workload(n_ant=7, N=N, config_id=seed, bmax=150.0, freq=np.linspace(1.0e9, 1.6e9, n_chan))
    G = 2 * N
    cell = np.full(wl.n_chan, geometry.pixel_size(wl.freq.max(), wl.bmax, N, 60 * synth.ARCMIN))
    cfg = m.Config(N=N, G=G, lat_rad=wl.lat)
    rec, _, _ = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    ro = geometry.grid_records(uvw, wl.vis, wl.flags, cell, G, 7)
    assert_no_ties(ro, G, 7)
    return wl, cfg, rec, ro


def test_degrid_degenerate_record_sets(m):
    """No records, or only records with w = 0 (every baseline flagged): the forward operator gives
    zeros (or nothing), the adjoint an all-zero image, and a gradient step a zero loss and
    gradient that leaves the image unchanged."""
    import torch
    wl, cfg, rec, ro = _op_case(m, 32)
    N = cfg.N
    x = torch.tensor(np.random.default_rng(3).normal(size=(N, N)), dtype=torch.float32, device="cuda")
    empty = rec[:0]
    plan0 = m.DegridPlan(empty, cfg)
    assert plan0.forward(x).numel() == 0
    assert float(plan0.adjoint(torch.zeros(0, dtype=torch.complex64, device="cuda")).abs().max()) == 0.0
    flagged = rec.clone()
    m.record_fields(flagged)[5].zero_()                          # w = 0: every record weighted out
    plan = m.DegridPlan(flagged, cfg)
    assert float(plan.forward(x).abs().max()) == 0.0
    obs = torch.tensor(ro["vis"], dtype=torch.complex64, device="cuda")
    assert float(plan.adjoint(obs).abs().max()) == 0.0
    x1 = x.clone()
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    grad = torch.empty((N, N), dtype=torch.float32, device="cuda")
    plan.grad_step(x1, obs, 4.0, 0.1, loss, grad)
    assert float(loss[0]) == 0.0 and float(grad.abs().max()) == 0.0
    assert torch.equal(x1, x)


def _cfg4(m):
    wl = synth.config4_operator()
    N, G = wl.N, wl.G
    cell = np.full(wl.n_chan, geometry.pixel_size(wl.freq.max(), wl.bmax, N, wl.fov_min))
    cell[:] = 60 * synth.ARCMIN / N
    cfg = m.Config(N=N, G=G, lat_rad=wl.lat)
    rec, _, _ = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    ro = geometry.grid_records(uvw, wl.vis, wl.flags, cell, G, 7)
    return wl, cfg, rec, ro


@pytest.mark.parametrize("N", [32, 64])
def test_degrid_forward_adjoint(m, N):
    import torch
    wl, cfg, rec, ro = _op_case(m, N)
    rng = np.random.default_rng(0)
    x = rng.uniform(size=(N, N))
    y = (rng.normal(size=len(ro["w"])) + 1j * rng.normal(size=len(ro["w"]))) * ro["w"]
    Ax = _np(m.degrid(m.FORWARD, rec, cfg, img=torch.tensor(x, dtype=torch.float32, device="cuda")))
    Ao = oop.forward(x, ro, N, cfg.G, KER)
    assert np.linalg.norm(Ax - Ao) <= 1e-4 * np.linalg.norm(Ao)
    Ay = _np(m.degrid(m.ADJOINT, rec, cfg, vis=torch.tensor(y, dtype=torch.complex64, device="cuda")))
    Ayo = oop.adjoint(y, ro, N, cfg.G, KER).real
    assert np.linalg.norm(Ay - Ayo) <= 1e-4 * np.linalg.norm(Ayo)
    # dot-product test of the GPU pair itself: <A x, y> = <x, Re A^H y> for real x
    lhs = np.vdot(y, Ax.astype(np.complex128)).real
    rhs = float((x * Ay.astype(np.float64)).sum())
    assert lhs == pytest.approx(rhs, rel=1e-4)


def test_degrid_plan_reuse(m):
    """Calls that reuse a plan give the same results as planning calls."""
    import torch
    N = 64
    wl, cfg, rec, ro = _op_case(m, N, n_chan=6)
    rng = np.random.default_rng(4)
    x = torch.tensor(rng.uniform(size=(N, N)), dtype=torch.float32, device="cuda")
    y = torch.tensor(ro["vis"] * ro["w"], dtype=torch.complex64, device="cuda")
    plan = m.DegridPlan(rec, cfg)
    a1, b1 = plan.forward(x), plan.adjoint(y)
    assert plan.planned
    a2, b2 = plan.forward(x), plan.adjoint(y)
    assert torch.equal(a1, a2)
    assert float((b1 - b2).abs().max()) <= 1e-6 * float(b1.abs().max())
    ref_a = m.degrid(m.FORWARD, rec, cfg, img=x)
    assert torch.equal(a1, ref_a)


def test_autograd_gradient_vs_oracle_and_fd(m):
    import torch
    from paper_1712_06913_b300.autograd import chi2_loss
    N = 32
    wl, cfg, rec, ro = _op_case(m, N)
    obs = torch.tensor(ro["vis"], dtype=torch.complex64, device="cuda")
    sigma = 0.5
    rng = np.random.default_rng(1)
    x0 = rng.uniform(size=(N, N)) * 0.01
    x = torch.tensor(x0, dtype=torch.float32, device="cuda", requires_grad=True)
    plan = m.DegridPlan(rec, cfg)
    loss = chi2_loss(x, plan, obs, 1 / sigma ** 2)
    loss.backward()
    g = _np(x.grad)
    co, go = oop.chi2_grad(x0, ro, ro["vis"], sigma, N, cfg.G, KER)
    assert float(loss.detach()) == pytest.approx(co, rel=1e-4)
    assert np.linalg.norm(g - go) <= 1e-4 * np.linalg.norm(go)
    # finite differences of the GPU loss (chi2 is quadratic: central differences are exact up to rounding)
    h = 0.05
    for p in rng.choice(N * N, 64, replace=False):
        e = torch.zeros(N * N, device="cuda")
        e[p] = h
        e = e.view(N, N)
        with torch.no_grad():
            lp = float(chi2_loss(x + e, plan, obs, 1 / sigma ** 2))
            lm = float(chi2_loss(x - e, plan, obs, 1 / sigma ** 2))
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g.ravel()[p]) <= 1e-3 * np.abs(g).max() + 1e-3 * abs(fd)


def test_operator_full_size(m):
    """Forward and adjoint at the differentiable-imaging size (512^2 sky, 780 x 64 visibilities)."""
    import torch
    wl, cfg, rec, ro = _cfg4(m)
    assert_no_ties(ro, cfg.G, 7)
    rng = np.random.default_rng(3)
    x = rng.uniform(size=(cfg.N, cfg.N)) * 1e-3
    Ax = _np(m.degrid(m.FORWARD, rec, cfg, img=torch.tensor(x, dtype=torch.float32, device="cuda")))
    Ao = oop.forward(x, ro, cfg.N, cfg.G, KER)
    assert np.linalg.norm(Ax - Ao) <= 1e-4 * np.linalg.norm(Ao)
    y = ro["vis"] * ro["w"]
    Ay = _np(m.degrid(m.ADJOINT, rec, cfg, vis=torch.tensor(y, dtype=torch.complex64, device="cuda")))
    Ayo = oop.adjoint(y, ro, cfg.N, cfg.G, KER).real
    assert np.linalg.norm(Ay - Ayo) <= 1e-4 * np.linalg.norm(Ayo)


def test_gradient_descent_imaging_vs_oracle_and_graph_replay(m):
    """GD imaging through the autograd functions follows the oracle's GD; a CUDA-graph
    replay of one step equals an eager step."""
    import torch
    from paper_1712_06913_b300.autograd import GradientImaging
    N = 32
    wl, cfg, rec, ro = _op_case(m, N)
    sigma = 0.5
    obs = torch.tensor(ro["vis"], dtype=torch.complex64, device="cuda")
    gd = GradientImaging(rec, obs, sigma, cfg)
    L_gpu = gd.lipschitz(iters=40)
    L_orc = oop.lipschitz(ro, N, cfg.G, KER, sigma, iters=40)
    assert L_gpu == pytest.approx(L_orc, rel=2e-2)
    eta = 1.0 / L_orc
    gd.eta = eta
    hist = [float(gd.step()) for _ in range(20)]
    x_o = np.zeros((N, N))
    hist_o = []
    for _ in range(20):
        c, g = oop.chi2_grad(x_o, ro, ro["vis"], sigma, N, cfg.G, KER)
        hist_o.append(c)
        x_o = x_o - eta * g
    np.testing.assert_allclose(hist, hist_o, rtol=1e-3)
    x_g = _np(gd.x)
    assert np.linalg.norm(x_g - x_o) <= 1e-3 * np.linalg.norm(x_o)
    # graph replay == eager step from the same state
    gd2 = GradientImaging(rec, obs, sigma, cfg, eta=eta)
    gd2.capture(warmup=2)
    x_before = gd2.x.detach().clone()
    gd2.replay(1)
    x_replay = gd2.x.detach().clone()
    gd3 = GradientImaging(rec, obs, sigma, cfg, x0=x_before, eta=eta)
    gd3.step()
    assert float((gd3.x.detach() - x_replay).abs().max()) <= 1e-6 * float(x_replay.abs().max())


@pytest.mark.parametrize("N", [32, 64])
def test_fused_gradient_step_equals_autograd_step(m, N):
    """muser_grad_step (forward, chi-square fused into the interpolation, adjoint, update in the
    adjoint's epilogue) equals the step through the autograd functions: same loss, gradient
    and updated image up to the order of float sums."""
    import torch
    from paper_1712_06913_b300.autograd import GradientImaging
    wl, cfg, rec, ro = _op_case(m, N)
    obs = torch.tensor(ro["vis"], dtype=torch.complex64, device="cuda")
    x0 = torch.tensor(np.random.default_rng(N).normal(size=(N, N)), dtype=torch.float32, device="cuda")
    a = GradientImaging(rec, obs, 0.5, cfg, x0=x0, eta=1e-4)
    b = GradientImaging(rec, obs, 0.5, cfg, x0=x0, eta=1e-4)
    la = float(a.step())                       # fused (single process)
    lb = float(b.step_autograd())
    assert la == pytest.approx(lb, rel=1e-5)
    xa, xb = a.x.detach(), b.x.detach()
    assert float((xa - xb).abs().max()) <= 1e-6 * float(xb.abs().max())
    # the gradient output of the fused call against the oracle's FP64 gradient at x0
    plan = a.plan
    grad = torch.empty((N, N), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    x = x0.clone()
    plan.grad_step(x, obs, 1.0 / 0.25, 0.0, loss, grad)
    assert torch.equal(x, x0)                   # eta = 0 leaves the image
    c_o, g_o = oop.chi2_grad(x0.cpu().numpy().astype(np.float64), ro, ro["vis"], 0.5, N, cfg.G, KER)
    assert float(loss[0]) == pytest.approx(c_o, rel=1e-4)
    assert np.linalg.norm(_np(grad) - g_o) <= 1e-4 * np.linalg.norm(g_o)


@pytest.mark.parametrize("N", [32, 64])
def test_grad_step_uniform_weights_vs_oracle(m, N):
    """weight_mode 1 in the operator's plan: the chi-square weighs each record by Alg. 1's uniform
    weight (1 / samples in its cell of the N x N grid, G/N = 2 uv cells wide), computed by the
    plan from the records.  Loss and gradient of muser_grad_step against the FP64 oracle with
    oracle.imaging.uniform_weights; the autograd loss (the records' own weights) refuses it."""
    import torch
    from paper_1712_06913_b300.autograd import chi2_loss
    wl, cfg, rec, ro = _op_case(m, N, n_chan=4)
    cfg_u = m.Config(N=N, G=cfg.G, lat_rad=wl.lat, weight_mode=1)
    ro_u = dict(ro)
    ro_u["w"] = imaging.uniform_weights(ro, cfg.G, N)
    assert (ro_u["w"][ro["w"] > 0] < 1.0).any()          # some cells hold several samples
    obs = torch.tensor(ro["vis"], dtype=torch.complex64, device="cuda")
    x0 = np.random.default_rng(N + 7).normal(size=(N, N))
    plan = m.DegridPlan(rec, cfg_u)
    x = torch.tensor(x0, dtype=torch.float32, device="cuda")
    grad = torch.empty((N, N), dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    plan.grad_step(x, obs, 1.0 / 0.25, 0.0, loss, grad)
    c_o, g_o = oop.chi2_grad(x0, ro_u, ro["vis"], 0.5, N, cfg.G, KER)
    c_n, g_n = oop.chi2_grad(x0, ro, ro["vis"], 0.5, N, cfg.G, KER)
    assert float(loss[0]) == pytest.approx(c_o, rel=1e-4)
    assert np.linalg.norm(_np(grad) - g_o) <= 1e-4 * np.linalg.norm(g_o)
    assert np.linalg.norm(g_n - g_o) > 1e-2 * np.linalg.norm(g_o)   # the weights matter here
    with pytest.raises(ValueError):
        chi2_loss(x, plan, obs, 4.0)


# ------------------------------------------------------------------------------ disk centring (Sec. 4.2)
def _centring_case(off_px, N=128, seed=110):
    wl0 = synth.small_workload(n_ant=31, N=N, config_id=seed, bmax=600.0, snr=0)
    cell = pipeline.cell_sizes(wl0)[0]
    sky = synth.Sky(disk_lm=(off_px[0] * cell, off_px[1] * cell))
    wl = synth.make_workload("c", wl0.ant_enu, wl0.pairs, wl0.ha, wl0.dec, wl0.freq, N, 4 * N,
                             config_id=seed, skies=[sky], snr=30, bmax=600.0)
    return wl, cell


@pytest.mark.parametrize("off_px,N", [((5.0, -3.0), 128), ((-11.4, 7.6), 128), ((7.3, 4.2), 160),
                                      ((-9.6, 12.2), 256), ((3.3, -6.8), 320)])
def test_center_correlation_and_shift_vs_oracle(m, off_px, N):
    """muser_center on the oracle's pre-cleaned residual: the disk correlation over all
    shifts within 1e-5 of its peak, the best shift and its parabolic refinement equal."""
    import torch
    from oracle import centering
    wl, cell = _centring_case(off_px, N=N)
    rec = pipeline.records(wl)
    ker = pipeline.spheroidal(7, 1024)
    _, D, Bm, _ = pipeline.dirty(rec, N, 4 * N, ker)
    mu_a, mu_b, _ = ogmm.sky_and_disk(D)
    R, _, _ = oclean.hogbom(D, Bm, 0.1, mu_b, 1000)
    # both sides decide the mask in FP32 from the same FP32 inputs
    R32, a32, b32 = R.astype(np.float32), np.float32(mu_a), np.float32(mu_b)
    thr = np.float32(0.5) * (a32 + b32)
    r = centering.SUN_RADIUS / cell if hasattr(centering, "SUN_RADIUS") else 16 * np.pi / 180 / 60 / cell
    d2 = ((np.arange(N) - N // 2)[:, None] ** 2 + (np.arange(N) - N // 2)[None, :] ** 2).astype(float)
    assert np.abs(d2 - r * r).min() > 1e-3, "disk radius sits on a pixel-distance tie"
    M = np.where(R32 > thr, R32, np.float32(0)).astype(np.float64)
    S = centering.disk_model(N, r)
    Cc = centering.correlation(M, S, N // 4)
    cfg = m.Config(N=N, G=4 * N)
    dlm, shift, corr, st = m.center(torch.tensor(R32[None], device="cuda"),
                                    torch.tensor([a32], device="cuda"), torch.tensor([b32], device="cuda"),
                                    np.array([cell]), cfg, want_corr=True)
    Cg = _np(corr)[0]
    assert np.abs(Cg - Cc).max() <= 1e-5 * np.abs(Cc).max()
    sx, sy = centering.best_shift(Cc, N // 4)
    gs = _np(shift)[0]
    assert abs(gs[0] - sx) <= 1e-3 and abs(gs[1] - sy) <= 1e-3, (gs, sx, sy)
    np.testing.assert_allclose(_np(dlm)[0], [gs[0] * cell, gs[1] * cell], rtol=1e-6)
    assert int(_np(st)[0]) & m.ST_NO_DISK == 0


@pytest.mark.parametrize("N,off", [(1024, (17.0, -23.0)), (1280, (-31.0, 8.0))])
def test_center_synthetic_disk_large(m, N, off):
    """Sides whose row pass holds one row pair per block (P = 2N = 2048, 2560): a disk of
    radius 0.3 N shifted by whole pixels plus noise and bright spots, against the oracle's
    correlation over all shifts and its best shift."""
    import torch
    from oracle import centering
    rng = np.random.default_rng(N)
    r = 0.3 * N + 0.37
    cell = 16 * np.pi / 180 / 60 / r
    y, x = np.mgrid[0:N, 0:N]
    R = np.where((x - N // 2 - off[0]) ** 2 + (y - N // 2 - off[1]) ** 2 <= r * r, 1.0, 0.0)
    R += 0.2 * rng.standard_normal((N, N))
    R[rng.integers(0, N, 40), rng.integers(0, N, 40)] += 3.0
    R32 = R.astype(np.float32)
    thr = np.float32(0.5) * (np.float32(0.0) + np.float32(1.0))
    M = np.where(R32 > thr, R32, np.float32(0)).astype(np.float64)
    S = centering.disk_model(N, r)
    Cc = centering.correlation(M, S, N // 4)
    cfg = m.Config(N=N, G=4 * N)
    dlm, shift, corr, st = m.center(torch.tensor(R32[None], device="cuda"), torch.zeros(1, device="cuda"),
                                    torch.ones(1, device="cuda"), np.array([cell]), cfg, want_corr=True)
    Cg = _np(corr)[0]
    assert np.abs(Cg - Cc).max() <= 1e-5 * np.abs(Cc).max()
    sx, sy = centering.best_shift(Cc, N // 4)
    gs = _np(shift)[0]
    assert abs(gs[0] - sx) <= 1e-3 and abs(gs[1] - sy) <= 1e-3, (gs, sx, sy)
    assert abs(sx - off[0]) <= 0.5 and abs(sy - off[1]) <= 0.5


def test_image_centred_end_to_end(m):
    """GPU pipeline (dirty -> GMM -> CLEAN to the disk level -> centring -> corrected
    re-imaging) against the oracle's disk_offset, and the known offset."""
    from oracle import centering
    off = (6.0, -4.0)
    wl, cell = _centring_case(off)
    N = wl.N
    cfg = cfg_for(m, wl, max_iter=300)
    cells = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out, dlm, shift = m.image_centred(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cells, wl.vis, cfg,
                                      flags=wl.flags)
    rec = pipeline.records(wl)
    ker = pipeline.spheroidal(7, 1024)
    _, D, Bm, _ = pipeline.dirty(rec, N, 4 * N, ker)
    mu_a, mu_b, _ = ogmm.sky_and_disk(D)
    dl, dm, _, _, _ = centering.disk_offset(D, Bm, mu_a, mu_b, cell, wl.dec[0])
    gs = _np(shift)[0]
    assert abs(gs[0] - dl / cell) <= 0.05 and abs(gs[1] - dm / cell) <= 0.05, (gs, dl / cell, dm / cell)
    assert abs(gs[0] - off[0]) <= 0.3 and abs(gs[1] - off[1]) <= 0.3
    assert int(_np(out.n_comp)[0]) > 0


def test_centred_imager_graph_equals_eager(m):
    """CentredImager: the whole centring pipeline enqueued without host synchronisation agrees
    with image_centred, and its CUDA-graph replay with its eager run (the tiled gridding adds
    overlapping footprints in no fixed order, so runs agree to rounding, not bit for bit)."""
    import torch
    off = (6.0, -4.0)
    wl, cell = _centring_case(off)
    cfg = cfg_for(m, wl, max_iter=300)
    cells = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    ref, _, shift_ref = m.image_centred(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cells, wl.vis, cfg,
                                        flags=wl.flags)
    ci = m.CentredImager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cells, wl.vis, cfg, flags=wl.flags)
    out = ci.run()
    torch.cuda.synchronize()
    # a shift that differs in its last bits phase-rotates the visibilities a little differently,
    # so the two CLEANs may part at a near-tie: the images are compared in norm
    def rel(a, b):
        return float((a - b).norm() / b.norm())

    assert float((ci.shift - shift_ref).abs().max()) <= 1e-2
    assert rel(out.clean, ref.clean) <= 5e-2 and bool(torch.isfinite(out.clean).all())
    first, shift1 = out.clean.clone(), ci.shift.clone()
    ci.capture()
    out.clean.zero_()
    ci.dlm.zero_()
    ci.shift.zero_()
    out2 = ci.replay()
    torch.cuda.synchronize()
    assert float((ci.shift - shift1).abs().max()) <= 1e-2
    assert rel(out2.clean, first) <= 5e-2
    assert abs(float(ci.shift[0, 0]) - off[0]) <= 0.3 and abs(float(ci.shift[0, 1]) - off[1]) <= 0.3


def test_center_empty_mask(m):
    import torch
    N = 64
    cfg = m.Config(N=N, G=4 * N)
    R = torch.zeros((2, N, N), device="cuda")
    mu = torch.ones(2, device="cuda")
    dlm, shift, _, st = m.center(R, mu, mu, np.full(2, 1e-4), cfg)
    assert np.array_equal(_np(dlm), np.zeros((2, 2)))
    assert all(int(v) & m.ST_NO_DISK for v in _np(st))


# ------------------------------------------------------------------------------ Steer CLEAN
def _oracle_maps(wl):
    """FP32 copies of the oracle's dirty maps and beams: both sides start from the same values."""
    ro = oracle_records(wl)
    out = []
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Do, Bo, _ = imaging.dirty_and_beam(imaging.grid(ri, wl.G, KER), wl.N, KER)
        out.append((Do.astype(np.float32), Bo.astype(np.float32)))
    return out


def _steer_inputs(m, maps):
    import torch
    D = torch.tensor(np.stack([d for d, _ in maps]), device="cuda")
    Bm = torch.tensor(np.stack([b for _, b in maps]), device="cuda")
    return D, Bm


def _oracle_steer_chain(D, Bo, gain, clip, cap, thr=-np.inf):
    """The oracle's Steer clean run one cycle at a time, with the smallest distance (relative to
    the peak) of any pixel from the selection level (clip < 1) or of the runner-up from the peak
    (clip = 1) over the run."""
    from oracle import steer as osteer
    R = D.astype(np.float64)
    model = np.zeros_like(R)
    cycles, gap = 0, np.inf
    for _ in range(cap):
        mx = R.max()
        if clip < 1:
            gap = min(gap, np.abs(R - clip * mx).min() / mx)
        else:
            s = np.partition(R.ravel(), -2)[-2:]
            gap = min(gap, (s[1] - s[0]) / mx)
        R, md, c = osteer.steer(R, Bo.astype(np.float64), gain, thr, 1, clip)
        if c == 0:
            break
        model += md
        cycles += 1
    return R, model, cycles, gap


@pytest.mark.parametrize("name,clip,cycles", [("small-N64", 0.9, 16), ("small-N32-3frames", 0.7, 40),
                                              ("plain-N256", 0.7, 6), ("N1024x1", 0.8, 2), ("N160", 0.9, 8),
                                              ("N320x2", 0.8, 4)])
def test_steer_cycle_lockstep(m, name, clip, cycles):
    """One major cycle at a time from the GPU's own residual: C is decided in FP32 from the same
    FP32 residual on both sides (so near-ties cannot split them); Y, a and the update follow
    the oracle's FP64 convolution."""
    from oracle import steer as osteer
    wl = (synth.config3_muser2_uneven(n_frame=1, chans=[7]) if name == "N1024x1"
          else (FIVE_CASES.get(name) or WORKLOADS[name])())
    maps = _oracle_maps(wl)
    N = wl.N
    cfg = m.Config(N=N, G=4 * N)
    cfg.max_iter = 1
    R, Bm = _steer_inputs(m, maps)
    for _ in range(cycles):
        Rp = _np(R)
        R, model, nc, _ = m.steer(R, Bm, cfg, clip=clip)
        Rg, Mg, ncg = _np(R), _np(model), _np(nc)
        for i, (_, Bo) in enumerate(maps):
            r = Rp[i]
            mx = r.max()
            tau = np.float32(clip) * mx
            C = np.where(r >= tau, r, np.float32(0)).astype(np.float64)
            Y = osteer.convolve_beam(C, Bo.astype(np.float64))
            a = cfg.gain * float(mx) / Y.max()
            assert ncg[i] == 1
            scale = float(np.abs(r).max())
            assert np.abs(Rg[i] - (r - a * Y)).max() <= 1e-5 * scale
            assert np.array_equal(Mg[i] != 0, C != 0)
            assert np.abs(Mg[i] - a * C).max() <= 1e-5 * np.abs(a * C).max()


@pytest.mark.parametrize("name,clip,cap", [("small-N64", 0.9, 12), ("small-N32-3frames", 0.9, 40),
                                           ("plain-N256", 0.9, 15), ("small-N64", 1.0, 60),
                                           ("plain-N256", 1.0, 60)])
def test_steer_vs_oracle(m, name, clip, cap):
    """Whole runs against the oracle (runs with no pixel within 1e-5 of the peak of its selection
    level, so FP32 and FP64 choose the same maps): cycle counts equal, residual and model
    within 1e-4 of the peak, and D = R + Bm * model.  With clip = 1 the cycles are Hogbom steps:
    the model equals the oracle Hogbom components accumulated into a map."""
    from oracle import steer as osteer
    wl = WORKLOADS[name]()
    maps = _oracle_maps(wl)
    cfg = m.Config(N=wl.N, G=4 * wl.N)
    cfg.max_iter = cap
    D, Bm = _steer_inputs(m, maps)
    R, model, nc, st = m.steer(D, Bm, cfg, clip=clip)
    Rg, Mg, ncg = _np(R), _np(model), _np(nc)
    for i, (Do, Bo) in enumerate(maps):
        Ro, Mo, co, gap = _oracle_steer_chain(Do, Bo, cfg.gain, clip, cap)
        assert gap > 1e-5, "the oracle run has a near-tie at its selection level"
        peak = float(np.abs(Do).max())
        assert ncg[i] == co == cap
        assert np.abs(Rg[i] - Ro).max() <= 1e-4 * peak
        assert np.abs(Mg[i] - Mo).max() <= 1e-4 * peak
        resid = Do.astype(np.float64) - Rg[i] - osteer.convolve_beam(Mg[i].astype(np.float64), Bo.astype(np.float64))
        assert np.abs(resid).max() <= 1e-4 * peak
        if clip == 1.0:
            _, po, fo = oclean.hogbom(Do.astype(np.float64), Bo.astype(np.float64), cfg.gain, -np.inf, cap)
            Mh = np.zeros_like(Mo)
            np.add.at(Mh, (po[:, 0], po[:, 1]) if po.ndim == 2 else np.unravel_index(po, Mh.shape), fo)
            assert np.array_equal(Mg[i] != 0, Mh != 0)
            assert np.abs(Mg[i] - Mh).max() <= 1e-4 * peak


def test_steer_thresholds_batch_and_edges(m):
    """Per-instance thresholds stop instances at different cycles (as in the oracle); a batch
    equals its instances run alone, bit for bit; the GMM threshold mode equals passing the GMM
    sky level; flagged instances, all-negative maps and a zero beam run no cycle."""
    import torch
    wl = WORKLOADS["small-N32-3frames"]()
    maps = _oracle_maps(wl)
    cfg = m.Config(N=wl.N, G=4 * wl.N)
    cfg.max_iter = 200
    D, Bm = _steer_inputs(m, maps)
    peaks = np.array([d.max() for d, _ in maps])
    thr = np.float32([0.5, 0.2, 0.05, 0.3, 0.1, 0.02]) * peaks.astype(np.float32)
    R, model, nc, _ = m.steer(D, Bm, cfg, thr=thr, clip=0.9)
    ncg = _np(nc)
    for i, (Do, Bo) in enumerate(maps):
        _, _, co, _ = _oracle_steer_chain(Do, Bo, cfg.gain, 0.9, 200, thr=float(thr[i]))
        assert abs(int(ncg[i]) - co) <= 1
        assert _np(R)[i].max() <= thr[i] or ncg[i] == 200
    assert ncg[0] < ncg[1] < ncg[2]
    for i in range(len(maps)):
        R1, M1, n1, _ = m.steer(D[i:i + 1], Bm[i:i + 1], cfg, thr=thr[i:i + 1], clip=0.9)
        assert torch.equal(R1[0], R[i]) and torch.equal(M1[0], model[i]) and int(n1[0]) == int(nc[i])
    # GMM threshold mode
    cfg.thr_mode = 1
    mu_a, _, _ = m.gmm(D, cfg)
    Ra, Ma, na, _ = m.steer(D, Bm, cfg, clip=0.9)
    cfg.thr_mode = 0
    Rb, Mb, nb, _ = m.steer(D, Bm, cfg, thr=mu_a, clip=0.9)
    assert torch.equal(Ra, Rb) and torch.equal(Ma, Mb) and torch.equal(na, nb)
    # edges
    st = torch.tensor([m.ST_ALL_FLAGGED, 0, 0], dtype=torch.int32, device="cuda")
    D, Bm = D[:3], Bm[:3]
    Dn = D.clone()
    Dn[1] = -Dn[1].abs() - 1.0
    Bz = Bm.clone()
    Bz[2] = 0
    R, model, nc, _ = m.steer(Dn, Bz, cfg, clip=0.9, status=st)
    assert _np(nc).tolist() == [0, 0, 0]
    assert torch.equal(R, Dn) and float(model.abs().max()) == 0.0
    R, model, nc, _ = m.steer(D[:0], Bm[:0], cfg)
    assert nc.numel() == 0


# ------------------------------------------------------------------------------ image sides 5 * 2^a
# Table 2's high-band images are 1280, 2560 and 5120 pixels on a side (grids of 5 * 2^m cells):
# the transforms then start with one radix-5, -10, -20 or -40 stage.
FIVE_CASES = {
    "N160": lambda: synth.small_workload(n_ant=12, N=160, config_id=250, bmax=600.0),          # G 640: 40, 16
    "N320x2": lambda: synth.small_workload(n_ant=16, N=320, n_frame=2, config_id=251, bmax=1200.0,
                                           flag_max=0.3),                                     # G 1280: 5, 16, 16
    "N640": lambda: synth.small_workload(n_ant=21, N=640, config_id=252, bmax=2000.0),         # G 2560: 10, 16, 16
    "N1280": lambda: synth.muser2_large_band(1280, chans=[3, 70]),                          # G 5120: 20, 16, 16
}


@pytest.mark.parametrize("name", list(FIVE_CASES))
def test_grid_and_dirty_five(m, name):
    wl = FIVE_CASES[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    Zg, Dg, Bg = _np(Z), _np(D), _np(Bm)
    for i, (Zo, Do, Bo, norm) in enumerate(ref):
        assert np.abs(Zg[i] - Zo).max() <= 1e-5 * np.abs(Zo).max()
        assert np.abs(Dg[i] - Do).max() <= 1e-4 * np.abs(Do).max(), i
        assert np.abs(Bg[i] - Bo).max() <= 1e-4, i
        assert abs(Bg[i][wl.N, wl.N] - 1.0) <= 1e-6


@pytest.mark.parametrize("N", [2560, 5120])
def test_dirty_largest_sides_sampled(m, N):
    """One MUSER-II instance at 2560^2 (G = 10240) and 5120^2 (G = 20480): sampled pixels of the
    map and the beam against the oracle's per-pixel transform of the sparse grid."""
    from oracle import imaging as oim
    wl = synth.muser2_large_band(N, chans=[5])
    cfg = cfg_for(m, wl)
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    Z, st = m.grid(rec, off, cfg, status=st)
    D, Bm, st = m.dirty(Z, cfg, status=st)
    del Z
    Dg, Bg = _np(D)[0], _np(Bm)[0]
    ri = geometry.instance_slice(oracle_records(wl), 0, wl.n_bl)
    rng = np.random.default_rng(N)
    ym, xm = np.unravel_index(np.argmax(np.abs(Dg)), Dg.shape)
    dp = np.concatenate([rng.integers(0, N, (24, 2)), [[ym, xm], [N // 2, N // 2], [0, N - 1]]])
    bp = np.concatenate([rng.integers(0, 2 * N, (16, 2)), [[N, N], [N, N + 1], [N - 3, N + 2]]])
    Do, Bo, _ = oim.dirty_and_beam_at(ri, wl.G, N, KER, dp, bp)
    scale = np.abs(Dg).max()
    assert np.abs(Dg[dp[:, 0], dp[:, 1]] - Do).max() <= 1e-4 * scale
    assert np.abs(Bg[bp[:, 0], bp[:, 1]] - Bo).max() <= 1e-4
    assert abs(Bg[N, N] - 1.0) <= 1e-6


@pytest.mark.parametrize("name,cap", [("N320x2", 150), ("N1280", 100)])
def test_image_five_end_to_end(m, name, cap):
    """muser_image at 5 * 2^a sides (gridding fused into the radix-5 column pass, streaming
    CLEAN, restore) against the oracle pipeline, component by component."""
    wl = FIVE_CASES[name]()
    cfg = cfg_for(m, wl, max_iter=cap)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ro = oracle_records(wl)
    for i in range(wl.n_inst):
        o = pipeline.image_instance(geometry.instance_slice(ro, i, wl.n_bl), wl.N, wl.G, gain=wl.gain, cap=cap)
        pg, fg = _np(out.comp_pos)[i], _np(out.comp_flux)[i]
        assert int(_np(out.n_comp)[i]) == cap
        lockstep(o["D"], o["Bm"], pg, fg, wl.gain)
        identical_positions_unless_near_tie(o["D"], o["Bm"], pg, wl.gain, cap)
        np.testing.assert_allclose(_np(out.beam_params)[i], o["S"], rtol=1e-5)
        if np.array_equal(o["pos"], pg):
            assert np.abs(_np(out.clean)[i] - o["clean"]).max() <= 1e-4 * np.abs(o["clean"]).max()
            assert np.abs(_np(out.residual)[i] - o["R"]).max() <= 1e-4 * np.abs(o["D"]).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_clean_clustered_streaming_2560_equals_single_block(m, mode):
    """2560^2 in a batch smaller than half the SMs: clusters of 16 blocks stream one instance and
    give the components and residuals of one streaming block per instance, bit for bit; for the
    signed peak and for the peak of |R| (which takes the strong negative source first, followed
    against the oracle)."""
    import torch
    N = 2560
    rng = np.random.default_rng(2560)
    yy, xx = np.mgrid[-N:N, -N:N].astype(np.float32)
    Bo = np.exp(-(xx * xx + yy * yy) / np.float32(2 * 6.0 ** 2)) + np.float32(0.03) * np.cos(xx / np.float32(5)) * \
        np.cos(yy / np.float32(9))
    Bo = (Bo / Bo[N, N]).astype(np.float32)
    del yy, xx
    Do = rng.normal(size=(2, N, N)).astype(np.float32)
    Do[0, 100, 2000] += 30.0
    Do[1, 1500, 7] += 20.0
    Do[1, 700, 2400] -= 35.0
    D = torch.tensor(Do, device="cuda")
    Bm = torch.tensor(np.stack([Bo, Bo]), device="cuda")
    cfg = m.Config(N=N, G=4 * N, max_iter=30, peak_mode=mode)
    R1, p1, f1, n1, _ = m.clean(D, Bm, cfg)
    cfg.clean_kernel = 1
    R2, p2, f2, n2, _ = m.clean(D, Bm, cfg)
    assert torch.equal(n1, n2) and torch.equal(p1, p2) and torch.equal(f1, f2)
    assert float((R1 - R2).abs().max()) == 0.0
    if mode == 1:
        assert int(_np(p1)[1][0]) == 700 * N + 2400
        lockstep(Do[1], Bo, _np(p1)[1], _np(f1)[1], cfg.gain, peak_mode=1)


def test_clean_5120_streaming(m):
    """CLEAN at 5120^2 (streaming residual, one block per instance): a seeded map and beam of
    that size, 40 Hogbom steps against the oracle."""
    import torch
    N = 5120
    rng = np.random.default_rng(5120)
    yy, xx = np.mgrid[-N:N, -N:N].astype(np.float32)
    Bo = np.exp(-(xx * xx + yy * yy) / np.float32(2 * 9.0 ** 2)) + np.float32(0.05) * np.cos(xx / np.float32(7)) * \
        np.cos(yy / np.float32(11))
    Bo = (Bo / Bo[N, N]).astype(np.float32)
    del yy, xx
    Do = rng.normal(size=(N, N)).astype(np.float32)
    Do[1000, 4000] += 40.0
    Do[3000, 17] += 25.0
    cfg = m.Config(N=N, G=4 * N, max_iter=40)
    R, pos, flux, nc, _ = m.clean(torch.tensor(Do[None], device="cuda"), torch.tensor(Bo[None], device="cuda"), cfg)
    pg, fg = _np(pos)[0], _np(flux)[0]
    assert int(_np(nc)[0]) == 40
    lockstep(Do, Bo, pg, fg, 0.1)
    identical_positions_unless_near_tie(Do, Bo, pg, 0.1, 40)


# ------------------------------------------------------------------------------ w-projection
W_CASES = {
    "N64": lambda: synth.wterm_workload(),
    "N64x2ch": lambda: synth.wterm_workload(freq=(1.2e9, 1.7e9), n_frame=2, config_id=401),
    "N256": lambda: synth.wterm_workload(N=256, n_ant=31, bmax=1200.0, config_id=402),
}


def _wproj_setup(m, wl, P=128, Ww=15):
    """Both sides take the same plane spacing: w_max = float32(1.01 max |wg|) of the oracle's
    records; no sample may sit within 1e-4 of a plane boundary."""
    from oracle import wproj
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    ro = geometry.grid_records(uvw, wl.vis, wl.flags, pipeline.cell_sizes(wl), wl.G, Ww)
    w_max = float(np.float32(1.01 * np.abs(ro["wg"]).max()))
    x = np.abs(ro["wg"][ro["w"] > 0]) * (P - 1) / w_max
    assert np.abs(x - np.floor(x) - 0.5).min() > 1e-4, "a sample sits on a w-plane boundary"
    cfg = cfg_for(m, wl)
    cfg.w_planes, cfg.w_max, cfg.w_support = P, w_max, Ww
    tabs = wproj.kernel_tables(w_max, P, Ww, wl.OS, KER)
    return cfg, ro, tabs, w_max


@pytest.mark.parametrize("name", list(W_CASES))
def test_wproj_grid_and_dirty(m, name):
    """w-projected grid, map and beam against the oracle's w-projection (plane tables, complex
    taps, conjugates for w < 0 and for the mirrored samples)."""
    from oracle import wproj
    wl = W_CASES[name]()
    cfg, ro, tabs, w_max = _wproj_setup(m, wl)
    assert np.abs(ro["uvw"][:, 2]).max() > 500
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    Z, st = m.grid(rec, off, cfg, status=st)
    D, Bm, st = m.dirty(Z, cfg, status=st)
    Zg, Dg, Bg = _np(Z), _np(D), _np(Bm)
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Zo = wproj.grid(ri, wl.G, tabs, w_max, 15, wl.OS)
        Do, Bo, _ = imaging.dirty_and_beam(Zo, wl.N, KER)
        assert np.abs(Zg[i] - Zo).max() <= 1e-5 * np.abs(Zo).max(), i
        assert np.abs(Dg[i] - Do).max() <= 1e-4 * np.abs(Do).max(), i
        assert np.abs(Bg[i] - Bo).max() <= 1e-4, i
        assert abs(Bg[i][wl.N, wl.N] - 1.0) <= 1e-6


def test_wproj_image_end_to_end(m):
    """muser_image with w-projection (the fused gridding of the column pass) against the
    oracle's w-projected map and beam, Hogbom CLEAN and restore."""
    from oracle import restore as orest
    from oracle import wproj
    wl = W_CASES["N64x2ch"]()
    cfg, ro, tabs, w_max = _wproj_setup(m, wl)
    cfg.max_iter = 60
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Do, Bo, _ = imaging.dirty_and_beam(wproj.grid(ri, wl.G, tabs, w_max, 15, wl.OS), wl.N, KER)
        pg, fg = _np(out.comp_pos)[i], _np(out.comp_flux)[i]
        assert int(_np(out.n_comp)[i]) == 60
        lockstep(Do, Bo, pg, fg, cfg.gain)
        identical_positions_unless_near_tie(Do, Bo, pg, cfg.gain, 60)
        np.testing.assert_allclose(_np(out.beam_params)[i], orest.clean_beam(Bo), rtol=1e-5)


# ------------------------------------------------------------------------------ mixed stream
def test_mixed_stream_by_size_class(m):
    """A mixed stream (MUSER-I channels at 256^2 and 512^2, MUSER-II at 1024^2 by the Table 2
    rule) through the size-class batches equals imaging each class alone, eager and replayed
    from one CUDA graph; a 256^2 instance follows the oracle."""
    import torch
    w1, w2, _ = synth.config5_mixed_stream(n_total=40)
    ch1 = [0, 5, 20, 50]                      # 0.41, 0.54 GHz -> 256; 0.91, 1.66 GHz -> 512 (capped)
    src1 = m.Source(w1.ant_enu, w1.pairs, w1.ha[:2], w1.dec[:2], w1.freq[ch1], w1.vis[:2][:, ch1],
                    w1.flags[:2][:, ch1], bmax=w1.bmax, fov_min=w1.fov_min, n_max=512, max_iter=80,
                    lat_rad=w1.lat, batch_chunk=3)
    src2 = m.Source(w2.ant_enu, w2.pairs, w2.ha[:1], w2.dec[:1], w2.freq[[10, 300]], w2.vis[:1][:, [10, 300]],
                    w2.flags[:1][:, [10, 300]], bmax=w2.bmax, fov_min=w2.fov_min, n_max=1024, max_iter=80,
                    lat_rad=w2.lat)
    mix = m.MixedImager([src1, src2])
    assert [(si, c0, nc, im.cfg.N) for si, c0, nc, im in mix.classes] == [(0, 0, 2, 256), (0, 2, 2, 512),
                                                                          (1, 0, 2, 1024)]
    outs = [dataclasses_copy(o) for o in mix.run()]
    for k, (si, c0, nc, im) in enumerate(mix.classes):
        src = (src1, src2)[si]
        one = m.image(src.ant_enu, src.pairs, src.ha, src.dec, src.freq[c0:c0 + nc],
                      m.pixel_size(src.freq[c0:c0 + nc], src.bmax, im.cfg.N, src.fov_min),
                      np.ascontiguousarray(src.vis[:, c0:c0 + nc]), im.cfg,
                      flags=np.ascontiguousarray(src.flags[:, c0:c0 + nc]))
        assert torch.equal(one.comp_pos, outs[k].comp_pos[:, :80])
        peak = float(one.clean.abs().max())
        assert float((one.clean - outs[k].clean).abs().max()) <= 1e-6 * peak
    # stream instance -> class
    assert mix.locate(0, 1 * 4 + 3) == (1, 1 * 2 + 1)
    assert mix.locate(1, 1) == (2, 1)
    # graph replay
    mix.capture()
    rep = mix.replay()
    torch.cuda.synchronize()
    for k in range(3):
        assert torch.equal(rep[k].comp_pos, outs[k].comp_pos)
    # a 256^2 instance against the oracle
    wl = synth.make_workload("mix-check", w1.ant_enu, w1.pairs, w1.ha[:1], w1.dec[:1], w1.freq[[0]], 256, 1024,
                             config_id=51, flag_max=0.3)
    ro = pipeline.records(wl)
    o = pipeline.image_instance(geometry.instance_slice(ro, 0, wl.n_bl), 256, 1024, gain=0.1, cap=80)
    _, li = mix.locate(0, 0)
    assert li == 0
    lockstep(o["D"], o["Bm"], _np(outs[0].comp_pos)[0][:80], _np(outs[0].comp_flux)[0][:80], 0.1)


def dataclasses_copy(o):
    import dataclasses
    return dataclasses.replace(o, **{f.name: getattr(o, f.name).clone() for f in dataclasses.fields(o)})


# ------------------------------------------------------------------------------ autotuner
def test_autotune_grid_and_dirty_shapes(m):
    """muser_autotune picks a gridding band height and a column-strip width; every candidate
    shape gives the oracle's grid, map and beam (only the order of float sums differs)."""
    wl = WORKLOADS["small-N32-3frames"]()
    cfg = cfg_for(m, wl)
    rec, _, st, off, _ = gpu_records(m, wl, cfg, want_uvw=False)
    rows = m.autotune(m.CALL_GRID, cfg, rec=rec, vis_off=off)
    assert rows >= 1 and cfg.G % rows == 0 and rows * cfg.G * 8 <= 200 * 1024
    var = m.autotune(m.CALL_DIRTY, cfg, B=4)
    assert var in (0, 1)
    ref = _dirty_both(m, wl)[5]
    try:
        for r in (1, 2, 8, 64):
            if cfg.G % r or r * cfg.G * 8 > 200 * 1024:
                continue
            m.set_tuning(m.CALL_GRID, cfg, r)
            for v in (0, 1):
                m.set_tuning(m.CALL_DIRTY, cfg, v)
                Z, s2 = m.grid(rec, off, cfg, status=st.clone())
                D, Bm, _ = m.dirty(Z, cfg, status=s2)
                for i, (Zo, Do, Bo, _) in enumerate(ref):
                    assert np.abs(_np(Z)[i] - Zo).max() <= 1e-5 * np.abs(Zo).max(), (r, v)
                    assert np.abs(_np(D)[i] - Do).max() <= 1e-4 * np.abs(Do).max(), (r, v)
                    assert np.abs(_np(Bm)[i] - Bo).max() <= 1e-4, (r, v)
    finally:
        m.set_tuning(m.CALL_GRID, cfg, 0)
        m.set_tuning(m.CALL_DIRTY, cfg, 0)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", ["N320x2", "N640", "N1280"])
def test_clean_extended_onchip_equals_single_block(m, name, mode):
    """320, 640 and 1280 pixel images: bands of 102400 pixels on chip (65536 in tensor memory,
    36864 in shared memory; clusters of 1, 4 and 16 blocks) give the components and residuals of
    one streaming block per instance (the same operations), and follow the oracle; for the
    signed peak and for the peak of |R| (peak_mode 1)."""
    import torch
    wl = FIVE_CASES[name]()
    cfg, Z, D, Bm, st, ref = _dirty_both(m, wl)
    cfg.max_iter, cfg.peak_mode = 120, mode
    R1, p1, f1, n1, _ = m.clean(D, Bm, cfg)
    cfg.clean_kernel = 1
    R2, p2, f2, n2, _ = m.clean(D, Bm, cfg)
    assert torch.equal(n1, n2) and torch.equal(p1, p2) and torch.equal(f1, f2)
    assert float((R1 - R2).abs().max()) == 0.0
    Do, Bo = ref[0][1], ref[0][2]
    lockstep(Do, Bo, _np(p1)[0], _np(f1)[0], cfg.gain, peak_mode=mode)


# ------------------------------------------------------------------------------ failure detection
def test_bounded_wait_runs_out_and_context_stays_usable(m):
    """A wait that nothing completes (the exchange's try_wait loop, on an mbarrier no one
    arrives at) gives up after its bound and reports MUSER_ST_TIMEOUT; the next calls work."""
    import ctypes
    import time
    import torch
    from paper_1712_06913_b300 import _lib
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    _lib.check(_lib.load().muser_selftest_wait(1 << 27, ctypes.c_void_p(st.data_ptr()),
                                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    torch.cuda.synchronize()
    assert int(st[0]) == m.ST_TIMEOUT
    assert time.perf_counter() - t0 < 10.0
    # the context is usable: a CLEAN right after follows the oracle
    test_clean_threshold_and_abs_mode(m)


def test_image_with_steer_clean_end_to_end(m):
    """muser_image with Steer clean (clean_variant 1): cycles, residual and the restored image
    (residual + model map convolved with the fitted clean beam) against the oracle's dirty map,
    Steer cycles and restore of the model's pixels."""
    from oracle import restore as orest
    wl = synth.small_workload(n_ant=10, N=64, n_frame=2, config_id=263, bmax=300.0)
    cfg = cfg_for(m, wl, max_iter=12)
    cfg.clean_variant, cfg.steer_clip = 1, 0.9
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    out = m.image(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    ro = oracle_records(wl)
    for i in range(wl.n_inst):
        ri = geometry.instance_slice(ro, i, wl.n_bl)
        Do, Bo, _ = imaging.dirty_and_beam(imaging.grid(ri, wl.G, KER), wl.N, KER)
        Ro, Mo, co, gap = _oracle_steer_chain(Do, Bo, cfg.gain, 0.9, 12)
        assert gap > 3e-5, "the oracle run has a near-tie at its selection level"
        assert int(_np(out.n_comp)[i]) == co == 12
        peak = float(np.abs(Do).max())
        assert np.abs(_np(out.residual)[i] - Ro).max() <= 1e-4 * peak
        S = orest.clean_beam(Bo)
        np.testing.assert_allclose(_np(out.beam_params)[i], S, rtol=1e-5)
        nz = np.flatnonzero(Mo)
        Io = orest.restore(Ro, nz, Mo.ravel()[nz], S)
        assert np.abs(_np(out.clean)[i] - Io).max() <= 1e-4 * np.abs(Io).max()
