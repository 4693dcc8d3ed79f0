"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
invariant, a library routine that computes the same object another way, brute
force on a tiny input, or a value printed in the paper.
"""
import math
import os

import numpy as np
import pytest
from scipy.special import pro_ang1, pro_cv

import synth
from oracle import centering, clean, geometry, gmm, imaging, operator, pipeline, restore, steer
from oracle.pswf import Spheroidal

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
KER = pipeline.spheroidal(7, 1024)


# ----------------------------------------------------------------------------- geometry
def test_local_xyz_equator_and_pole():
    enu = np.array([[1.0, 2.0, 3.0]])
    # at the equator the pole axis is north and X points up (textbook frame)
    np.testing.assert_allclose(geometry.local_xyz(enu, 0.0), [[3.0, 1.0, 2.0]], atol=1e-15)
    # at the north pole, up is the pole axis and north points along -X
    np.testing.assert_allclose(geometry.local_xyz(enu, math.pi / 2), [[-2.0, 1.0, 3.0]], atol=1e-15)


def test_uvw_closed_form_pole_source():
    """H = 0, dec = 90 deg: (u, v, w) = (by, -bx, bz) / lambda."""
    rng = np.random.default_rng(1)
    enu = rng.normal(size=(6, 3)) * 500
    pairs = synth.baseline_pairs(6)
    lat = 0.7
    out = geometry.uvw(enu, pairs, lat, np.array([0.0]), np.array([math.pi / 2]), np.array([1.5e9]))
    xyz = geometry.local_xyz(enu, lat)
    b = xyz[pairs[:, 1]] - xyz[pairs[:, 0]]
    lam = geometry.C_LIGHT / 1.5e9
    exp = np.stack([b[:, 1], -b[:, 0], b[:, 2]], -1) / lam
    np.testing.assert_allclose(out[0, 0], exp, rtol=0, atol=1e-12 * np.abs(exp).max())


def test_uvw_rotation_invariance_and_source_direction():
    """|(u,v,w)| lambda = |b| for any H, dec; a baseline along the source has u = v = 0."""
    enu = synth.muser1_array()
    pairs = synth.baseline_pairs(40)
    ha = np.array([-1.0, 0.3, 2.0])
    dec = np.array([-0.25, 0.1, 1.2])
    freq = np.array([0.4e9, 2e9])
    out = geometry.uvw(enu, pairs, synth.MINGANTU_LAT, ha, dec, freq)
    xyz = geometry.local_xyz(enu, synth.MINGANTU_LAT)
    blen = np.linalg.norm(xyz[pairs[:, 1]] - xyz[pairs[:, 0]], axis=1)
    for c, f in enumerate(freq):
        lam = geometry.C_LIGHT / f
        np.testing.assert_allclose(np.linalg.norm(out[:, c], axis=-1) * lam, np.broadcast_to(blen, (3, len(blen))), rtol=1e-12)
    # baseline pointing at the source: X_j - X_i parallel to s0 = (cos d cos H, -cos d sin H, sin d)
    H, d = 0.4, 0.3
    s0 = np.array([math.cos(d) * math.cos(H), -math.cos(d) * math.sin(H), math.sin(d)])
    lat = 0.5
    # invert local_xyz: E = Y, N = cos(lat) Z - sin(lat) X, U = cos(lat) X + sin(lat) Z
    X, Y, Z = 1000 * s0
    enu2 = np.array([[0, 0, 0], [Y, math.cos(lat) * Z - math.sin(lat) * X, math.cos(lat) * X + math.sin(lat) * Z]])
    o = geometry.uvw(enu2, np.array([[0, 1]]), lat, np.array([H]), np.array([d]), np.array([geometry.C_LIGHT]))
    np.testing.assert_allclose(o[0, 0, 0], [0, 0, 1000], atol=1e-9)


def test_table2_resolution_and_pixel_rule():
    """Table 2: resolution = lambda / 3 km and three pixels per resolution element."""
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_resolution.txt"))
    arcsec = 180 * 3600 / math.pi
    for f, res, pix, exact in rows:
        ours = geometry.resolution(f * 1e9, 3000.0) * arcsec
        if exact:
            assert abs(ours - res) <= 0.08, (f, ours, res)
        assert abs(res / 3 - pix) <= 0.06, (f, res, pix)
        # with the FOV floor inactive the pixel rule is exactly resolution / 3
        p = geometry.pixel_size(f * 1e9, 3000.0, 1 << 20, 1e-9) * arcsec
        assert abs(p - ours / 3) < 1e-9


def test_pixel_floor():
    """Reading A5: the pixel is at least fov_min / N."""
    p = geometry.pixel_size(15e9, 3000.0, 1024, 60 * synth.ARCMIN)
    assert p == pytest.approx(60 * synth.ARCMIN / 1024)


# ----------------------------------------------------------------------------- spheroidal
def test_pswf_eigenvalue_matches_scipy_characteristic_value():
    for W in (5, 7, 9):
        k = Spheroidal(W, 256)
        assert k.eigenvalue == pytest.approx(pro_cv(0, 0, k.c), rel=1e-12)


def test_pswf_shape_matches_scipy_angular_function():
    eta = np.linspace(-0.99, 0.99, 41)
    s, _ = pro_ang1(0, 0, KER.c, eta)
    s0, _ = pro_ang1(0, 0, KER.c, 0.0)
    np.testing.assert_allclose(KER.psi(eta), s / s0, rtol=1e-7, atol=1e-9)


def test_pswf_finite_fourier_eigen_relation():
    """Transform of the truncated kernel = K gc(xi) (the grid correction is exact)."""
    t, wq = np.polynomial.legendre.leggauss(400)
    half = KER.W / 2
    d = t * half
    K = KER.integral()
    for xi in (0.0, 0.05, 0.125, 0.2, 0.25, 0.4):
        ft = np.sum(wq * KER.kernel_exact(d) * np.cos(2 * math.pi * d * xi)) * half
        gc = KER.psi(2 * xi)
        assert ft == pytest.approx(K * gc, rel=1e-10, abs=1e-13)


def test_kernel_table_interpolation_error():
    d = np.linspace(-3.5, 3.5, 10001)
    err = np.abs(KER.kernel(d) - KER.kernel_exact(d)).max()
    assert err < 2e-6
    assert KER.kernel(0.0) == 1.0
    assert KER.kernel(3.6) == 0.0


# ----------------------------------------------------------------------------- grid + image
def _tiny(N=32, n_ant=7, snr=30.0, seed_cfg=101, bmax=200.0):
    wl = synth.small_workload(n_ant=n_ant, N=N, config_id=seed_cfg, bmax=bmax, snr=snr)
    rec = pipeline.records(wl)
    return wl, rec


def test_grid_hermitian_visibility_part():
    """Z = Z_V + i Z_1 with Z_V Hermitian: its transform (the dirty map) is real."""
    wl, rec = _tiny(N=32)
    Z = imaging.grid(rec, wl.G, KER)
    G = wl.G
    assert np.all(Z[0, :] == 0) and np.all(Z[:, 0] == 0)
    Zm = np.zeros_like(Z)
    Zm[1:, 1:] = np.conj(Z[1:, 1:][::-1, ::-1])           # conj Z[G - k]
    ZV = (Z + Zm) / 2
    Z1 = (Z - Zm) / 2j
    I_V = imaging.centred_inverse_dft2(ZV)
    I_1 = imaging.centred_inverse_dft2(Z1)
    assert np.abs(I_V.imag).max() < 1e-12 * np.abs(I_V).max()
    assert np.abs(I_1.imag).max() < 1e-12 * np.abs(I_1).max()
    np.testing.assert_allclose(Z1.imag, 0, atol=1e-12 * np.abs(Z1).max())
    assert Z1.real.min() > -1e-12


def test_parseval():
    wl, rec = _tiny(N=32)
    Z = imaging.grid(rec, wl.G, KER)
    I = imaging.centred_inverse_dft2(Z)
    assert (np.abs(I) ** 2).sum() == pytest.approx(wl.G ** 2 * (np.abs(Z) ** 2).sum(), rel=1e-12)


def test_phase_centre_point_source():
    """Flat visibilities V = F: D is F times the central N x N of the beam; Bm(0) = 1."""
    wl, rec = _tiny(N=32, snr=0)
    rec = dict(rec)
    rec["vis"] = np.where(rec["w"] > 0, 2.5 + 0j, 0)
    Z = imaging.grid(rec, wl.G, KER)
    D, Bm, norm = imaging.dirty_and_beam(Z, wl.N, KER)
    N = wl.N
    assert Bm[N, N] == 1.0
    np.testing.assert_allclose(D, 2.5 * Bm[N // 2:N // 2 + N, N // 2:N // 2 + N], rtol=0, atol=1e-14 * 2.5)


def test_phase_rotation_moves_a_point_source_to_the_centre():
    """A unit point source (a, b) pixels from the phase centre has V = exp(-2 pi i (u l0 + v m0))
    with l0 = a cell, m0 = b cell; since l = (x - N/2) cell and m = (y - N/2) cell (the direct
    transform of the definition), its dirty map peaks at row N/2 + b, column N/2 + a.  Rotating
    each visibility by exp(+2 pi i (u l0 + v m0)) (Sec. 4.2, the phase correction of Alg. 1) makes
    it a source at the centre: the peak moves to (N/2, N/2) and the map is the beam's central
    N x N (V' = 1)."""
    wl, _ = _tiny(N=32, snr=0)
    N, G = wl.N, wl.G
    cell = pipeline.cell_sizes(wl)
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    a, b = 5, -3
    l0, m0 = a * cell[None, :, None], b * cell[None, :, None]
    V = np.exp(-2j * math.pi * (uvw[..., 0] * l0 + uvw[..., 1] * m0))
    flags = np.zeros(V.shape, np.uint8)
    F, C = V.shape[:2]
    dlm = np.stack([np.broadcast_to(a * cell, (F, C)), np.broadcast_to(b * cell, (F, C))], -1).reshape(F * C, 2)
    for rot, centre in ((None, (N // 2 + b, N // 2 + a)), (dlm, (N // 2, N // 2))):
        rec = geometry.grid_records(uvw, V, flags, cell, G, wl.W, rot)
        _, D, Bm, _ = pipeline.dirty(geometry.instance_slice(rec, 0, wl.n_bl), N, G, KER)
        assert np.unravel_index(np.argmax(D), D.shape) == centre
    np.testing.assert_allclose(D, Bm[N // 2:N // 2 + N, N // 2:N // 2 + N], rtol=0, atol=1e-12)


def test_dirty_beam_is_point_symmetric_about_its_centre():
    """Every sample is gridded at +uv and at -uv with the same weight (Sec. 3.2.3), so the beam
    part of the grid is real and even about the grid centre and so is its transform: over the
    2N x 2N beam, Bm(N + dy, N + dx) = Bm(N - dy, N - dx) (row and column 0 have no mirror
    inside the beam), and the largest value is the unit centre."""
    for N in (32, 40):
        wl, rec = _tiny(N=N, n_ant=9, seed_cfg=107)
        Z = imaging.grid(rec, wl.G, KER)
        _, Bm, _ = imaging.dirty_and_beam(Z, N, KER)
        A = Bm[1:, 1:]
        np.testing.assert_allclose(A, A[::-1, ::-1], rtol=0, atol=1e-12)
        assert Bm[N, N] == 1.0
        assert np.unravel_index(np.argmax(Bm), Bm.shape) == (N, N)


@pytest.mark.parametrize("N,n_ant,cfg", [(32, 7, 102), (64, 10, 103)])
def test_gridded_image_matches_direct_dft(N, n_ant, cfg):
    """Gridding + FFT + correction approximates the direct transform (reading A6 bound)."""
    wl, rec = _tiny(N=N, n_ant=n_ant, seed_cfg=cfg, bmax=40.0 * N / 32 * 5)
    Z = imaging.grid(rec, wl.G, KER)
    D, Bm, _ = imaging.dirty_and_beam(Z, N, KER)
    cell = pipeline.cell_sizes(wl)[0]
    Dd, Bd = imaging.direct_dirty(rec, N, cell)
    assert rec["w"].sum() >= 10
    assert np.abs(D - Dd).max() <= 2e-4 * np.abs(Dd).max()
    assert np.abs(Bm - Bd).max() <= 4e-4


@pytest.mark.parametrize("N,n_ant,cfg", [(32, 7, 105), (40, 9, 106)])
def test_gridded_image_at_5x2a_side_matches_direct_dft(N, n_ant, cfg):
    """Image sides 5 * 2^a (grids of 5 * 2^(a+2) cells, the 1280-5120 pixel images of Table 2):
    the same bound against the direct transform, and the sparse per-pixel evaluation equals the
    dense transform at sampled pixels."""
    wl, rec = _tiny(N=N, n_ant=n_ant, seed_cfg=cfg, bmax=40.0 * N / 32 * 5)
    Z = imaging.grid(rec, wl.G, KER)
    D, Bm, norm = imaging.dirty_and_beam(Z, N, KER)
    if N % 5 == 0:
        Dd, Bd = imaging.direct_dirty(rec, N, pipeline.cell_sizes(wl)[0])
        assert np.abs(D - Dd).max() <= 2e-4 * np.abs(Dd).max()
        assert np.abs(Bm - Bd).max() <= 4e-4
    rng = np.random.default_rng(cfg)
    dp = np.concatenate([rng.integers(0, N, (12, 2)), [[N // 2, N // 2], [0, 0], [N - 1, N - 1]]])
    bp = np.concatenate([rng.integers(0, 2 * N, (12, 2)), [[N, N], [0, 2 * N - 1]]])
    Ds, Bs, ns = imaging.dirty_and_beam_at(rec, wl.G, N, KER, dp, bp)
    assert ns == pytest.approx(norm, rel=1e-12)
    np.testing.assert_allclose(Ds, D[dp[:, 0], dp[:, 1]], rtol=0, atol=1e-10 * np.abs(D).max())
    np.testing.assert_allclose(Bs, Bm[bp[:, 0], bp[:, 1]], rtol=0, atol=1e-10)


def test_uniform_weights_matches_weighted_dft_and_sums_to_one_per_cell():
    wl, rec = _tiny(N=32, n_ant=10, seed_cfg=104, bmax=200.0)
    w = imaging.uniform_weights(rec, wl.G, wl.N)
    keep = rec["w"] > 0
    assert np.all(w[keep] > 0) and np.all(w[keep] <= 1) and np.all(w[~keep] == 0)
    assert np.any(w[keep] < 1)          # some cells hold several samples
    # every occupied N-grid cell carries total weight 1 (2 samples per visibility)
    N, G = wl.N, wl.G
    gN = (rec["ku"][keep] - rec["fu"][keep] - G / 2) / (G / N) + N / 2
    assert np.all(np.abs(gN - np.round(gN)) != 0.5)
    Z = imaging.grid(rec, G, KER, w)
    D, Bm, _ = imaging.dirty_and_beam(Z, N, KER)
    Dd, Bd = imaging.direct_dirty(rec, N, pipeline.cell_sizes(wl)[0], w)
    assert np.abs(D - Dd).max() <= 2e-4 * np.abs(Dd).max()
    assert np.abs(Bm - Bd).max() <= 4e-4


def test_uniform_weights_from_fp64_uv_cells():
    """Uniform weighting decided independently of the oracle's FP32 cell rule: the N-grid
    cell of every sample is taken in FP64 straight from (u, v) (cell = floor(u N cell_rad +
    N/2 + 1/2), the mirror at -u, -v), on inputs with no sample near a cell boundary.  Then
    every occupied cell carries total weight 1 and all its samples the same weight 1/count
    (Alg. 1 weighting mode; the count includes the -uv mirrors)."""
    wl, rec = _tiny(N=32, n_ant=10, seed_cfg=104, bmax=200.0)
    N, G = wl.N, wl.G
    w = imaging.uniform_weights(rec, G, N)
    keep = np.nonzero(rec["w"] > 0)[0]
    cell = pipeline.cell_sizes(wl)[0]
    u = rec["uvw"][keep, 0] * N * cell
    v = rec["uvw"][keep, 1] * N * cell
    for t in (u, v):
        frac = t - np.floor(t)
        assert np.all(np.abs(frac - 0.5) > 1e-6), "seeded input has a sample on an N-grid cell boundary"
    cu = np.floor(u + N / 2 + 0.5).astype(int)
    cv = np.floor(v + N / 2 + 0.5).astype(int)
    mu = np.floor(-u + N / 2 + 0.5).astype(int)
    mv = np.floor(-v + N / 2 + 0.5).astype(int)
    members = {}
    for j, i in enumerate(keep):
        members.setdefault((cv[j], cu[j]), []).append(w[i])
        members.setdefault((mv[j], mu[j]), []).append(w[i])
    assert any(len(ws) > 1 for ws in members.values())
    for key, ws in members.items():
        ws = np.asarray(ws)
        assert np.all(ws == ws[0]), key
        assert ws.sum() == pytest.approx(1.0, abs=1e-12), key


# ----------------------------------------------------------------------------- GMM
def test_gmm_recovers_known_mixture():
    rng = np.random.default_rng(5)
    mus, sig, n = [0.0, 5.0, 12.0], [1.0, 0.8, 1.5], [600_000, 300_000, 100_000]
    data = np.concatenate([rng.normal(m, s, k) for m, s, k in zip(mus, sig, n)])
    h, x, lo, width = gmm.histogram(data)
    mu, var, pi, it, _ = gmm.em(h, x, width)
    np.testing.assert_allclose(mu, mus, atol=0.01)
    np.testing.assert_allclose(np.sqrt(var), sig, rtol=0.02)
    np.testing.assert_allclose(pi, np.array(n) / sum(n), atol=0.005)
    assert h.sum() == data.size


def test_gmm_histogram_matches_numpy_and_affine_invariance():
    rng = np.random.default_rng(6)
    data = np.concatenate([rng.normal(0, 1, 50_000), rng.normal(4, 0.5, 20_000), rng.normal(9, 1, 5_000)])
    h, x, lo, width = gmm.histogram(data)
    hn, edges = np.histogram(data, bins=2000, range=(data.min(), data.max()))
    assert np.abs(h - hn).sum() <= 4          # edge rounding may move a sample by one bin
    a, b = 3.0, -2.0
    mu_a, mu_b, _ = gmm.sky_and_disk(data)
    mu_a2, mu_b2, _ = gmm.sky_and_disk(a * data + b)
    assert mu_a2 == pytest.approx(a * mu_a + b, abs=1e-6 * a)
    assert mu_b2 == pytest.approx(a * mu_b + b, abs=1e-6 * a)


# ----------------------------------------------------------------------------- CLEAN
def _beam(N, seed=7):
    wl = synth.small_workload(n_ant=10, N=N, config_id=seed, bmax=300.0, snr=0)
    rec = pipeline.records(wl)
    Z = imaging.grid(rec, wl.G, KER)
    _, Bm, _ = imaging.dirty_and_beam(Z, N, KER)
    return Bm


def test_hogbom_isolated_point_source_closed_form():
    N = 64
    Bm = _beam(N)
    F, py, px = 3.0, 20, 37
    D = F * Bm[N - py:2 * N - py, N - px:2 * N - px]
    n = 40
    R, pos, flux = clean.hogbom(D, Bm, 0.1, -np.inf, n)
    assert len(pos) == n and np.all(pos == py * N + px)
    assert R[py, px] == pytest.approx(F * 0.9 ** n, rel=1e-12)
    assert flux.sum() == pytest.approx(F * (1 - 0.9 ** n), rel=1e-12)
    np.testing.assert_allclose(flux, 0.1 * F * 0.9 ** np.arange(n), rtol=1e-12)
    # threshold: stops at the first peak <= thr
    R2, pos2, _ = clean.hogbom(D, Bm, 0.1, F * 0.9 ** 10 * 1.0000001, 1000)
    assert len(pos2) == 10


def test_hogbom_two_separated_sources():
    N = 64
    yy, xx = np.mgrid[-N:N, -N:N]
    Bm = np.exp(-(xx ** 2 + yy ** 2) / (2 * 1.5 ** 2))       # compact beam, no sidelobes
    D = 2.0 * Bm[N - 10:2 * N - 10, N - 12:2 * N - 12] + 1.0 * Bm[N - 50:2 * N - 50, N - 45:2 * N - 45]
    _, pos, flux = clean.hogbom(D, Bm, 0.1, 1e-3, 1000)
    assert set(pos.tolist()) == {10 * N + 12, 50 * N + 45}
    assert flux[pos == 10 * N + 12].sum() == pytest.approx(2.0, rel=2e-3)
    assert flux[pos == 50 * N + 45].sum() == pytest.approx(1.0, rel=2e-3)


def test_hogbom_tie_break_and_abs_mode():
    N = 8
    Bm = np.zeros((2 * N, 2 * N))
    Bm[N, N] = 1.0
    D = np.zeros((N, N))
    D[2, 5] = D[1, 6] = 1.0
    D[3, 3] = -2.0
    _, pos, _ = clean.hogbom(D, Bm, 0.5, 0.0, 1)
    assert pos[0] == 1 * N + 6                 # lowest row-major index among equal peaks
    _, pos, flux = clean.hogbom(D, Bm, 0.5, 0.0, 1, peak_mode=1)
    assert pos[0] == 3 * N + 3 and flux[0] == -1.0


# ----------------------------------------------------------------------------- restore
# ----------------------------------------------------------------------------- Steer clean
def test_steer_beam_convolution_fft_equals_bruteforce():
    rng = np.random.default_rng(3)
    N = 12
    Bm = rng.normal(size=(2 * N, 2 * N))
    C = np.where(rng.uniform(size=(N, N)) < 0.2, rng.normal(size=(N, N)), 0.0)
    np.testing.assert_allclose(steer.convolve_beam(C, Bm), steer.convolve_beam_bruteforce(C, Bm), atol=1e-12)


def test_steer_with_clip_one_is_hogbom():
    """clip = 1 keeps the peak alone: every cycle is one Hogbom step with the same gain."""
    wl = synth.small_workload(n_ant=10, N=32, config_id=131, bmax=300.0)
    _, D, Bm, _ = pipeline.dirty(pipeline.records(wl), 32, 128, KER)
    R_h, pos, flux = clean.hogbom(D, Bm, 0.1, -np.inf, 25)
    R_s, model, cycles = steer.steer(D, Bm, 0.1, -np.inf, 25, clip=1.0)
    assert cycles == 25
    expect = np.zeros_like(D)
    np.add.at(expect.ravel(), pos, flux)
    np.testing.assert_allclose(model, expect, atol=1e-12 * np.abs(D).max())
    np.testing.assert_allclose(R_s, R_h, atol=1e-12 * np.abs(D).max())


def test_steer_linear_invariant_and_threshold():
    """D = R + Bm * model after any number of cycles; the stop rule is the peak threshold."""
    wl = synth.small_workload(n_ant=12, N=32, config_id=132, bmax=300.0)
    _, D, Bm, _ = pipeline.dirty(pipeline.records(wl), 32, 128, KER)
    R, model, cycles = steer.steer(D, Bm, 0.1, -np.inf, 30, clip=0.9)
    assert cycles == 30 and np.count_nonzero(model) > 30      # several pixels per cycle
    np.testing.assert_allclose(R + steer.convolve_beam(model, Bm), D, atol=1e-10 * np.abs(D).max())
    thr = 0.5 * D.max()
    R2, _, c2 = steer.steer(D, Bm, 0.1, thr, 1000, clip=0.9)
    assert R2.max() <= thr and c2 > 0
    # every cycle removes gain times the peak at most (the scaling of the subtraction)
    Rp, _, _ = steer.steer(D, Bm, 0.1, -np.inf, 1, clip=0.9)
    assert (D - Rp).max() == pytest.approx(0.1 * D.max(), rel=1e-12)


def test_clean_beam_of_exact_gaussian():
    """The moment fit returns the covariance of a sampled Gaussian beam; the pixel
    lattice's boundary error shrinks with the lobe area (about 9 % at 27 pixels,
    under 0.5 % at 1000 pixels)."""
    N = 96
    yy, xx = np.mgrid[-N:N, -N:N]
    for S, tol in (((400.0, 50.0, 300.0), 0.005), ((9.0, 2.5, 5.0), 0.10)):
        Bm = restore.gaussian(S, xx, yy)
        got = np.array(restore.clean_beam(Bm))
        scale = np.array([S[0], math.sqrt(S[0] * S[2]), S[2]])
        assert np.all(np.abs(got - S) <= tol * scale), (S, got)
        lobe = restore.main_lobe(Bm)
        assert lobe[N, N] and not lobe[0, 0]


def test_restore_point_component():
    N = 32
    R = np.zeros((N, N))
    S = (2.0, 0.3, 1.5)
    img = restore.restore(R, np.array([5 * N + 7, 5 * N + 7]), np.array([1.0, 0.5]), S)
    assert img[5, 7] == pytest.approx(1.5)
    # one pixel east: exp(-(Sinv_xx) / 2) with Sinv_xx = Syy / det
    det = S[0] * S[2] - S[1] ** 2
    assert img[5, 8] == pytest.approx(1.5 * math.exp(-0.5 * S[2] / det))
    assert img[6, 7] == pytest.approx(1.5 * math.exp(-0.5 * S[0] / det))


# ----------------------------------------------------------------------------- centring
def test_correlation_fft_equals_bruteforce():
    rng = np.random.default_rng(3)
    M = (rng.uniform(size=(24, 24)) > 0.7).astype(float)
    S = centering.disk_model(24, 5.0)
    M = M * rng.uniform(size=M.shape)
    np.testing.assert_allclose(centering.correlation(M, S, 6), centering.correlation_bruteforce(M, S, 6), atol=1e-10)


def test_centering_shift_of_a_displaced_disk_and_parabolic_peak():
    """Cc(s) = sum_p M(p) S(p - s) is largest where the mask's disk sits (Sec. 4.2 step 2): a model
    disk moved by 4 columns and -3 rows gives the shift (4, -3) (x along columns, y along rows),
    the parabolic refinement adding nothing at the symmetric peak; on samples of a quadratic bowl
    whose top is at (2.3, -1.4) the three-point parabolas recover the fractional parts exactly."""
    N, smax = 48, 12
    S = centering.disk_model(N, 9.0)
    M = np.roll(np.roll(S, -3, axis=0), 4, axis=1)
    assert centering.best_shift(centering.correlation(M, S, smax), smax) == (4.0, -3.0)
    yy, xx = np.mgrid[0:2 * smax + 1, 0:2 * smax + 1] - smax
    sx, sy = centering.best_shift(-((xx - 2.3) ** 2) - 0.5 * (yy + 1.4) ** 2, smax)
    assert sx == pytest.approx(2.3, abs=1e-12) and sy == pytest.approx(-1.4, abs=1e-12)


@pytest.mark.slow
@pytest.mark.parametrize("off_px", [(0, 0), (9.0, -6.0), (-15.0, 12.0), (3.4, -7.7)])
def test_centering_recovers_known_disk_offset(off_px):
    """A quiet-Sun disk displaced by a known offset is found within 0.25 px and
    re-centred by the phase correction (noise at SNR 30, no bursts)."""
    N = 128
    wl0 = synth.small_workload(n_ant=31, N=N, config_id=110, bmax=600.0, snr=0)
    cell = pipeline.cell_sizes(wl0)[0]
    lm = (off_px[0] * cell, off_px[1] * cell)
    sky = synth.Sky(disk_lm=lm)
    wl = synth.make_workload("c", wl0.ant_enu, wl0.pairs, wl0.ha, wl0.dec, wl0.freq, N, 4 * N,
                             config_id=110, skies=[sky], snr=30, bmax=600.0)
    rec = pipeline.records(wl)
    _, D, Bm, _ = pipeline.dirty(rec, N, 4 * N, KER)
    mu_a, mu_b, _ = gmm.sky_and_disk(D)
    dl, dm, ra, de, M = centering.disk_offset(D, Bm, mu_a, mu_b, cell, wl.dec[0])
    assert abs(dl / cell - off_px[0]) <= 0.25 and abs(dm / cell - off_px[1]) <= 0.25
    # after the phase correction the disk is centred: the brightness-weighted centroid
    # of the points above the sky/disk midpoint sits at the image centre
    rec2 = pipeline.records(wl, dlm=np.array([[dl, dm]]))
    _, D2, _, _ = pipeline.dirty(rec2, N, 4 * N, KER)
    Mv = np.where(D2 > 0.5 * (mu_a + mu_b), D2, 0.0)
    yy, xx = np.mgrid[0:N, 0:N]
    cx = (Mv * (xx - N // 2)).sum() / Mv.sum()
    cy = (Mv * (yy - N // 2)).sum() / Mv.sum()
    assert abs(cx) <= 0.25 and abs(cy) <= 0.25, (cx, cy)


# ----------------------------------------------------------------------------- operator
def _op_case(N=32, seed=120, n_chan=3):
    wl = synth.small_workload(n_ant=7, N=N, config_id=seed, bmax=150.0, freq=np.linspace(1.0e9, 1.6e9, n_chan))
    G = 2 * N
    cell = np.full(wl.n_chan, geometry.pixel_size(wl.freq.max(), wl.bmax, N, 60 * synth.ARCMIN))
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    rec = geometry.grid_records(uvw, wl.vis, wl.flags, cell, G, 7)
    return wl, rec, G, cell[0]


def test_operator_dot_product_adjoint():
    N = 32
    wl, rec, G, cell = _op_case(N)
    rng = np.random.default_rng(0)
    x = rng.normal(size=(N, N))
    y = (rng.normal(size=len(rec["w"])) + 1j * rng.normal(size=len(rec["w"]))) * rec["w"]
    lhs = np.vdot(y, operator.forward(x, rec, N, G, KER))
    rhs = np.vdot(operator.adjoint(y, rec, N, G, KER), x.astype(complex))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_operator_matches_direct_transform():
    N = 32
    wl, rec, G, cell = _op_case(N)
    rng = np.random.default_rng(1)
    x = rng.uniform(size=(N, N))
    A = operator.forward(x, rec, N, G, KER)
    Dx = operator.direct(x, rec, N, cell)
    keep = rec["w"] > 0
    assert keep.sum() > 20
    assert np.abs(A - Dx)[keep].max() <= 5e-4 * np.abs(Dx[keep]).max()


def test_chi2_gradient_finite_differences():
    N = 32
    wl, rec, G, cell = _op_case(N)
    V = rec["vis"]
    rng = np.random.default_rng(2)
    x = rng.uniform(size=(N, N)) * 0.01
    sigma = 0.3
    _, g = operator.chi2_grad(x, rec, V, sigma, N, G, KER)
    h = 1e-3
    for p in rng.choice(N * N, 16, replace=False):
        e = np.zeros(N * N)
        e[p] = h
        e = e.reshape(N, N)
        cp, _ = operator.chi2_grad(x + e, rec, V, sigma, N, G, KER)
        cm, _ = operator.chi2_grad(x - e, rec, V, sigma, N, G, KER)
        fd = (cp - cm) / (2 * h)
        assert fd == pytest.approx(g.ravel()[p], rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_chi2_with_fractional_weights():
    """The chi-square is linear in the weights, sum_k w_k |A x - V_k|^2 / sigma^2, for any weights
    (uniform weighting makes them fractional): at x = 0 it is sum_k w_k |V_k|^2 / sigma^2, and its
    gradient is the central finite difference of the loss with those weights."""
    N = 32
    wl, rec, G, cell = _op_case(N)
    rng = np.random.default_rng(5)
    r = dict(rec)
    r["w"] = np.where(rec["w"] > 0, rng.uniform(0.1, 1.0, size=len(rec["w"])), 0.0)
    V = rec["vis"]
    sigma = 0.7
    c0, _ = operator.chi2_grad(np.zeros((N, N)), r, V, sigma, N, G, KER)
    assert c0 == pytest.approx(float((r["w"] * np.abs(V) ** 2).sum()) / sigma ** 2, rel=1e-12)
    x = rng.uniform(size=(N, N)) * 0.01
    _, g = operator.chi2_grad(x, r, V, sigma, N, G, KER)
    h = 1e-3
    for p in rng.choice(N * N, 8, replace=False):
        e = np.zeros(N * N)
        e[p] = h
        e = e.reshape(N, N)
        cp, _ = operator.chi2_grad(x + e, r, V, sigma, N, G, KER)
        cm, _ = operator.chi2_grad(x - e, r, V, sigma, N, G, KER)
        assert (cp - cm) / (2 * h) == pytest.approx(g.ravel()[p], rel=1e-6, abs=1e-9 * np.abs(g).max())


def test_gradient_at_zero_is_scaled_dirty_image():
    """grad chi2(0) = -(2 sum w / sigma^2) D_dft (the dirty image is the adjoint)."""
    N = 32
    wl, rec, G, cell = _op_case(N)
    sigma = 0.5
    _, g = operator.chi2_grad(np.zeros((N, N)), rec, rec["vis"], sigma, N, G, KER)
    Dd, _ = imaging.direct_dirty(rec, N, cell)
    scale = -2 * rec["w"].sum() / sigma ** 2
    assert np.abs(g - scale * Dd).max() <= 1e-3 * np.abs(scale * Dd).max()


def test_gradient_descent_decreases_chi2():
    N = 32
    wl, rec, G, cell = _op_case(N)
    x, hist = operator.gradient_descent(rec, rec["vis"], 0.5, N, G, KER, steps=15)
    assert np.all(np.diff(hist) <= 1e-9 * hist[0])
    assert hist[-1] < 0.5 * hist[0]


def _hessian_from_gradients(rec, N, G, sigma):
    """Dense Hessian of chi2 on a tiny image, column j = grad(e_j) - grad(0) (chi2 is
    quadratic, so this is exact up to rounding; the gradient itself is pinned by finite
    differences of chi2 above)."""
    g0 = operator.chi2_grad(np.zeros((N, N)), rec, rec["vis"], sigma, N, G, KER)[1].ravel()
    H = np.zeros((N * N, N * N))
    for j in range(N * N):
        e = np.zeros(N * N)
        e[j] = 1.0
        H[:, j] = operator.chi2_grad(e.reshape(N, N), rec, rec["vis"], sigma, N, G, KER)[1].ravel() - g0
    return H


def _tiny_operator(N=8):
    wl = synth.small_workload(n_ant=7, N=N, config_id=122, bmax=20.0, freq=np.linspace(1.0e9, 1.6e9, 3))
    G = 2 * N
    cell = np.full(wl.n_chan, geometry.pixel_size(wl.freq.max(), wl.bmax, N, 60 * synth.ARCMIN))
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    rec = geometry.grid_records(uvw, wl.vis, wl.flags, cell, G, 7)
    assert (rec["w"] > 0).sum() >= 40
    return rec, G


def test_lipschitz_is_the_largest_hessian_eigenvalue():
    """The step size of gradient imaging, eta = 1/L: L from power iteration equals the largest
    eigenvalue of the dense chi2 Hessian (numpy eigvalsh) on an 8 x 8 image."""
    N, sigma = 8, 0.7
    rec, G = _tiny_operator(N)
    H = _hessian_from_gradients(rec, N, G, sigma)
    assert np.abs(H - H.T).max() <= 1e-9 * np.abs(H).max()      # a Hessian is symmetric
    ev = np.linalg.eigvalsh(0.5 * (H + H.T))
    assert ev[0] >= -1e-9 * ev[-1]                              # and positive semi-definite
    L = operator.lipschitz(rec, N, G, KER, sigma, iters=120)
    assert L == pytest.approx(ev[-1], rel=1e-10)


# ----------------------------------------------------------------------------- w-projection
def _wterm_case(Ww=15):
    wl = synth.wterm_workload()
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    rec = geometry.grid_records(uvw, wl.vis, wl.flags, pipeline.cell_sizes(wl), wl.G, Ww)
    return wl, rec


def test_wproj_plane0_kernel_is_the_spheroidal():
    """k_0 (no w) transforms back to the spheroidal kernel up to its aliasing (Sec. 3.2.3)."""
    from oracle import wproj
    tabs = wproj.kernel_tables(10.0, 8, 15, 1024, KER)
    d = np.arange(tabs.shape[1]) / 1024
    assert np.abs(tabs[0].imag).max() < 1e-14
    assert np.abs(tabs[0] - KER.kernel(d)).max() <= 3e-4
    # tabulated kernel as a function of wg: only the first plane is real
    assert np.abs(tabs[1].imag).max() > 1e-3


def test_wproj_kernel_image_plane_is_screen_times_correction():
    """The transform of k_p over its support is gc(xi) exp(-i pi wg_p xi^2) (normalised) inside
    the band that the kernel support resolves."""
    from oracle import wproj
    P, Ww, OS, wgmax = 5, 21, 256, 8.0
    tabs = wproj.kernel_tables(wgmax, P, Ww, OS, KER)
    d = np.arange(-(Ww // 2) * OS, (Ww // 2) * OS + 1) / OS
    xi = np.linspace(-0.35, 0.35, 15)
    g_norm = np.sum(np.polynomial.legendre.leggauss(256)[1] * 0.5 * KER.psi(np.polynomial.legendre.leggauss(256)[0]))
    for p in range(P):
        k = wproj.lookup(tabs[p], OS, d)
        ft = (k[None, :] * np.exp(2j * np.pi * np.outer(xi, d))).sum(1) / OS
        want = KER.psi(2 * xi) * np.exp(-1j * np.pi * p * wgmax / (P - 1) * xi * xi) / g_norm
        assert np.abs(ft - want).max() <= 2e-3, p


def test_wproj_dirty_matches_direct_transform_with_w():
    """Far from transit (|w| up to 1550 wavelengths, phase error ~1 rad at the field edge) the
    w-projected map and beam follow the direct transform with the w-term; 2-D gridding
    does not (Sec. 6.1)."""
    from oracle import wproj
    wl, rec = _wterm_case()
    assert np.abs(rec["uvw"][:, 2]).max() > 1000
    wgmax = np.abs(rec["wg"]).max()
    tabs = wproj.kernel_tables(wgmax, 128, 15, 1024, KER)
    Z = wproj.grid(rec, wl.G, tabs, wgmax, 15, 1024)
    D, Bm, _ = imaging.dirty_and_beam(Z, wl.N, KER)
    Dd, Bd = wproj.direct_dirty_w(rec, wl.N, pipeline.cell_sizes(wl)[0])
    err_d = np.abs(D - Dd).max() / np.abs(Dd).max()
    err_b = np.abs(Bm - Bd).max()
    assert err_d <= 5e-4 and err_b <= 2.5e-3
    D2, B2, _ = imaging.dirty_and_beam(imaging.grid(rec, wl.G, KER), wl.N, KER)
    assert np.abs(D2 - Dd).max() / np.abs(Dd).max() > 20 * 5e-4
    assert np.abs(B2 - Bd).max() > 20 * 2.5e-3
    # map and beam are real transforms of Hermitian grids
    G = wl.G
    ZV = 0.5 * (Z + np.conj(Z[(-np.arange(G)) % G][:, (-np.arange(G)) % G]))
    I = imaging.centred_inverse_dft2(ZV)
    assert np.abs(I.imag).max() <= 1e-9 * np.abs(I.real).max()


def test_wproj_zero_w_is_plain_gridding_with_plane0():
    """With every w = 0 the w-projected grid is the 2-D grid of the plane-0 kernel, which is the
    spheroidal up to its aliasing."""
    from oracle import wproj
    wl, rec = _wterm_case(Ww=7)
    rec = dict(rec)
    rec["wg"] = np.zeros_like(rec["wg"])
    tabs = wproj.kernel_tables(5.0, 16, 7, 1024, KER)
    Z = wproj.grid(rec, wl.G, tabs, 5.0, 7, 1024)
    Z0 = imaging.grid(rec, wl.G, KER)
    assert np.abs(Z - Z0).max() <= 1e-3 * np.abs(Z0).max()
