"""Seeded synthetic MUSER workloads: array geometry, observing set-up and visibilities.

This module produces INPUTS only. It is shared by the test-suite, the benchmark and
the CPU oracle's callers, and it holds none of the imaging method's arithmetic: no
(u, v, w) formula, no gridding, no kernel, no FFT, no CLEAN.

To evaluate the analytic sky (a uniform solar disk plus Gaussian bursts) it needs the
projection of each baseline on the sky plane.  It builds that projection with vector
algebra (cross products of the pole and the phase-centre direction), so neither the
oracle nor the GPU path can inherit a mistake from it: both recompute (u, v, w) from the
raw antenna positions, hour angles and declinations handed to them.

Parameters follow the paper's instrument description (Table 1, Sec. 1: 40 antennas for
MUSER-I at 0.4-2 GHz in 64 channels of 25 MHz with 25 ms time resolution; 60 antennas for
MUSER-II at 2-15 GHz in 33 bands of 16 channels with 206.25 ms resolution; baselines of
a few metres to about 3 km) and the site latitude of Sec. 3.2.2.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy.special import j1

C_LIGHT = 299_792_458.0
ARCSEC = math.pi / (180.0 * 3600.0)
ARCMIN = 60.0 * ARCSEC
MINGANTU_LAT = math.radians(42.211833333)      # Sec. 3.2.2 site latitude
SUN_RADIUS = 16.0 * ARCMIN
EARTH_RATE = 7.2921e-5                          # rad / s
SEED_ROOT = 1712


# --------------------------------------------------------------------------- array
def spiral_array(n_ant: int, r0: float, centre: bool, bmax: float = 3000.0) -> np.ndarray:
    """ENU positions (metres, U = 0) of a 3-arm logarithmic spiral.

    Arms start at 0, 120 and 240 degrees; on each arm the radii grow geometrically
    from r0 to R and the angle turns by ln(r/r0)/ln(R/r0) radians, so the outermost
    antennas of two arms are 120 degrees apart and the longest baseline is R*sqrt(3).
    The array is finally scaled so that the longest baseline is exactly ``bmax``.
    """
    per_arm = (n_ant - 1) // 3 if centre else n_ant // 3
    if 3 * per_arm + (1 if centre else 0) != n_ant:
        raise ValueError("n_ant must be 3k (+1 with a centre antenna)")
    R = bmax / math.sqrt(3.0)
    pos = [(0.0, 0.0)] if centre else []
    for arm in range(3):
        a0 = arm * 2.0 * math.pi / 3.0
        for k in range(per_arm):
            r = r0 * (R / r0) ** (k / (per_arm - 1))
            ang = a0 + math.log(r / r0) / math.log(R / r0)
            pos.append((r * math.cos(ang), r * math.sin(ang)))
    enu = np.zeros((n_ant, 3))
    enu[:, :2] = np.asarray(pos)
    d = enu[:, None, :] - enu[None, :, :]
    enu *= bmax / np.sqrt((d ** 2).sum(-1)).max()
    return enu


def baseline_pairs(n_ant: int) -> np.ndarray:
    """(i, j) with i < j in lexicographic order, int32 [n_ant*(n_ant-1)/2, 2]."""
    i, j = np.triu_indices(n_ant, k=1)
    return np.stack([i, j], -1).astype(np.int32)


def muser1_channels() -> np.ndarray:
    """64 channel centres over 0.4-2.0 GHz (25 MHz channels), Hz."""
    return (0.4125 + 0.025 * np.arange(64)) * 1e9


def muser2_channels() -> np.ndarray:
    """528 channel centres: 33 bands of 16 x 25 MHz over 2-15 GHz, Hz.

    Bands 0..31 start at 2.0 + 0.4 b GHz; band 32 starts at 14.6 GHz, so its first
    8 channels repeat the last 8 of band 31 (the paper notes 8 repeated channels).
    """
    starts = [2.0 + 0.4 * b for b in range(32)] + [14.6]
    return np.array([(s + 0.025 * (k + 0.5)) * 1e9 for s in starts for k in range(16)])


# --------------------------------------------------------------------------- sky
@dataclasses.dataclass
class Sky:
    """Analytic sky for one frame: uniform disk + circular Gaussian bursts (SFU)."""
    disk_radius: float = SUN_RADIUS
    disk_flux: float = 1.0
    disk_lm: tuple = (0.0, 0.0)
    burst_lm: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros((0, 2)))
    burst_sigma: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))
    burst_flux: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(0))


def draw_sky(rng: np.random.Generator, n_bursts: int = 3, disk_lm=(0.0, 0.0)) -> Sky:
    """Bursts: sigma ~ U[20", 60"], flux ~ U[0.1, 2] SFU, centre uniform in 0.8 r_disk."""
    r = 0.8 * SUN_RADIUS * np.sqrt(rng.uniform(size=n_bursts))
    t = rng.uniform(0, 2 * math.pi, size=n_bursts)
    lm = np.stack([r * np.cos(t), r * np.sin(t)], -1) + np.asarray(disk_lm)[None, :]
    return Sky(disk_lm=tuple(disk_lm), burst_lm=lm,
               burst_sigma=rng.uniform(20.0, 60.0, size=n_bursts) * ARCSEC,
               burst_flux=rng.uniform(0.1, 2.0, size=n_bursts))


def _sky_plane_projection(ant_enu, pairs, lat, ha, dec, freq, with_w=False):
    """Baseline projections (u, v) in wavelengths via the sky-plane basis vectors.

    The local frame is expressed in equatorial axes (x: meridian on the equator,
    y: east, z: pole); the phase centre s0 points to (ha, dec); e_u = unit(z x s0)
    and e_v = s0 x e_u.  Returns u, v of shape [F, C, n_bl] (and w = b . s0 with with_w).
    """
    east = np.array([0.0, 1.0, 0.0])
    north = np.array([-math.sin(lat), 0.0, math.cos(lat)])
    up = np.array([math.cos(lat), 0.0, math.sin(lat)])
    basis = np.stack([east, north, up])                     # rows: E, N, U in eq. axes
    ant_eq = ant_enu @ basis
    b = ant_eq[pairs[:, 1]] - ant_eq[pairs[:, 0]]            # [nb, 3] metres
    F, C = len(ha), len(freq)
    u = np.empty((F, C, len(pairs)))
    v = np.empty_like(u)
    w = np.empty_like(u)
    zhat = np.array([0.0, 0.0, 1.0])
    for f in range(F):
        s0 = np.array([math.cos(dec[f]) * math.cos(-ha[f]),
                       math.cos(dec[f]) * math.sin(-ha[f]),
                       math.sin(dec[f])])
        eu = np.cross(zhat, s0)
        eu /= np.linalg.norm(eu)
        ev = np.cross(s0, eu)
        bu, bv = b @ eu, b @ ev
        inv_lam = freq / C_LIGHT
        u[f] = inv_lam[:, None] * bu[None, :]
        v[f] = inv_lam[:, None] * bv[None, :]
        w[f] = inv_lam[:, None] * (b @ s0)[None, :]
    return (u, v, w) if with_w else (u, v)


def sky_visibilities(sky: Sky, u: np.ndarray, v: np.ndarray) -> np.ndarray:
    """Noise-free visibilities V(u, v) = sum of component transforms (e^{-2 pi i (ul+vm)})."""
    q = np.hypot(u, v)
    x = 2 * math.pi * q * sky.disk_radius
    with np.errstate(invalid="ignore", divide="ignore"):
        disk = np.where(x > 1e-12, 2.0 * j1(x) / np.where(x > 1e-12, x, 1.0), 1.0)
    l0, m0 = sky.disk_lm
    V = sky.disk_flux * disk * np.exp(-2j * math.pi * (u * l0 + v * m0))
    for (lb, mb), s, S in zip(sky.burst_lm, sky.burst_sigma, sky.burst_flux):
        V = V + S * np.exp(-2 * math.pi ** 2 * s ** 2 * q ** 2) * np.exp(-2j * math.pi * (u * lb + v * mb))
    return V


def point_visibilities_w(points, u, v, w):
    """Noise-free visibilities of point sources [(l, m, flux), ...] with the w-term:
    V = sum_j F_j exp(-2 pi i (u l_j + v m_j + w (n_j - 1))), n_j = sqrt(1 - l_j^2 - m_j^2)."""
    V = np.zeros(np.shape(u), np.complex128)
    for l, m, f in points:
        n = math.sqrt(1.0 - l * l - m * m)
        V = V + f * np.exp(-2j * math.pi * (u * l + v * m + w * (n - 1.0)))
    return V


# --------------------------------------------------------------------------- workloads
@dataclasses.dataclass
class Workload:
    """Everything the imaging path consumes for one batch of (frame, channel) instances.

    Instance index = frame * n_chan + chan.  ``vis`` and ``flags`` are
    [n_frame, n_chan, n_bl]; a flag of 1 marks a baseline that must not be imaged.
    """
    name: str
    ant_enu: np.ndarray        # [n_ant, 3] f64 metres (east, north, up)
    pairs: np.ndarray          # [n_bl, 2] int32
    lat: float                 # rad
    ha: np.ndarray             # [n_frame] f64 rad
    dec: np.ndarray            # [n_frame] f64 rad
    freq: np.ndarray           # [n_chan] f64 Hz
    vis: np.ndarray            # [n_frame, n_chan, n_bl] complex64
    flags: np.ndarray          # [n_frame, n_chan, n_bl] uint8
    N: int                     # image side
    G: int                     # uv grid side
    bmax: float = 3000.0       # longest baseline (m), for the pixel-size rule
    fov_min: float = 60.0 * ARCMIN   # smallest field of view, for the pixel-size rule
    W: int = 7
    OS: int = 1024
    gain: float = 0.1
    max_iter: int = 200
    thr_mode: int = 0          # 0: fixed threshold (-inf), 1: GMM sky level
    skies: list = dataclasses.field(default_factory=list)

    @property
    def n_frame(self): return len(self.ha)

    @property
    def n_chan(self): return len(self.freq)

    @property
    def n_bl(self): return len(self.pairs)

    @property
    def n_inst(self): return self.n_frame * self.n_chan


def make_workload(name, ant_enu, pairs, ha, dec, freq, N, G, *, config_id, skies=None,
                  flag_max=0.0, snr=30.0, frames_redraw=True, disk_lm=(0.0, 0.0),
                  lat=MINGANTU_LAT, **kw) -> Workload:
    """Seeded visibilities for every (frame, channel): sky + complex Gaussian noise.

    Seeds: bursts of frame f from SeedSequence([1712, config_id, f]); flags of frame f
    from SeedSequence([1712, config_id, f, 1 << 20]); noise of (f, c) from
    SeedSequence([1712, config_id, f, c]); all PCG64.  The noise has
    sigma_c = rms|V_model| / snr per instance, split evenly between Re and Im.
    """
    F, C = len(ha), len(freq)
    nb = len(pairs)
    u, v = _sky_plane_projection(ant_enu, pairs, lat, ha, dec, freq)
    vis = np.empty((F, C, nb), np.complex64)
    flags = np.zeros((F, C, nb), np.uint8)
    if skies is None:
        skies = []
        for f in range(F):
            rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id, f if frames_redraw else 0])))
            skies.append(draw_sky(rng, disk_lm=disk_lm))
    for f in range(F):
        Vm = sky_visibilities(skies[f], u[f], v[f])                 # [C, nb]
        if flag_max > 0:
            rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id, f, 1 << 20])))
            frac = rng.uniform(0.0, flag_max)
            sel = rng.permutation(nb)[: int(round(frac * nb))]
            flags[f, :, sel] = 1
        for c in range(C):
            rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id, f, c])))
            sig = math.sqrt(np.mean(np.abs(Vm[c]) ** 2)) / snr if snr else 0.0
            noise = rng.normal(size=(nb, 2)) * (sig / math.sqrt(2.0))
            vis[f, c] = (Vm[c] + noise[:, 0] + 1j * noise[:, 1]).astype(np.complex64)
    return Workload(name=name, ant_enu=ant_enu, pairs=pairs, lat=lat, ha=np.asarray(ha, float),
                    dec=np.asarray(dec, float), freq=np.asarray(freq, float), vis=vis,
                    flags=flags, N=N, G=G, skies=skies, **kw)


DEC_SUN = math.radians(-14.3)


def muser1_array():
    return spiral_array(40, 8.0, centre=True)


def muser2_array():
    return spiral_array(60, 4.0, centre=False)


def config1_plain_frame() -> Workload:
    """One frame, 40 antennas (780 baselines), 1 channel at 1.7 GHz, N = 256, 200 iterations."""
    ant = muser1_array()
    return make_workload("plain-1frame-N256", ant, baseline_pairs(40), np.array([0.0]),
                         np.array([DEC_SUN]), np.array([1.7e9]), 256, 1024, config_id=1,
                         max_iter=200)


def config2_muser1_band(n_frame=32, chans=None) -> Workload:
    """MUSER-I band: 64 channels x 32 frames of 25 ms, N = 512, GMM threshold, cap 1000."""
    ant = muser1_array()
    freq = muser1_channels() if chans is None else muser1_channels()[chans]
    ha = EARTH_RATE * 0.025 * np.arange(n_frame)
    return make_workload("muser1-band-N512", ant, baseline_pairs(40), ha,
                         np.full(n_frame, DEC_SUN), freq, 512, 2048, config_id=2,
                         max_iter=1000, thr_mode=1)


def config3_muser2_uneven(n_frame=8, chans=None) -> Workload:
    """MUSER-II: 528 channels x 8 frames of 206.25 ms, 60 antennas (1770 baselines),
    0-30 % of baselines flagged per frame, N = 1024, 1000 iterations."""
    ant = muser2_array()
    freq = muser2_channels() if chans is None else muser2_channels()[chans]
    ha = EARTH_RATE * 0.20625 * np.arange(n_frame)
    return make_workload("muser2-uneven-N1024", ant, baseline_pairs(60), ha,
                         np.full(n_frame, DEC_SUN), freq, 1024, 4096, config_id=3,
                         flag_max=0.3, max_iter=1000)


LARGE_BANDS = {1280: (2.0e9, 4.0e9), 2560: (4.0e9, 8.0e9), 5120: (8.0e9, 15.0e9)}


def muser2_large_band(N=2560, n_frame=1, chans=None) -> Workload:
    """MUSER-II high-band images of Table 2: 2-4 GHz at 1280^2, 4-8 GHz at 2560^2, 8-15 GHz at
    5120^2 (G = 4N), 60 antennas, 0-30 % of baselines flagged per frame, 1000 iterations.
    ``chans`` indexes the channels of the band."""
    lo, hi = LARGE_BANDS[N]
    allf = muser2_channels()
    band = allf[(allf >= lo) & (allf <= hi)]
    freq = band if chans is None else band[chans]
    ant = muser2_array()
    ha = EARTH_RATE * 0.20625 * np.arange(n_frame)
    return make_workload(f"muser2-band-N{N}", ant, baseline_pairs(60), ha, np.full(n_frame, DEC_SUN), freq,
                         N, 4 * N, config_id=5 + N, flag_max=0.3, max_iter=1000)


def wterm_workload(N=64, n_ant=10, bmax=300.0, ha=0.8, freq=(1.7e9,), n_frame=1, config_id=400,
                   snr=100.0) -> Workload:
    """Point sources seen far from transit (hour angle ``ha`` rad), so that |w| reaches the
    longest baselines and the w-term phase pi (l^2 + m^2) w is of order 1 rad at the edge of
    the field (Sec. 6.1): seven sources over the image, visibilities with the w-term."""
    ant = spiral_array(n_ant, 4.0, centre=(n_ant % 3 == 1), bmax=bmax)
    pairs = baseline_pairs(n_ant)
    has = ha + EARTH_RATE * 0.025 * np.arange(n_frame)
    dec = np.full(n_frame, DEC_SUN)
    freq = np.asarray(freq, float)
    u, v, w = _sky_plane_projection(ant, pairs, MINGANTU_LAT, has, dec, freq, with_w=True)
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id])))
    fov = 60.0 * ARCMIN
    pts = [(float(a), float(b), float(c)) for a, b, c in
           zip(rng.uniform(-0.45, 0.45, 7) * fov, rng.uniform(-0.45, 0.45, 7) * fov, rng.uniform(0.3, 1.0, 7))]
    vis = np.empty((n_frame, len(freq), len(pairs)), np.complex64)
    for f in range(n_frame):
        Vm = point_visibilities_w(pts, u[f], v[f], w[f])
        for c in range(len(freq)):
            nrng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED_ROOT, config_id, f, c])))
            sig = math.sqrt(np.mean(np.abs(Vm[c]) ** 2)) / snr
            noise = nrng.normal(size=(len(pairs), 2)) * (sig / math.sqrt(2.0))
            vis[f, c] = (Vm[c] + noise[:, 0] + 1j * noise[:, 1]).astype(np.complex64)
    return Workload(name=f"wterm-N{N}", ant_enu=ant, pairs=pairs, lat=MINGANTU_LAT, ha=has, dec=dec, freq=freq,
                    vis=vis, flags=np.zeros(vis.shape, np.uint8), N=N, G=4 * N, bmax=bmax, max_iter=100,
                    skies=[pts])


def config5_mixed_stream(n_total=10000):
    """Mixed stream: n_total (frame, channel) instances, half MUSER-I (40 antennas, 64 channels
    per 25 ms frame, 0.4-2 GHz) and half MUSER-II (60 antennas, 528 channels per 206.25 ms
    frame, 2-15 GHz), 0-30 % of baselines flagged per frame, 1000 iterations.

    Returns (muser1, muser2, order): the two workloads (whole frames, the last one trimmed in
    channels) and the stream order, a list of (instrument 0/1, instance) pairs interleaving
    the two instruments frame by frame."""
    n1 = n_total // 2
    n2 = n_total - n1
    f1, f2 = -(-n1 // 64), -(-n2 // 528)
    ant1, ant2 = muser1_array(), muser2_array()
    w1 = make_workload("mixed-muser1", ant1, baseline_pairs(40), EARTH_RATE * 0.025 * np.arange(f1),
                       np.full(f1, DEC_SUN), muser1_channels(), 512, 2048, config_id=51, flag_max=0.3, max_iter=1000)
    w2 = make_workload("mixed-muser2", ant2, baseline_pairs(60), EARTH_RATE * 0.20625 * np.arange(f2),
                       np.full(f2, DEC_SUN), muser2_channels(), 1024, 4096, config_id=52, flag_max=0.3,
                       max_iter=1000)
    order, i1, i2 = [], 0, 0
    while i1 < n1 or i2 < n2:                      # 8 MUSER-I frames per MUSER-II frame (25 vs 206 ms)
        for _ in range(8 * 64):
            if i1 < n1:
                order.append((0, i1))
                i1 += 1
        for _ in range(528):
            if i2 < n2:
                order.append((1, i2))
                i2 += 1
    return w1, w2, order


def config4_operator() -> Workload:
    """Differentiable imaging: 512 x 512 sky, 780 baselines x 64 channels, G = 2N."""
    ant = muser1_array()
    return make_workload("degrid-512", ant, baseline_pairs(40), np.array([0.0]),
                         np.array([DEC_SUN]), muser1_channels(), 512, 1024, config_id=4)


def small_workload(n_ant=10, N=64, freq=(1.7e9,), n_frame=1, config_id=100, flag_max=0.0,
                   bmax=300.0, max_iter=50, snr=30.0) -> Workload:
    """A tiny array for oracle pins and quick parity cases (baselines up to ``bmax``)."""
    ant = spiral_array(n_ant, 4.0, centre=(n_ant % 3 == 1), bmax=bmax)
    ha = EARTH_RATE * 0.025 * np.arange(n_frame)
    return make_workload(f"small-{n_ant}ant-N{N}", ant, baseline_pairs(n_ant), ha,
                         np.full(n_frame, DEC_SUN), np.asarray(freq, float), N, 4 * N,
                         config_id=config_id, flag_max=flag_max, bmax=bmax, snr=snr,
                         max_iter=max_iter)
