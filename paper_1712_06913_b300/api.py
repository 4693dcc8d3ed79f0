"""PyTorch-facing wrappers of the libmuser C ABI: argument marshalling only.

Tensors supply device memory and the current CUDA stream; every computation runs in
the library's kernels.  Each wrapper allocates its outputs and the workspace the call
asks for with torch, then passes raw pointers.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math

import numpy as np
import torch

from . import _lib
from ._lib import CALL_CENTER, CALL_CHI2, CALL_GRAD, CALL_STEER, CALL_CLEAN, CALL_DEGRID, CALL_DIRTY, CALL_GRID, CALL_IMAGE, check

RECORD_FLOATS = 8          # 32-byte record viewed as float32[8]


@dataclasses.dataclass
class Config:
    """Mirror of muser_config_t."""
    N: int
    G: int
    W: int = 7
    os: int = 1024
    weight_mode: int = 0
    peak_mode: int = 0
    thr_mode: int = 0
    max_iter: int = 200
    gain: float = 0.1
    gmm_bins: int = 2000
    lat_rad: float = 0.0
    batch_chunk: int = 0
    clean_kernel: int = 0       # 0 auto (on-chip residual when possible), 1 streaming
    w_planes: int = 0           # w-projection planes (0: 2-D imaging)
    w_max: float = 0.0          # largest |wg| = |w| (G cell)^2 the planes cover
    w_support: int = 15         # w-kernel support (cells, odd)
    clean_variant: int = 0      # muser_image: 0 Hogbom, 1 Steer (max_iter major cycles)
    steer_clip: float = 0.9     # Steer selection level

    def c(self) -> _lib.Config:
        return _lib.Config(self.N, self.G, self.W, self.os, self.weight_mode, self.peak_mode, self.thr_mode,
                           self.max_iter, self.gain, self.gmm_bins, self.lat_rad, self.batch_chunk,
                           self.clean_kernel, self.w_planes, self.w_max, self.w_support, self.clean_variant,
                           self.steer_clip)


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dev(t, dtype=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        t = torch.as_tensor(np.ascontiguousarray(t))
    if dtype is not None:
        t = t.to(dtype)
    return t.to("cuda").contiguous()


def workspace_size(call_id, B, n_vis, cfg: Config) -> int:
    c = cfg.c() if cfg is not None else None
    n = _lib.load().muser_workspace_size(call_id, B, n_vis, ctypes.byref(c) if c is not None else None)
    if n == ctypes.c_size_t(-1).value:
        raise _lib.MuserError(_lib.MUSER_ERR_ARG, "invalid workspace query: " + _lib.load().muser_last_error().decode())
    return n


class Workspace:
    """A reusable 256-byte aligned device workspace."""

    def __init__(self):
        self.buf = None

    def get(self, nbytes):
        if nbytes == 0:
            return None, 0
        if self.buf is None or self.buf.numel() < nbytes + 256:
            self.buf = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        off = (-self.buf.data_ptr()) % 256
        return ctypes.c_void_p(self.buf.data_ptr() + off), self.buf.numel() - off


_default_ws = Workspace()


def launch_count() -> int:
    """Kernels the library has enqueued from the host so far (graph replays not included)."""
    return int(_lib.load().muser_launch_count())


def pixel_size(freq_hz, bmax_m, N, fov_min_rad):
    """Host rule of Table 2 (three pixels per resolution element, floored at fov_min / N)."""
    f = np.ascontiguousarray(freq_hz, dtype=np.float64)
    out = np.empty_like(f)
    check(_lib.load().muser_pixel_size(f.ctypes.data_as(ctypes.c_void_p), len(f), float(bmax_m), int(N),
                                       float(fov_min_rad), out.ctypes.data_as(ctypes.c_void_p)))
    return out


def uvw(ant_enu, pairs, ha, dec, freq, cell, vis, cfg: Config, flags=None, dlm=None, want_uvw=False, status=None):
    """Records [F*C*nb, 8] float32 (32-byte muser_vis_record_t), optional uvw [F*C*nb, 3] f64."""
    ant = _dev(ant_enu, torch.float64)
    pr = _dev(pairs, torch.int32)
    ha_t, dec_t = _dev(ha, torch.float64), _dev(dec, torch.float64)
    fr, ce = _dev(freq, torch.float64), _dev(cell, torch.float64)
    V = _dev(vis, torch.complex64)
    F, C, nb = len(ha_t), len(fr), pr.shape[0]
    fl = _dev(flags, torch.uint8) if flags is not None else None
    dl = _dev(dlm, torch.float64) if dlm is not None else None
    rec = torch.empty((F * C * nb, RECORD_FLOATS), dtype=torch.float32, device="cuda")
    uv = torch.empty((F * C * nb, 3), dtype=torch.float64, device="cuda") if want_uvw else None
    st = status if status is not None else torch.zeros(F * C, dtype=torch.int32, device="cuda")
    c = cfg.c()
    check(_lib.load().muser_uvw(_p(ant), ant.shape[0], _p(pr), nb, _p(ha_t), _p(dec_t), F, _p(fr), _p(ce), C,
                                _p(V), _p(fl), _p(dl), ctypes.byref(c), _p(rec), _p(uv), _p(st), _stream()))
    return rec, uv, st


def record_fields(rec: torch.Tensor):
    """Split [n, 8] float32 records into (vis complex64, fu, fv, ku, kv, w, wg)."""
    vis = torch.complex(rec[:, 0], rec[:, 1])
    k = rec[:, 4].contiguous().view(torch.int16)
    return vis, rec[:, 2], rec[:, 3], k[0::2].to(torch.int64), k[1::2].to(torch.int64), rec[:, 5], rec[:, 6]


def grid(rec, vis_off, cfg: Config, status=None, ws: Workspace = None, out=None, n_vis=None):
    """uv grids Z [B, G, G] complex64 from CSR records.  `out`: a contiguous complex64 tensor of
    that shape to write into (else one is allocated); `n_vis`: vis_off[B] when the caller knows
    it (else it is read back from the device)."""
    vo = _dev(vis_off, torch.int64)
    B = vo.numel() - 1
    n = int(n_vis) if n_vis is not None else (int(vo[-1].item()) if B > 0 else 0)
    if out is not None:
        if tuple(out.shape) != (B, cfg.G, cfg.G) or out.dtype != torch.complex64 or not out.is_contiguous():
            raise ValueError("out must be a contiguous complex64 tensor of shape (B, G, G)")
        Z = out
    else:
        Z = torch.empty((B, cfg.G, cfg.G), dtype=torch.complex64, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_GRID, B, n, cfg))
    check(_lib.load().muser_grid(_p(rec), _p(vo), B, n, ctypes.byref(c), _p(Z), w, wb, _p(st), _stream()))
    return Z, st


def dirty(Z, cfg: Config, status=None, ws: Workspace = None, out=None):
    """(dirty [B, N, N], beam [B, 2N, 2N], status) from grids.  `out`: a pair (D, Bm) of
    contiguous float32 tensors of those shapes to write into (else they are allocated)."""
    B = Z.shape[0]
    N = cfg.N
    if out is not None:
        D, Bm = out
        if (tuple(D.shape) != (B, N, N) or tuple(Bm.shape) != (B, 2 * N, 2 * N) or D.dtype != torch.float32
                or Bm.dtype != torch.float32 or not D.is_contiguous() or not Bm.is_contiguous()):
            raise ValueError("out must be contiguous float32 tensors of shapes (B, N, N) and (B, 2N, 2N)")
    else:
        D = torch.empty((B, N, N), dtype=torch.float32, device="cuda")
        Bm = torch.empty((B, 2 * N, 2 * N), dtype=torch.float32, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_DIRTY, B, 0, cfg))
    check(_lib.load().muser_dirty(_p(Z.contiguous()), B, ctypes.byref(c), _p(D), _p(Bm), w, wb, _p(st), _stream()))
    return D, Bm, st


def gmm(D, cfg: Config, status=None):
    B = D.shape[0]
    mu_a = torch.empty(B, dtype=torch.float32, device="cuda")
    mu_b = torch.empty(B, dtype=torch.float32, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    c = cfg.c()
    check(_lib.load().muser_gmm(_p(D.contiguous()), B, ctypes.byref(c), _p(mu_a), _p(mu_b), None, 0, _p(st),
                                _stream()))
    return mu_a, mu_b, st


def clean(D, Bm, cfg: Config, thr=None, status=None, ws: Workspace = None):
    """Hogbom CLEAN: (residual, comp_pos [B, cap], comp_flux, n_comp, status).  D is not modified."""
    B = D.shape[0]
    R = D.clone()
    cap = cfg.max_iter
    pos = torch.zeros((B, max(cap, 1)), dtype=torch.int32, device="cuda")
    flux = torch.zeros((B, max(cap, 1)), dtype=torch.float32, device="cuda")
    nc = torch.empty(B, dtype=torch.int32, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    th = _dev(thr, torch.float32) if thr is not None else None
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_CLEAN, B, 0, cfg))
    check(_lib.load().muser_clean(_p(R), _p(Bm.contiguous()), B, ctypes.byref(c), _p(th), _p(pos), _p(flux), _p(nc),
                                  w, wb, _p(st), _stream()))
    return R, pos[:, :cap], flux[:, :cap], nc, st


def center(R, mu_a, mu_b, cell, cfg: Config, status=None, want_corr=False, ws: Workspace = None):
    """Disk offsets of residuals CLEANed to the disk level: (dlm [B, 2] rad, shift [B, 2] px,
    corr [B, N/2+1, N/2+1] or None, status)."""
    B, N = R.shape[0], cfg.N
    dlm = torch.empty((B, 2), dtype=torch.float64, device="cuda")
    shift = torch.empty((B, 2), dtype=torch.float32, device="cuda")
    corr = torch.empty((B, N // 2 + 1, N // 2 + 1), dtype=torch.float32, device="cuda") if want_corr else None
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    cl = _dev(cell, torch.float64)
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_CENTER, B, 0, cfg))
    check(_lib.load().muser_center(_p(R.contiguous()), _p(mu_a), _p(mu_b), _p(cl), B, ctypes.byref(c), _p(corr),
                                   _p(dlm), _p(shift), w, wb, _p(st), _stream()))
    return dlm, shift, corr, st


def steer(D, Bm, cfg: Config, thr=None, clip=0.9, status=None, ws: Workspace = None):
    """Steer CLEAN in major cycles (cfg.max_iter cycles at most): (residual, model, n_cycles,
    status).  D is not modified."""
    B, N = D.shape[0], cfg.N
    R = D.clone()
    model = torch.empty((B, N, N), dtype=torch.float32, device="cuda")
    nc = torch.empty(B, dtype=torch.int32, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    th = _dev(thr, torch.float32) if thr is not None else None
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_STEER, B, 0, cfg))
    check(_lib.load().muser_steer(_p(R), _p(Bm.contiguous()), B, ctypes.byref(c), _p(th), float(clip), _p(model),
                                  _p(nc), w, wb, _p(st), _stream()))
    return R, model, nc, st


def restore(R, Bm, pos, flux, n_comp, cfg: Config, status=None):
    B = R.shape[0]
    out = torch.empty_like(R)
    params = torch.empty((B, 3), dtype=torch.float32, device="cuda")
    st = status if status is not None else torch.zeros(max(B, 1), dtype=torch.int32, device="cuda")
    cap = cfg.max_iter
    pos_c = torch.zeros((B, max(cap, 1)), dtype=torch.int32, device="cuda")
    flux_c = torch.zeros((B, max(cap, 1)), dtype=torch.float32, device="cuda")
    pos_c[:, :cap] = pos
    flux_c[:, :cap] = flux
    c = cfg.c()
    check(_lib.load().muser_restore(_p(R.contiguous()), _p(Bm.contiguous()), _p(pos_c), _p(flux_c), _p(n_comp), B,
                                    ctypes.byref(c), _p(out), _p(params), None, 0, _p(st), _stream()))
    return out, params, st


@dataclasses.dataclass
class ImageResult:
    clean: torch.Tensor
    residual: torch.Tensor
    comp_pos: torch.Tensor
    comp_flux: torch.Tensor
    n_comp: torch.Tensor
    thr: torch.Tensor
    beam_params: torch.Tensor
    status: torch.Tensor


class Imager:
    """Device-resident inputs and outputs for repeated muser_image calls on one batch shape."""

    def __init__(self, ant_enu, pairs, ha, dec, freq, cell, vis, cfg: Config, flags=None, dlm=None):
        self.cfg = cfg
        self.ant = _dev(ant_enu, torch.float64)
        self.pairs = _dev(pairs, torch.int32)
        self.ha, self.dec = _dev(ha, torch.float64), _dev(dec, torch.float64)
        self.freq, self.cell = _dev(freq, torch.float64), _dev(cell, torch.float64)
        self.vis = _dev(vis, torch.complex64)
        self.flags = _dev(flags, torch.uint8) if flags is not None else None
        self.dlm = _dev(dlm, torch.float64) if dlm is not None else None
        self.F, self.C, self.nb = len(self.ha), len(self.freq), self.pairs.shape[0]
        B, N, cap = self.F * self.C, cfg.N, cfg.max_iter
        self.B = B
        self.out = self.new_output()
        self.ws = Workspace()
        self.ws_bytes = workspace_size(CALL_IMAGE, B, self.nb, cfg)
        self.c = cfg.c()

    def new_output(self):
        """A fresh set of output tensors for this batch shape (e.g. a second set, so that one
        batch's results can be copied out while the next batch is imaged)."""
        B, N, cap, dev = self.B, self.cfg.N, self.cfg.max_iter, "cuda"
        return ImageResult(
            clean=torch.empty((B, N, N), dtype=torch.float32, device=dev),
            residual=torch.empty((B, N, N), dtype=torch.float32, device=dev),
            comp_pos=torch.zeros((B, max(cap, 1)), dtype=torch.int32, device=dev),
            comp_flux=torch.zeros((B, max(cap, 1)), dtype=torch.float32, device=dev),
            n_comp=torch.empty(B, dtype=torch.int32, device=dev),
            thr=torch.empty(B, dtype=torch.float32, device=dev),
            beam_params=torch.empty((B, 3), dtype=torch.float32, device=dev),
            status=torch.empty(B, dtype=torch.int32, device=dev))

    @property
    def chunks(self):
        """(first instance, instances) of each chunk muser_image images in turn."""
        b = self.cfg.batch_chunk if 0 < self.cfg.batch_chunk < self.B else self.B
        return [(c0, min(b, self.B - c0)) for c0 in range(0, self.B, b)]

    def run(self, vis=None, out=None, chunk_done=None):
        """Launch the whole batch on the current stream (no host synchronisation), writing
        `out` (default: self.out).  chunk_done: torch.cuda.Event per chunk (see `chunks`), each
        recorded on the current stream once its chunk's results are complete (muser_image_events),
        so that another stream can copy them out while the next chunks are imaged."""
        V = self.vis if vis is None else vis
        o = self.out if out is None else out
        w, wb = self.ws.get(self.ws_bytes)
        args = (_p(self.ant), self.ant.shape[0], _p(self.pairs), self.nb, _p(self.ha), _p(self.dec), self.F,
                _p(self.freq), _p(self.cell), self.C, _p(V), _p(self.flags), _p(self.dlm), ctypes.byref(self.c),
                _p(o.clean), _p(o.residual), _p(o.comp_pos), _p(o.comp_flux), _p(o.n_comp), _p(o.thr),
                _p(o.beam_params), w, wb, _p(o.status))
        if chunk_done is None:
            check(_lib.load().muser_image(*args, _stream()))
            return o
        for e in chunk_done:
            if not e.cuda_event:            # torch creates the CUDA event at its first record
                e.record()
        ev = (ctypes.c_void_p * max(1, len(chunk_done)))(*[e.cuda_event for e in chunk_done])
        check(_lib.load().muser_image_events(*args, ev, len(chunk_done), _stream()))
        return o

    def capture(self):
        """Record the whole batch (every chunk, both of muser_image's streams) in one CUDA graph.

        One eager run first creates the library's streams and plans outside the capture.
        `replay()` then re-runs the batch with no host work, reading the visibilities from
        `self.vis` (copy new data into it before a replay) and writing `self.out`.
        """
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self

    def replay(self):
        self.graph.replay()
        return self.out


def autotune(call_id, cfg: Config, rec=None, vis_off=None, B=1):
    """Time the launch-shape candidates of muser_grid (band rows; needs rec, vis_off), muser_dirty
    (column-strip width) or muser_image (gridding tile and FFT radix; needs rec of B instances with
    the same number of records each) on one batch and keep the fastest; returns the choice."""
    vo = _dev(vis_off, torch.int64) if vis_off is not None else None
    if vo is not None:
        B = vo.numel() - 1
    n = int(vo[-1].item()) if vo is not None and B > 0 else 0
    if call_id == CALL_IMAGE:
        n = rec.shape[0] if rec is not None else 0
        vo = None
    out = ctypes.c_int32(0)
    c = cfg.c()
    check(_lib.load().muser_autotune(call_id, _p(rec), _p(vo), B, n, ctypes.byref(c), ctypes.byref(out), _stream()))
    return out.value


def set_tuning(call_id, cfg: Config, value: int):
    c = cfg.c()
    check(_lib.load().muser_set_tuning(call_id, ctypes.byref(c), int(value)))


# Table 2: image side by observing frequency (upper band edges in Hz)
TABLE2_SIDES = ((0.6e9, 256), (1.2e9, 512), (2.0e9, 1024), (4.0e9, 1280), (8.0e9, 2560), (float("inf"), 5120))


def image_side(freq_hz, n_max=5120):
    """Image side of Table 2 for each channel frequency (0.4-0.6 GHz: 256 ... 8-15 GHz: 5120),
    capped at n_max."""
    out = []
    for f in np.atleast_1d(np.asarray(freq_hz, float)):
        side = next(n for edge, n in TABLE2_SIDES if f < edge)
        out.append(min(side, n_max))
    return np.array(out, np.int64)


@dataclasses.dataclass
class Source:
    """One array's observations for a mixed stream: [F, C, nb] visibilities, imaging parameters
    shared by its channels; image sides come from Table 2 (capped at n_max)."""
    ant_enu: object
    pairs: object
    ha: object
    dec: object
    freq: object
    vis: object
    flags: object = None
    bmax: float = 3000.0
    fov_min: float = math.pi / 180.0
    n_max: int = 1024
    W: int = 7
    os: int = 1024
    gain: float = 0.1
    max_iter: int = 1000
    lat_rad: float = 0.0
    batch_chunk: int = 296


def size_classes(freq_hz, n_max=5120):
    """Runs of consecutive channels with the same Table 2 side: [(first, end, side), ...]."""
    sides = image_side(freq_hz, n_max)
    runs, c0 = [], 0
    while c0 < len(sides):
        c1 = c0
        while c1 < len(sides) and sides[c1] == sides[c0]:
            c1 += 1
        runs.append((c0, c1, int(sides[c0])))
        c0 = c1
    return runs


class MixedImager:
    """A stream of instances of several image sizes, batched by size class: each source's channels
    are split into runs of equal Table 2 side, each run imaged as one muser_image batch (chunked
    inside), all batches launched back to back on the current stream or replayed from one CUDA
    graph.  `locate(source, instance)` maps a stream instance (frame * n_chan + chan of its
    source) to (class, index in that class's ImageResult)."""

    def __init__(self, sources):
        self.classes = []           # (source index, first channel, n channels, Imager)
        for si, src in enumerate(sources):
            freq = np.asarray(src.freq, float)
            for c0, c1, N in size_classes(freq, src.n_max):
                cfg = Config(N=N, G=4 * N, W=src.W, os=src.os, max_iter=src.max_iter, gain=src.gain,
                             lat_rad=src.lat_rad, batch_chunk=src.batch_chunk)
                fr = freq[c0:c1]
                cell = pixel_size(fr, src.bmax, N, src.fov_min)
                vis = np.asarray(src.vis)[:, c0:c1]
                flags = np.asarray(src.flags)[:, c0:c1] if src.flags is not None else None
                im = Imager(src.ant_enu, src.pairs, src.ha, src.dec, fr, cell, np.ascontiguousarray(vis), cfg,
                            flags=None if flags is None else np.ascontiguousarray(flags))
                self.classes.append((si, c0, c1 - c0, im))
        self.n_chan = [len(np.asarray(src.freq)) for src in sources]
        self.graph = None

    def locate(self, source, instance):
        f, c = divmod(instance, self.n_chan[source])
        for k, (si, c0, nc, im) in enumerate(self.classes):
            if si == source and c0 <= c < c0 + nc:
                return k, f * nc + (c - c0)
        raise IndexError("instance not in any size class")

    def run(self):
        return [im.run() for _, _, _, im in self.classes]

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self

    def replay(self):
        self.graph.replay()
        return [im.out for _, _, _, im in self.classes]


def image(ant_enu, pairs, ha, dec, freq, cell, vis, cfg: Config, flags=None, dlm=None):
    """Whole hot path for a batch; returns an ImageResult with comp arrays cut to max_iter."""
    im = Imager(ant_enu, pairs, ha, dec, freq, cell, vis, cfg, flags, dlm)
    o = im.run()
    cap = cfg.max_iter
    return dataclasses.replace(o, comp_pos=o.comp_pos[:, :cap], comp_flux=o.comp_flux[:, :cap])


def image_centred(ant_enu, pairs, ha, dec, freq, cell, vis, cfg: Config, flags=None, pre_cap=1000):
    """Alg. 1 with the centring of Sec. 4.2: dirty map -> GMM levels -> CLEAN down to the disk
    level mu_b (at most pre_cap iterations) -> disk offset (muser_center) -> phase-corrected
    re-imaging with the sky threshold mu_a (muser_image, thr_mode 1).

    Returns (ImageResult of the corrected visibilities, dlm [B, 2] rad, shift [B, 2] px).
    The first pass holds every instance's G x G grid at once: call it on batches that fit.
    """
    F, C = len(ha), len(freq)
    pre = Config(**{**cfg.__dict__, "thr_mode": 0, "max_iter": pre_cap})
    rec, _, st = uvw(ant_enu, pairs, ha, dec, freq, cell, vis, pre, flags=flags)
    nb = int(np.asarray(pairs).shape[0])
    off = torch.arange(F * C + 1, dtype=torch.int64, device="cuda") * nb
    Z, st = grid(rec, off, pre, status=st)
    D, Bm, st = dirty(Z, pre, status=st)
    del Z
    mu_a, mu_b, st = gmm(D, pre, status=st)
    R, _, _, _, st = clean(D, Bm, pre, thr=mu_b, status=st)
    dlm, shift, _, st = center(R, mu_a, mu_b, np.tile(np.asarray(cell, float), F), pre, status=st)
    out = image(ant_enu, pairs, ha, dec, freq, cell, vis, Config(**{**cfg.__dict__, "thr_mode": 1}), flags=flags,
                dlm=dlm)
    return out, dlm, shift


class CentredImager:
    """image_centred on device-resident inputs, enqueued with no host synchronisation and
    replayable from one CUDA graph: uvw -> grid -> dirty -> GMM -> CLEAN down to the disk level
    mu_b -> disk offset (muser_center) -> phase-corrected muser_image with the sky threshold.
    `run()` launches it all; `capture()` records it once; `replay()` re-runs the graph (copy new
    visibilities into `self.vis` first).  Outputs: `self.imager.out` (ImageResult), `self.dlm`
    [B, 2] rad and `self.shift` [B, 2] px.  The first pass holds every instance's G x G grid."""

    def __init__(self, ant_enu, pairs, ha, dec, freq, cell, vis, cfg: Config, flags=None, pre_cap=1000):
        self.pre = Config(**{**cfg.__dict__, "thr_mode": 0, "max_iter": pre_cap})
        self.ant, self.pairs = _dev(ant_enu, torch.float64), _dev(pairs, torch.int32)
        self.ha, self.dec = _dev(ha, torch.float64), _dev(dec, torch.float64)
        self.freq, self.cell = _dev(freq, torch.float64), _dev(cell, torch.float64)
        self.vis = _dev(vis, torch.complex64)
        self.flags = _dev(flags, torch.uint8) if flags is not None else None
        F, C, self.nb = len(self.ha), len(self.freq), self.pairs.shape[0]
        self.B = F * C
        self.off = torch.arange(self.B + 1, dtype=torch.int64, device="cuda") * self.nb
        self.cell_b = self.cell.repeat(F)            # instance f * C + c
        self.dlm = torch.zeros((self.B, 2), dtype=torch.float64, device="cuda")
        self.shift = torch.zeros((self.B, 2), dtype=torch.float32, device="cuda")
        self.imager = Imager(self.ant, self.pairs, self.ha, self.dec, self.freq, self.cell, self.vis,
                             Config(**{**cfg.__dict__, "thr_mode": 1}), flags=self.flags, dlm=self.dlm)
        self.ws = Workspace()
        self.graph = None

    def run(self):
        pre = self.pre
        rec, _, st = uvw(self.ant, self.pairs, self.ha, self.dec, self.freq, self.cell, self.vis, pre, flags=self.flags)
        Z, st = grid(rec, self.off, pre, status=st, ws=self.ws, n_vis=self.B * self.nb)
        D, Bm, st = dirty(Z, pre, status=st, ws=self.ws)
        del Z
        mu_a, mu_b, st = gmm(D, pre, status=st)
        R, _, _, _, st = clean(D, Bm, pre, thr=mu_b, status=st, ws=self.ws)
        dlm, shift, _, st = center(R, mu_a, mu_b, self.cell_b, pre, status=st, ws=self.ws)
        self.dlm.copy_(dlm)
        self.shift.copy_(shift)
        return self.imager.run()

    def capture(self):
        """One eager run on a side stream (the library's streams, plans and workspaces), then
        the whole pipeline recorded in one CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self

    def replay(self):
        self.graph.replay()
        return self.imager.out


def degrid(direction, rec, cfg: Config, img=None, vis=None, ws: Workspace = None, reuse_plan=False):
    """FORWARD: img [N, N] f32 -> vis [n] complex64.  ADJOINT: vis -> img (real part of A^H vis).

    reuse_plan: `ws` already holds this record set's plan from an earlier call (see DegridPlan).
    """
    n = rec.shape[0]
    c = cfg.c()
    w, wb = (ws or _default_ws).get(workspace_size(CALL_DEGRID, 1, n, cfg))
    flag = _lib.REUSE_PLAN if reuse_plan else 0
    if direction == _lib.FORWARD:
        img = img.contiguous()
        out = torch.empty(n, dtype=torch.complex64, device="cuda")
        check(_lib.load().muser_degrid(_lib.FORWARD | flag, _p(img), _p(rec), n, _p(out), ctypes.byref(c), w, wb,
                                       _stream()))
        return out
    vis = vis.contiguous()
    out = torch.empty((cfg.N, cfg.N), dtype=torch.float32, device="cuda")
    check(_lib.load().muser_degrid(_lib.ADJOINT | flag, _p(out), _p(rec), n, _p(vis), ctypes.byref(c), w, wb,
                                   _stream()))
    return out


class DegridPlan:
    """The measurement operator of one record set (fixed uv coverage) with its own workspace.

    The first call plans (kernel table, grid correction, twiddles, the adjoint's tap lists by
    grid cell); later calls reuse the plan and only run the transforms.  The configuration
    structure, workspace and chi-square scratch are set up once, so an evaluation costs the
    library calls only.
    """

    def __init__(self, rec, cfg: Config):
        self.rec, self.cfg = rec, cfg
        self.n = rec.shape[0]
        self.c = cfg.c()
        self.ws = Workspace()
        # the gradient-step workspace holds the operator's at its start: one plan serves both
        self.w, self.wb = self.ws.get(workspace_size(CALL_GRAD, 1, self.n, cfg))
        self.cws = Workspace()
        self.cw, self.cwb = self.cws.get(workspace_size(CALL_CHI2, 1, self.n, None))
        self.planned = False
        self.lib = _lib.load()
        self.rows_ready = None        # the image whose forward row pass a chained step left in ws

    def clone(self):
        """A second operator over the same records that takes this one's plan (copied, not built
        again) and has a workspace of its own: the plan's record order and tap lists fix the
        order of every sum, so the two give identical results, while independently built plans
        agree only to rounding."""
        other = DegridPlan(self.rec, self.cfg)
        if self.planned:
            s0 = self.w.value - self.ws.buf.data_ptr()
            d0 = other.w.value - other.ws.buf.data_ptr()
            n = min(self.wb, other.wb)                   # both hold the whole workspace
            other.ws.buf[d0:d0 + n].copy_(self.ws.buf[s0:s0 + n])
            other.planned = True
        return other

    def _flag(self, d):
        f = d | (_lib.REUSE_PLAN if self.planned else 0)
        self.planned = True
        self.rows_ready = None
        return f

    def forward(self, img):
        img = img.contiguous()
        out = torch.empty(self.n, dtype=torch.complex64, device="cuda")
        check(self.lib.muser_degrid(self._flag(_lib.FORWARD), _p(img), _p(self.rec), self.n, _p(out),
                                    ctypes.byref(self.c), self.w, self.wb, _stream()))
        return out

    def adjoint(self, vis):
        vis = vis.contiguous()
        out = torch.empty((self.cfg.N, self.cfg.N), dtype=torch.float32, device="cuda")
        check(self.lib.muser_degrid(self._flag(_lib.ADJOINT), _p(out), _p(self.rec), self.n, _p(vis),
                                    ctypes.byref(self.c), self.w, self.wb, _stream()))
        return out

    def grad_step(self, img, obs, inv_sigma2: float, eta: float, loss, grad=None, chain=False):
        """img -= eta grad chi2(img) in place (one library call, muser_grad_step); loss [1] (device)
        receives chi2 at the incoming img, grad (optional [N, N]) the gradient.  chain=True leaves
        the next step's first pass in the workspace; a following chained step on the same image
        tensor (changed by nothing else in between) then skips that pass."""
        flags = _lib.REUSE_PLAN if self.planned else 0
        if chain:
            flags |= _lib.GRAD_CHAIN
            if self.planned and self.rows_ready == img.data_ptr():
                flags |= _lib.GRAD_ROWS_READY
        check(self.lib.muser_grad_step(flags, _p(img), _p(self.rec), self.n, _p(obs), float(inv_sigma2), float(eta),
                                       _p(loss), _p(grad), ctypes.byref(self.c), self.w, self.wb, _stream()))
        self.planned = True
        self.rows_ready = img.data_ptr() if chain else None

    def normal_apply(self, v, inv_sigma2: float, out=None):
        """u = 2 Re A^H (w A v) / sigma^2, the chi-square Hessian applied to v (muser_normal_apply)."""
        v = v.contiguous()
        u = torch.empty((self.cfg.N, self.cfg.N), dtype=torch.float32, device="cuda") if out is None else out
        check(self.lib.muser_normal_apply(_lib.REUSE_PLAN if self.planned else 0, _p(v), _p(u), _p(self.rec), self.n,
                                          float(inv_sigma2), ctypes.byref(self.c), self.w, self.wb, _stream()))
        self.planned = True
        self.rows_ready = None
        return u

    def lipschitz(self, v, inv_sigma2: float, iters: int, L=None):
        """Power iteration on the chi-square Hessian from the start direction v (updated in place to
        the last unit direction): L [1] (device) = its largest eigenvalue (muser_lipschitz)."""
        L = torch.empty(1, dtype=torch.float32, device="cuda") if L is None else L
        check(self.lib.muser_lipschitz(_lib.REUSE_PLAN if self.planned else 0, _p(v), _p(self.rec), self.n,
                                       float(inv_sigma2), int(iters), _p(L), ctypes.byref(self.c), self.w, self.wb,
                                       _stream()))
        self.planned = True
        self.rows_ready = None
        return L

    def chi2(self, pred, obs, inv_sigma2: float):
        """(loss, residual seed) of predicted visibilities against obs (see muser_chi2)."""
        loss = torch.empty(1, dtype=torch.float32, device="cuda")
        resid = torch.empty(self.n, dtype=torch.complex64, device="cuda")
        check(self.lib.muser_chi2(_p(pred.contiguous()), _p(obs.contiguous()), _p(self.rec), self.n,
                                  float(inv_sigma2), _p(resid), _p(loss), self.cw, self.cwb, _stream()))
        return loss[0], resid


def chi2(pred, obs, rec, inv_sigma2: float, want_resid=True, ws: Workspace = None):
    n = rec.shape[0]
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    resid = torch.empty(n, dtype=torch.complex64, device="cuda") if want_resid else None
    w, wb = (ws or _default_ws).get(workspace_size(CALL_CHI2, 1, n, None))
    check(_lib.load().muser_chi2(_p(pred.contiguous()), _p(obs.contiguous()), _p(rec), n, float(inv_sigma2), _p(resid),
                                 _p(loss), w, wb, _stream()))
    return loss[0], resid


def normalize(u, v=None, norm=None):
    """norm [1] (device) = |u|_2 and v = u / norm (muser_normalize); v may be u itself."""
    v = torch.empty_like(u) if v is None else v
    norm = torch.empty(1, dtype=torch.float32, device="cuda") if norm is None else norm
    check(_lib.load().muser_normalize(_p(u), u.numel(), _p(v), _p(norm), _stream()))
    return v, norm


def axpy(y, x, alpha: float, alpha_dev=None):
    """y += alpha * (alpha_dev[0] if given else 1) * x in place (muser_axpy); complex tensors are
    taken as pairs of floats."""
    if y.is_complex():
        y, x = torch.view_as_real(y), torch.view_as_real(x)
    if not (y.is_contiguous() and x.is_contiguous() and y.numel() == x.numel()):
        raise ValueError("axpy: x and y must be contiguous and of one size")
    check(_lib.load().muser_axpy(_p(y), _p(x), y.numel(), float(alpha), _p(alpha_dev), _stream()))
    return y
