#!/usr/bin/env python
"""Benchmark of the MUSER imaging hot path on B300.

Workload (one step): the MUSER-II-like uneven batch -- 60 antennas (1770 baselines),
528 channels over 2-15 GHz x 8 frames = 4224 (frame, channel) instances, 0-30 % of the
baselines flagged per frame, 1024 x 1024 images on 4096 x 4096 grids, Hogbom CLEAN with
1000 iterations -- through uvw -> sorted gridding -> FFT dirty map/beam -> CLEAN ->
restore, batched in chunks of 296 instances (2 x 148 SMs).  Synthetic, seeded inputs.

Reported (one JSON line on rank 0):
  value      CLEANed images/s, inputs resident on the device (muser_image per step)
  e2e        the same with the visibilities copied from pinned host memory every step and
             the restored images, component lists, counts and status read back (on a copy
             stream, each chunk's as soon as muser_image_events announces it)
  roofline   the dominant kernel (CLEAN): its streaming-model bytes per second against the
             measured HBM copy bandwidth, with the DRAM and L2 fractions it actually reaches
  cpu_baseline  the FP64 oracle on a bounded sample on this host's cores
  extra      plain one-image-per-call throughput, gridding GB/s, gradient evaluations/s

--impl reference times the FP64 oracle (the CPU reference of this build) instead.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CLEANed images/s at 1024² batched vs plain; gridding GB/s; grad evals/s"
WORKLOAD = ("MUSER-II-like uneven batch: 60 antennas / 1770 baselines, 528 channels x 8 frames = 4224 instances, "
            "0-30% baselines flagged per frame, N=1024 (G=4096), spheroidal W=7, Hogbom gain 0.1, 1000 iterations")
CHUNK = 296


# ----------------------------------------------------------------------------- helpers

def steer_bytes(N):
    """Bytes one Steer major cycle moves per instance: R in and the column pass's half spectrum
    (N + 1 rows of N) out; the row pass reads that, the beam's half spectrum (N + 1 rows of 2N)
    and writes N + 1 rows of N; the inverse column pass reads them and writes Y; the update
    reads R, Y and the model and writes R and the model."""
    H = N + 1
    return 4.0 * N * N + 8.0 * H * N + (8.0 * H * N + 8.0 * H * 2 * N + 8.0 * H * N) + (8.0 * H * N + 4.0 * N * N) \
        + 20.0 * N * N


def center_bytes(N):
    """Bytes one disk-centring instance moves: residual in, forward columns out and back in,
    half spectrum (P/2 + 1 columns) out and back in, window columns out and back in, window out."""
    P, W = 2 * N, N // 2 + 1
    H = P // 2 + 1
    return 4.0 * N * N + 2 * 8.0 * N * P + 2 * 8.0 * H * P + 2 * 8.0 * W * H + 4.0 * W * W

STATUS_BITS = ("ALL_FLAGGED", "NONFINITE", "DROPPED", "GMM_DEGENERATE", "ITER_CAP", "BEAM_FIT", "TIMEOUT", "NO_DISK")


def status_histogram(status):
    """Instances per status bit (MUSER_ST_*), plus those with no bit set."""
    import numpy as np
    st = np.asarray(status)
    out = {name: int(((st >> b) & 1).sum()) for b, name in enumerate(STATUS_BITS)}
    out["none"] = int((st == 0).sum())
    out["unknown_bits"] = int((st & ~((1 << len(STATUS_BITS)) - 1) != 0).sum())
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6400.0), "measured"
    return 6400.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("clean.cu",):
        with open(os.path.join(ROOT, "paper_1712_06913_b300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """DRAM bytes per CLEAN launch from the committed ncu summary, if the kernel is unchanged."""
    p = os.path.join(ROOT, "profiles", "hogbom_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap,power.draw",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 7:
                    continue
                try:
                    sm.append(float(parts[0]))
                    smax = float(parts[1])
                except ValueError:
                    continue
                for n, v in zip(names, parts[2:6]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- oracle (CPU) legs
def _oracle_one(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np  # noqa: F401
    import synth
    from oracle import geometry, pipeline
    frame, chan, cap = args
    wl = synth.config3_muser2_uneven(n_frame=frame + 1, chans=[chan])
    rec = pipeline.records(wl, frames=slice(frame, frame + 1))
    t = time.perf_counter()
    rec_i = geometry.instance_slice(rec, 0, wl.n_bl)
    pipeline.image_instance(rec_i, wl.N, wl.G, gain=wl.gain, cap=wl.max_iter if cap is None else cap)
    return time.perf_counter() - t


def cpu_baseline(n_inst=None, cap=None):
    """Oracle images/s over `cores` instances run in parallel (spawned processes); `cap` cuts
    CLEAN short (a warm-up pass only: the figure is then not the workload's)."""
    cores = len(os.sched_getaffinity(0))
    n = n_inst or cores
    jobs = [(f % 8, (37 * f + 11) % 528, cap) for f in range(n)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(min(cores, n)) as pool:
        per = pool.map(_oracle_one, jobs)
    wall = time.perf_counter() - t0
    return {"value": n / wall, "unit": "images/s", "cores": min(cores, n), "kind": "oracle",
            "sample": f"{n} instances of the same workload (one per process, FP64 NumPy oracle, "
                      f"1 thread each); mean {statistics.mean(per):.1f} s per image incl. uvw, grid, FFT, "
                      f"1000 CLEAN iterations, restore"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    times = []
    base = None
    for i in range(args.warmup + args.steps):
        if i < args.warmup:          # untimed: one short oracle image (imports, page-in, pool start)
            cpu_baseline(n_inst=1, cap=5)
            continue
        t = time.perf_counter()
        b = cpu_baseline(n_inst=None)
        times.append(time.perf_counter() - t)
        base = b
    value = base["value"]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * statistics.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": base["sample"]},
            "cpu_baseline": base,
            "e2e": {"value": value, "unit": "images/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- GPU legs
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chunk", type=int, default=CHUNK)
    ap.add_argument("--frames", type=int, default=8, help="frames per rank (8 = the full workload)")
    ap.add_argument("--no-extras", action="store_true", help="skip plain/degrid/cpu-baseline legs")
    ap.add_argument("--case", choices=["clean", "dirty", "grid", "grad", "image0", "steer", "large", "large_clean", "wproj",
                                       "mixed", "center", "band2", "plain1", "steerimg"],
                    default=None,
                    help="small single-kernel case of the same workload (for ncu captures)")
    ap.add_argument("--instances", type=int, default=0, help="instances of a --case (default 148 / 8)")
    ap.add_argument("--iters", type=int, default=100, help="CLEAN iterations of --case clean")
    ap.add_argument("--size", type=int, default=2560, choices=[1280, 2560, 5120], help="image side of --case large")
    args = ap.parse_args()
    if args.case:
        run_case(args.case, args.instances, args.iters, args.size)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    import paper_1712_06913_b300 as m
    import synth

    # each rank images its own batch (different frames): weak scaling, no data-path collective
    from paper_1712_06913_b300 import dist as mdist
    wl = synth.config3_muser2_uneven(n_frame=args.frames * world)
    sl = mdist.block(args.frames * world, rank, world)
    ha, dec, vis, flags = wl.ha[sl], wl.dec[sl], wl.vis[sl], wl.flags[sl]
    B = len(ha) * wl.n_chan
    cfg = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=wl.max_iter, gain=wl.gain, lat_rad=wl.lat,
                   batch_chunk=args.chunk)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    stream = torch.cuda.current_stream()
    # muser_image's gridding tile and FFT radix, tuned on 32 instances of the workload (before any
    # timed run; the choice holds for every later call with this grid size)
    rec_t, _, _ = m.uvw(wl.ant_enu, wl.pairs, ha[:1], dec[:1], wl.freq[:32], cell[:32], vis[:1, :32], cfg,
                        flags=flags[:1, :32])
    image_variant = m.autotune(m.CALL_IMAGE, cfg, rec=rec_t, B=32)
    del rec_t
    imager = m.Imager(wl.ant_enu, wl.pairs, ha, dec, wl.freq, cell, vis, cfg, flags=flags)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        return mdist.all_max(x, device="cuda")

    # ---- warm-up
    for _ in range(args.warmup):
        imager.run()
    barrier()

    # ---- timed: device-resident inputs
    clocks = Clocks(local)
    clocks.start()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    barrier()
    launches0 = m.launch_count()
    ev[0].record(stream)
    for k in range(args.steps):
        imager.run()
        ev[k + 1].record(stream)
    launches1 = m.launch_count()
    barrier()
    clk = clocks.stop()
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)]
    total_ms = max_over_ranks(sum(step_ms))
    value = B * world * args.steps / (total_ms / 1e3)
    out = imager.out
    n_comp = out.n_comp.cpu().numpy()
    status = out.status.cpu().numpy()
    gpu_launches = launches1 - launches0   # counted by the library as it enqueues its kernels

    # ---- end to end: pinned host visibilities in; restored images, CLEAN model and status out,
    # every step.  Each chunk's results stream to the host on a copy stream as soon as the library
    # announces them (muser_image_events), while the following chunks are imaged; two output sets
    # alternate between steps.
    vis_host = torch.from_numpy(np.ascontiguousarray(vis.astype(np.complex64))).pin_memory()
    vis_dev = torch.empty_like(vis_host, device="cuda")
    outs = [out, imager.new_output()]
    clean_bytes_all = out.clean.numel() * 4
    avail = 0                              # room for every restored image in pinned host memory?
    try:
        with open("/proc/meminfo") as f:
            for ln in f:
                if ln.startswith("MemAvailable:"):
                    avail = int(ln.split()[1]) * 1024
    except OSError:
        pass
    n_img = B if avail > 3 * clean_bytes_all else max(1, min(B, int(avail // (3 * 4 * wl.N * wl.N))))
    clean_host = torch.empty((n_img, wl.N, wl.N), dtype=torch.float32).pin_memory()
    pos_host = torch.empty(out.comp_pos.shape, dtype=torch.int32).pin_memory()
    flux_host = torch.empty(out.comp_flux.shape, dtype=torch.float32).pin_memory()
    nc_host = torch.empty(B, dtype=torch.int32).pin_memory()
    st_host = torch.empty(B, dtype=torch.int32).pin_memory()
    h2d = vis_host.numel() * 8
    d2h = clean_host.numel() * 4 + pos_host.numel() * 4 + flux_host.numel() * 4 + 2 * B * 4
    copy_stream = torch.cuda.Stream()
    chunks = imager.chunks
    done = [[torch.cuda.Event() for _ in chunks] for _ in range(2)]
    copied = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for k in range(args.steps):
        j = k & 1
        if k >= 2:
            stream.wait_event(copied[j])    # this output set's copy from step k - 2 is done
        vis_dev.copy_(vis_host, non_blocking=True)
        o = imager.run(vis_dev, out=outs[j], chunk_done=done[j])
        with torch.cuda.stream(copy_stream):
            for (c0, n), ev in zip(chunks, done[j]):
                copy_stream.wait_event(ev)
                c1 = min(c0 + n, n_img)
                if c1 > c0:
                    clean_host[c0:c1].copy_(o.clean[c0:c1], non_blocking=True)
                pos_host[c0:c0 + n].copy_(o.comp_pos[c0:c0 + n], non_blocking=True)
                flux_host[c0:c0 + n].copy_(o.comp_flux[c0:c0 + n], non_blocking=True)
                nc_host[c0:c0 + n].copy_(o.n_comp[c0:c0 + n], non_blocking=True)
                st_host[c0:c0 + n].copy_(o.status[c0:c0 + n], non_blocking=True)
            copied[j].record(copy_stream)
    stream.wait_stream(copy_stream)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    e2e_value = B * world * args.steps / (e2e_ms / 1e3)
    assert np.array_equal(nc_host.numpy(), n_comp)
    e2e_images = ("every restored image" if n_img == B else
                  f"restored images of the first {n_img} of {B} instances (host memory)")
    del outs
    imager.out = out

    # ---- the same batch replayed from one CUDA graph (every chunk, both streams)
    imager.capture()
    barrier()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    for k in range(args.steps):
        imager.replay()
    g1.record(stream)
    barrier()
    graph_value = B * world * args.steps / (max_over_ranks(g0.elapsed_time(g1)) / 1e3)
    assert np.array_equal(imager.out.n_comp.cpu().numpy(), n_comp)

    # ---- per-phase timing (same kernels through the separate calls) for the roofline
    rec, _, st = m.uvw(wl.ant_enu, wl.pairs, ha, dec, wl.freq, cell, vis, cfg, flags=flags)
    off = torch.arange(B + 1, dtype=torch.int64, device="cuda") * wl.n_bl
    ws = m.Workspace()
    # launch shapes of the separate calls, tuned on one chunk (muser_autotune)
    tuned = {"image_variant": image_variant,
             "image_variant_meaning": "bit 0: half-width column strips in the fused gridding; bit 1: radix-8 FFT stages",
             "grid_band_rows": m.autotune(m.CALL_GRID, cfg, rec=rec, vis_off=off[:min(B, 32) + 1]),
             "dirty_column_variant": m.autotune(m.CALL_DIRTY, cfg, B=min(B, 32))}
    phase = {"grid": [], "dirty": [], "clean": [], "restore": []}
    clean_bytes, hbm_equiv_bytes = [], []
    N, G = wl.N, wl.G
    # grid, map and beam buffers of one chunk, allocated once (no timed call waits for an
    # allocation), and one untimed pass over the first chunk
    n0 = min(args.chunk, B)
    Zbuf = torch.empty((n0, G, G), dtype=torch.complex64, device="cuda")
    Dbuf = torch.empty((n0, N, N), dtype=torch.float32, device="cuda")
    Bbuf = torch.empty((n0, 2 * N, 2 * N), dtype=torch.float32, device="cuda")
    Z, stc = m.grid(rec, off[:n0 + 1], cfg, status=st[:n0].clone(), ws=ws, out=Zbuf, n_vis=n0 * wl.n_bl)
    m.dirty(Z, cfg, status=stc, ws=ws, out=(Dbuf, Bbuf))
    torch.cuda.synchronize()
    for c0 in range(0, min(B, 2 * args.chunk), args.chunk):
        n = min(args.chunk, B - c0)
        stn = st[c0:c0 + n].clone()
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        evs[0].record(stream)
        Z, stc = m.grid(rec, off[c0:c0 + n + 1], cfg, status=stn, ws=ws, out=Zbuf[:n], n_vis=(c0 + n) * wl.n_bl)
        evs[1].record(stream)
        D, Bm, stc = m.dirty(Z, cfg, status=stc, ws=ws, out=(Dbuf[:n], Bbuf[:n]))
        evs[2].record(stream)
        R, pos, flux, nc, stc = m.clean(D, Bm, cfg, status=stc, ws=ws)
        evs[3].record(stream)
        img, params, stc = m.restore(R, Bm, pos, flux, nc, cfg, status=stc)
        evs[4].record(stream)
        torch.cuda.synchronize()
        for j, k in enumerate(phase):
            phase[k].append(evs[j].elapsed_time(evs[j + 1]))
        if c0 == 0:                 # disk centring (Sec. 4.2) of the chunk's dirty maps, timed alone
            mu_a, mu_b, _ = m.gmm(D, cfg)
            cell_i = torch.tensor(np.tile(cell, len(ha))[:n], dtype=torch.float64, device="cuda")
            m.center(D, mu_a, mu_b, cell_i, cfg, ws=ws)
            ec = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
            ec[0].record(stream)
            m.center(D, mu_a, mu_b, cell_i, cfg, ws=ws)
            ec[1].record(stream)
            torch.cuda.synchronize()
            center_ms = ec[0].elapsed_time(ec[1])
            # Steer clean (Sec. 3.2) of the same chunk, 20 major cycles at clip 0.9, timed alone
            scfg = dataclasses.replace(cfg, max_iter=20)
            m.steer(D, Bm, scfg, clip=0.9, ws=ws)
            ec[0].record(stream)
            _, _, snc, _ = m.steer(D, Bm, scfg, clip=0.9, ws=ws)
            ec[1].record(stream)
            torch.cuda.synchronize()
            steer_ms = ec[0].elapsed_time(ec[1])
            steer_cycles = int(snc.sum())
        iters = nc.cpu().numpy().astype(np.float64)
        # on-chip CLEAN: beam copy (read the 2N x 2N beam, write one shifted copy), residual read
        # and written once, one N x N beam window read per iteration
        clean_bytes.append(float(np.sum(32.0 * N * N + 8.0 * N * N + iters * 4.0 * N * N)))
        hbm_equiv_bytes.append(float(np.sum(4.0 * N * N + iters * 12.0 * N * N)))
        del D, Bm, R, img
    del Z, Zbuf, Dbuf, Bbuf
    torch.cuda.empty_cache()
    clean_ms = statistics.mean(phase["clean"])
    peak, peak_kind = measured_peaks()
    tr = recorded_traffic()
    # algorithmic bytes of the CLEAN call by the streaming-residual model: every iteration reads the
    # residual and one beam window and writes the residual (12 N^2), plus the residual's first read
    stream_model = statistics.mean(hbm_equiv_bytes)
    achieved = stream_model / (clean_ms / 1e3) / 1e9
    traffic = statistics.mean(clean_bytes) * tr["dram_per_algorithmic"] if tr else None
    roofline = {"kernel": "muser_clean: k_beam_shift + k_hogbom_onchip", "bound": "latency",
                "bound_detail": ("the residual stays on chip, so DRAM is not the limit: an iteration is each "
                                 "SM's pass over its 256 KB band of L2-resident beam window (loads at the L2 "
                                 "latency of a fully loaded GPU, tensor-memory reads and writes) and then the "
                                 "16-block cluster exchange; a 256^2 kernel with no exchange iterates no faster "
                                 "under load, so the pass's latency sets the time"),
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_kind,
                "bytes_model": "12 N^2 per iteration (residual read + beam window read + residual write) + 4 N^2",
                "bytes_per_launch": stream_model, "launch_ms": clean_ms,
                "traffic": traffic,
                "traffic_source": (f"ncu dram bytes of {tr['case']}, scaled to this launch by on-chip-design "
                                   "bytes") if tr else None,
                "dram_GBps": traffic / (clean_ms / 1e3) / 1e9 if tr else None,
                "dram_frac": traffic / (clean_ms / 1e3) / 1e9 / peak if tr else None,
                "l2_frac": tr.get("lts_throughput") if tr else None,
                "onchip_design_GBps": statistics.mean(clean_bytes) / (clean_ms / 1e3) / 1e9,
                "onchip_design_bytes": "4 N^2 beam window per iteration + 8 N^2 residual in/out + 32 N^2 beam copy"}
    grid_bytes = args.chunk * (32.0 * wl.n_bl + 8.0 * G * G)
    extra = {"phase_ms_per_chunk": {k: statistics.mean(v) for k, v in phase.items()},
             "gridding_GBps": grid_bytes / (statistics.mean(phase["grid"]) / 1e3) / 1e9,
             "dirty_fft_GBps": args.chunk * (8.0 * G * G + 4.0 * G * G * 2 + 4.0 * N * N + 16.0 * N * N)
             / (statistics.mean(phase["dirty"]) / 1e3) / 1e9,
             "n_comp_min": int(n_comp.min()), "status_bits": status_histogram(status),
             "graph_replay_images_per_s": graph_value,
             "autotuned": tuned,
             "center_ms_per_chunk": center_ms,
             "center_instances_per_s": min(B, args.chunk) / (center_ms / 1e3),
             "center_GBps": min(B, args.chunk) * center_bytes(N) / (center_ms / 1e3) / 1e9,
             "steer_ms_per_chunk_20_cycles": steer_ms, "steer_instance_cycles": steer_cycles,
             "steer_us_per_instance_cycle": steer_ms * 1e3 / max(steer_cycles, 1),
             # per instance-cycle: selection 4 N^2 and update 20 N^2 bytes; the four FFT passes of
             # side 2N move 148.8 N^2 (half-planes where C or Y is zero, half beam spectrum)
             "steer_GBps": steer_bytes(N) * steer_cycles / (steer_ms / 1e3) / 1e9}

    # the extra legs need the device memory of the main batch
    del imager, out, o, vis_dev, ws, rec, st
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    if not args.no_extras and rank == 0:
        extra.update(plain_and_degrid(m, wl, cell, cfg, stream))

    cpu = None
    if rank == 0 and not args.no_extras:
        cpu = cpu_baseline()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "images/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "instances_per_gpu": B, "batch_chunk": args.chunk,
                           "l2": "inputs larger than L2: per step 17 GB of residual, 68 GB of beams (+ 1 shifted "
                                 "copy) and 283 GB of column-pass output stream through HBM"},
                "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_value, "unit": "images/s", "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h,
                        "copies": "visibilities H2D; " + e2e_images + ", component lists, counts and status D2H, "
                                  "each chunk's as soon as the library announces it (muser_image_events)"},
                "gpu_launches": gpu_launches, "clocks": clk, "extra": extra}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_case(case, n_inst=0, iters=100, size=2560):
    """Small cases of the benchmark workload, a few GB on the device, for profiler captures.

    grad:  10 eager gradient-descent steps of the 512^2 differentiable-imaging workload.

    clean: 148 instances of the MUSER-II batch (N = 1024), CLEAN with `iters` iterations.
    image0: muser_image on MUSER-II instances with max_iter 0 (the preparation kernels of the
            pipeline: uvw, strip sort, fused gridding + column pass, row pass, beam copies).
    steer: `n_inst` instances (default 8), Steer clean with `iters` major cycles at clip 0.9.
    large: the large-image leg of the benchmark at one image side (`size`).
    wproj: the w-projection leg (MUSER-I band, about `n_inst` instances) with and without it.
    mixed: the mixed stream of `n_inst` (default 10,000) MUSER-I / MUSER-II instances.
    large_clean: CLEAN (`iters` iterations) of `n_inst` (default 16) instances at side `size`.
    center: disk centring of `n_inst` (default 32) MUSER-II dirty maps.
    band2: the whole MUSER-I band (2048 instances of 512^2) with the GMM iteration estimate.
    plain1: one 256^2 image (one frame, one channel, 200 iterations) per call, device and end to end.
    steerimg: muser_image with Steer clean on four 296-instance chunks of the MUSER-II workload.
    dirty: 8 instances, gridding + FFT to dirty map and beam.
    grid:  8 instances, gridding only.
    """
    import torch
    import paper_1712_06913_b300 as m
    import synth
    if case == "mixed":
        print(json.dumps({"case": case, **mixed_stream(m, torch.cuda.current_stream(), n_total=n_inst or 10000)}))
        return
    if case == "wproj":
        print(json.dumps({"case": case, **wproj_leg(m, torch.cuda.current_stream(), n=n_inst or 296)}))
        return
    if case == "band2":
        print(json.dumps({"case": case, **config2_band(m, torch.cuda.current_stream())}))
        return
    if case == "steerimg":
        wls = synth.config3_muser2_uneven(n_frame=4, chans=list(range(296)))
        cfgs = m.Config(N=wls.N, G=wls.G, W=wls.W, os=wls.OS, gain=wls.gain, lat_rad=wls.lat)
        cells = m.pixel_size(wls.freq, wls.bmax, wls.N, wls.fov_min)
        print(json.dumps({"case": case, **steer_image_leg(m, wls, cells, cfgs, torch.cuda.current_stream())}))
        return
    if case == "plain1":
        print(json.dumps({"case": case, **config1_latency(m, torch.cuda.current_stream())}))
        return
    if case == "center":
        # disk centring (muser_center) of `n_inst` (default 32) MUSER-II dirty maps
        wlc = synth.config3_muser2_uneven(n_frame=1, chans=list(range(n_inst or 32)))
        cfgc = m.Config(N=wlc.N, G=wlc.G, W=wlc.W, os=wlc.OS, max_iter=0, gain=wlc.gain, lat_rad=wlc.lat)
        cellc = m.pixel_size(wlc.freq, wlc.bmax, wlc.N, wlc.fov_min)
        recc, _, stc = m.uvw(wlc.ant_enu, wlc.pairs, wlc.ha, wlc.dec, wlc.freq, cellc, wlc.vis, cfgc, flags=wlc.flags)
        offc = torch.arange(wlc.n_inst + 1, dtype=torch.int64, device="cuda") * wlc.n_bl
        Zc, s2 = m.grid(recc, offc, cfgc, status=stc)
        Dc, _, s2 = m.dirty(Zc, cfgc, status=s2)
        del Zc
        mu_a, mu_b, _ = m.gmm(Dc, cfgc)
        cells = torch.tensor(cellc, dtype=torch.float64, device="cuda")
        m.center(Dc, mu_a, mu_b, cells, cfgc)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        m.center(Dc, mu_a, mu_b, cells, cfgc)
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "instances": wlc.n_inst, "center_ms": e0.elapsed_time(e1)}))
        return
    if case == "large_clean":
        # streaming CLEAN of `n_inst` instances at a large image side (dirty maps built first)
        wlL = synth.muser2_large_band(size, chans=list(range(n_inst or 16)))
        cfgL = m.Config(N=size, G=4 * size, W=wlL.W, os=wlL.OS, max_iter=iters, gain=wlL.gain, lat_rad=wlL.lat)
        cellL = m.pixel_size(wlL.freq, wlL.bmax, size, wlL.fov_min)
        recL, _, stL = m.uvw(wlL.ant_enu, wlL.pairs, wlL.ha, wlL.dec, wlL.freq, cellL, wlL.vis, cfgL, flags=wlL.flags)
        B = wlL.n_inst
        offL = torch.arange(B + 1, dtype=torch.int64, device="cuda") * wlL.n_bl
        D = torch.empty((B, size, size), dtype=torch.float32, device="cuda")
        Bm = torch.empty((B, 2 * size, 2 * size), dtype=torch.float32, device="cuda")
        for i in range(B):
            Z, s2 = m.grid(recL, offL[i:i + 2], cfgL, status=stL[i:i + 1].clone())
            d, b, _ = m.dirty(Z, cfgL, status=s2)
            D[i], Bm[i] = d[0], b[0]
            del Z, d, b
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R, pos, flux, nc, _ = m.clean(D, Bm, cfgL)
        e1.record()
        torch.cuda.synchronize()
        it = float(nc.double().sum())
        print(json.dumps({"case": case, "N": size, "instances": B, "clean_ms": e0.elapsed_time(e1),
                          "GBps": 12.0 * size * size * it / (e0.elapsed_time(e1) / 1e3) / 1e9}))
        return
    if case == "large":
        print(json.dumps({"case": case, **large_images(m, torch.cuda.current_stream(), sizes=(size,))}))
        return
    if case == "grad":
        import numpy as np
        from paper_1712_06913_b300.autograd import GradientImaging
        w4 = synth.config4_operator()
        cfg4 = m.Config(N=w4.N, G=w4.G, lat_rad=w4.lat)
        cell4 = np.full(w4.n_chan, 60 * synth.ARCMIN / w4.N)
        rec, _, _ = m.uvw(w4.ant_enu, w4.pairs, w4.ha, w4.dec, w4.freq, cell4, w4.vis, cfg4, flags=w4.flags)
        obs = torch.tensor(w4.vis.reshape(-1), dtype=torch.complex64, device="cuda")
        gd = GradientImaging(rec, obs, float(np.sqrt(np.mean(np.abs(w4.vis) ** 2)) / 30.0), cfg4)
        gd.capture(steps=10)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        gd.replay(20)
        e1.record()
        torch.cuda.synchronize()
        graph_us = e0.elapsed_time(e1) * 1e3 / 200
        e0.record()
        for _ in range(20):
            gd.step()
        e1.record()
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "graph_us_per_eval": graph_us, "eager_us_per_eval": e0.elapsed_time(e1) * 1e3 / 20}))
        return
    n_inst = n_inst or (148 if case == "clean" else 8)
    wl = synth.config3_muser2_uneven(n_frame=1, chans=list(range(n_inst)))
    if case == "image0":
        cfg0 = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=0, gain=wl.gain, lat_rad=wl.lat)
        cell0 = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
        im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell0, wl.vis, cfg0, flags=wl.flags)
        im.run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        im.run()
        torch.cuda.synchronize()
        print(json.dumps({"case": case, "instances": n_inst, "s": time.perf_counter() - t0}))
        return
    cfg = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=iters, gain=wl.gain, lat_rad=wl.lat)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    rec, _, st = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    off = torch.arange(n_inst + 1, dtype=torch.int64, device="cuda") * wl.n_bl
    ws = m.Workspace()
    N = wl.N
    D = torch.empty((n_inst, N, N), dtype=torch.float32, device="cuda")
    Bm = torch.empty((n_inst, 2 * N, 2 * N), dtype=torch.float32, device="cuda")
    step = 8
    t0 = time.perf_counter()
    for c0 in range(0, n_inst, step):
        n = min(step, n_inst - c0)
        Z, s2 = m.grid(rec, off[c0:c0 + n + 1], cfg, status=st[c0:c0 + n].clone(), ws=ws)
        if case == "grid":
            break
        d, b, s2 = m.dirty(Z, cfg, status=s2, ws=ws)
        D[c0:c0 + n] = d
        Bm[c0:c0 + n] = b
        del Z, d, b
    torch.cuda.synchronize()
    if case == "steer":
        cfg.max_iter = iters
        m.steer(D, Bm, cfg, clip=0.9, ws=ws)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R, model, nc, s2 = m.steer(D, Bm, cfg, clip=0.9, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        cyc = int(nc.sum())
        print(json.dumps({"case": case, "instances": n_inst, "steer_ms": e0.elapsed_time(e1), "instance_cycles": cyc,
                          "us_per_instance_cycle": e0.elapsed_time(e1) * 1e3 / max(cyc, 1),
                          "GBps": steer_bytes(N) * cyc / (e0.elapsed_time(e1) / 1e3) / 1e9}))
        return
    if case == "clean":
        ws.buf = None
        torch.cuda.empty_cache()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        R, pos, flux, nc, s2 = m.clean(D, Bm, cfg, status=st, ws=ws)
        e1.record()
        torch.cuda.synchronize()
        it_sum = float(nc.sum().item())
        gb = (n_inst * 40.0 * N * N + it_sum * 4.0 * N * N) / 1e9   # same byte model as the roofline
        print(json.dumps({"case": case, "instances": n_inst, "clean_ms": e0.elapsed_time(e1),
                          "GBps": gb / (e0.elapsed_time(e1) / 1e3), "algorithmic_GB": gb,
                          "iterations": it_sum, "n_comp_min": int(nc.min())}))
    else:
        print(json.dumps({"case": case, "instances": n_inst, "s": time.perf_counter() - t0}))


def plain_and_degrid(m, wl, cell, cfg, stream):
    """Plain path (one image per muser_image call) and gradient evaluations/s."""
    import numpy as np
    import torch
    import synth
    from paper_1712_06913_b300.autograd import GradientImaging
    res = {}
    n_plain = 16
    cfg1 = m.Config(**{**cfg.__dict__, "batch_chunk": 0})
    ims = [m.Imager(wl.ant_enu, wl.pairs, wl.ha[:1], wl.dec[:1], wl.freq[c:c + 1], cell[c:c + 1],
                    wl.vis[:1, c:c + 1], cfg1, flags=wl.flags[:1, c:c + 1]) for c in range(n_plain)]
    for im in ims[:2]:
        im.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for im in ims:
        im.run()
    e1.record(stream)
    torch.cuda.synchronize()
    res["plain_images_per_s"] = n_plain / (e0.elapsed_time(e1) / 1e3)
    del ims
    torch.cuda.empty_cache()
    # differentiable imaging: 512^2 sky, 780 baselines x 64 channels, chi2 + gradient per evaluation
    w4 = synth.config4_operator()
    cfg4 = m.Config(N=w4.N, G=w4.G, lat_rad=w4.lat)
    cell4 = np.full(w4.n_chan, 60 * synth.ARCMIN / w4.N)
    rec, _, _ = m.uvw(w4.ant_enu, w4.pairs, w4.ha, w4.dec, w4.freq, cell4, w4.vis, cfg4, flags=w4.flags)
    obs = torch.tensor(w4.vis.reshape(-1), dtype=torch.complex64, device="cuda")
    sigma2 = float(np.mean(np.abs(w4.vis) ** 2)) / 900.0
    gd = GradientImaging(rec, obs, math.sqrt(sigma2), cfg4)
    gd.capture(steps=10)              # eta = 1/L from 20 power iterations, then 10 chained steps in a graph
    steps = 100                       # the 100-step descent of the workload: 10 replays
    torch.cuda.synchronize()
    e0.record(stream)
    gd.replay(steps // gd.graph_steps)
    e1.record(stream)
    torch.cuda.synchronize()
    res["grad_evals_per_s"] = steps / (e0.elapsed_time(e1) / 1e3)
    res["grad_eval_workload"] = ("512^2 sky, 780 baselines x 64 channels (49,920 visibilities), G=1024; one "
                                 "evaluation = forward + chi2 + adjoint + update; 100 steps as 10 replays of a "
                                 "CUDA graph of 10 chained steps")
    # eager (no graph) for comparison
    e0.record(stream)
    for _ in range(20):
        gd.step()
    e1.record(stream)
    torch.cuda.synchronize()
    res["grad_evals_per_s_eager"] = 20 / (e0.elapsed_time(e1) / 1e3)
    # algorithmic bytes of one evaluation: forward (image in, two FFT passes over the 2N x 2N
    # grid, gathers) and the adjoint (the same, transposed)
    N4, G4 = w4.N, w4.G
    ev_bytes = 2 * (4.0 * N4 * N4 + 2 * 16.0 * G4 * G4 + 8.0 * w4.vis.size)
    res["grad_GBps"] = res["grad_evals_per_s"] * ev_bytes / 1e9
    res.update(fft_vs_cufft(m, wl, cell, cfg, stream))
    del gd, obs, rec
    torch.cuda.empty_cache()
    res["large_images"] = large_images(m, stream)
    res["w_projection"] = wproj_leg(m, stream)
    res["steer_image"] = steer_image_leg(m, wl, cell, cfg, stream)
    res["config2_band"] = config2_band(m, stream)
    res["config1_plain"] = config1_latency(m, stream)
    res["mixed_stream"] = mixed_stream(m, stream)
    return res


def wproj_leg(m, stream, n=296, P=128):
    """MUSER-I band instances (N = 512, G = 2048; 1000 Hogbom iterations) imaged with and without
    w-projection (P planes, Ww-cell kernels, w_max from the instances' own records): images/s of
    each.  The kernel support is the one that resolves the w-chirp over the map's field,
    W + 2 |wg|_max / 8 cells (at most 63)."""
    import torch
    import synth
    wl = synth.config2_muser1_band(n_frame=-(-n // 64))
    cfg = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=1000, gain=wl.gain, lat_rad=wl.lat)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    rec, _, _ = m.uvw(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis,
                      m.Config(**{**cfg.__dict__, "w_planes": 2, "w_max": 1.0, "w_support": 63}), flags=wl.flags)
    w_max = float(m.record_fields(rec)[6].abs().max()) * 1.01
    del rec
    # support that resolves the chirp over the map's field (|xi| <= 1/8): W + 2 |wg| / 8
    Ww = min(63, 2 * ((wl.W + 2 * math.ceil(w_max / 8)) // 2) + 1)
    res = {"workload": f"MUSER-I band, {wl.n_inst} instances of 512^2 (G 2048), 1000 iterations"}
    for name, c in (("2d", cfg), ("wproj", m.Config(**{**cfg.__dict__, "w_planes": P, "w_max": w_max,
                                                      "w_support": Ww}))):
        im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, c, flags=wl.flags)
        im.run()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        im.run()
        e1.record(stream)
        torch.cuda.synchronize()
        res[f"{name}_images_per_s"] = wl.n_inst / (e0.elapsed_time(e1) / 1e3)
        del im
        torch.cuda.empty_cache()
    res.update(w_planes=P, w_support=Ww, w_max_grid_units=w_max)
    return res


def config2_band(m, stream):
    """The whole MUSER-I band as one batch: 64 channels x 32 frames = 2048 instances of 512^2
    (G 2048) through muser_image with the paper's iteration estimate (CLEAN down to the GMM sky
    level of each dirty map, at most 1000 iterations): images/s and the iterations run."""
    import torch
    import synth
    wl = synth.config2_muser1_band()
    # two chunks of 1024: the second chunk's gridding, transforms and GMM run beside the first
    # chunk's CLEAN (6876 against 6526 images/s as one chunk; 512: 6835, 296: 6779)
    cfg = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=wl.max_iter, gain=wl.gain, lat_rad=wl.lat,
                   thr_mode=wl.thr_mode, batch_chunk=1024)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    rec_t, _, _ = m.uvw(wl.ant_enu, wl.pairs, wl.ha[:1], wl.dec[:1], wl.freq[:32], cell[:32], wl.vis[:1, :32], cfg,
                        flags=wl.flags[:1, :32])
    variant = m.autotune(m.CALL_IMAGE, cfg, rec=rec_t, B=32)
    del rec_t
    im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    im.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = im.run()
    e1.record(stream)
    torch.cuda.synchronize()
    nc = out.n_comp.float()
    res = {"workload": f"MUSER-I band, {wl.n_inst} instances of 512^2 (G 2048), GMM threshold, cap 1000, "
                       f"chunks of {cfg.batch_chunk}",
           "images_per_s": wl.n_inst / (e0.elapsed_time(e1) / 1e3),
           "iterations_mean": float(nc.mean()), "iterations_max": int(nc.max()), "image_variant": variant}
    del im, out
    torch.cuda.empty_cache()
    return res


def config1_latency(m, stream, reps=20):
    """Config 1 (one frame, 780 baselines, 1 channel, 256^2, 200 iterations) as a plain
    pipeline: ms per image on the device (inputs resident), and end to end on the host clock
    (pinned visibilities to the device, muser_image, clean image back, synchronised)."""
    import time
    import torch
    import synth
    wl = synth.config1_plain_frame()
    cfg = m.Config(N=wl.N, G=wl.G, W=wl.W, os=wl.OS, max_iter=wl.max_iter, gain=wl.gain, lat_rad=wl.lat)
    cell = m.pixel_size(wl.freq, wl.bmax, wl.N, wl.fov_min)
    im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
    for _ in range(3):
        im.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        im.run()
    e1.record(stream)
    torch.cuda.synchronize()
    dev_ms = e0.elapsed_time(e1) / reps
    vis_h = torch.from_numpy(wl.vis.astype("complex64")).pin_memory()
    img_h = torch.empty(im.out.clean.shape, dtype=torch.float32).pin_memory()
    t0 = time.perf_counter()
    for _ in range(reps):
        im.vis.copy_(vis_h, non_blocking=True)
        out = im.run()
        img_h.copy_(out.clean, non_blocking=True)
        torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / reps
    res = {"workload": "one frame, 780 baselines, 1 channel at 1.7 GHz, 256^2 (G 1024), 200 iterations",
           "device_ms_per_image": dev_ms, "e2e_ms_per_image": e2e_ms}
    del im
    torch.cuda.empty_cache()
    return res


def mixed_stream(m, stream, n_total=10000, n_plain=8):
    """The mixed stream: n_total instances, half MUSER-I (256^2 or 512^2 by the Table 2 rule),
    half MUSER-II (1024^2), 1000 iterations, imaged by size class (MixedImager: one muser_image
    batch per class, all replayed from one CUDA graph) against the plain path (one instance per
    muser_image call), the latter timed on n_plain instances of each class."""
    import torch
    import synth
    w1, w2, _ = synth.config5_mixed_stream(n_total)
    n1 = n_total // 2

    def sources(w, n, n_max):
        F, rest = divmod(n, w.n_chan)
        kw = dict(bmax=w.bmax, fov_min=w.fov_min, n_max=n_max, max_iter=1000, lat_rad=w.lat, batch_chunk=296)
        out = [m.Source(w.ant_enu, w.pairs, w.ha[:F], w.dec[:F], w.freq, w.vis[:F], w.flags[:F], **kw)] if F else []
        if rest:
            out.append(m.Source(w.ant_enu, w.pairs, w.ha[F:F + 1], w.dec[F:F + 1], w.freq[:rest],
                                w.vis[F:F + 1, :rest], w.flags[F:F + 1, :rest], **kw))
        return out

    mix = m.MixedImager(sources(w1, n1, 512) + sources(w2, n_total - n1, 1024))
    mix.capture()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mix.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    t_batched = e0.elapsed_time(e1) / 1e3
    per_class, t_plain = {}, 0.0
    for si, c0, nc, im in mix.classes:
        n_cls = im.B
        cfg1 = m.Config(**{**im.cfg.__dict__, "batch_chunk": 0})
        ims = [m.Imager(im.ant, im.pairs, im.ha[:1], im.dec[:1], im.freq[c:c + 1], im.cell[c:c + 1],
                        im.vis[:1, c:c + 1], cfg1, flags=None if im.flags is None else im.flags[:1, c:c + 1])
               for c in range(min(n_plain, im.C))]
        ims[0].run()
        torch.cuda.synchronize()
        e0.record(stream)
        for one in ims:
            one.run()
        e1.record(stream)
        torch.cuda.synchronize()
        rate = len(ims) / (e0.elapsed_time(e1) / 1e3)
        key = f"N{im.cfg.N}"
        per_class[key] = per_class.get(key, 0) + n_cls
        t_plain += n_cls / rate
        del ims, cfg1
    res = {"instances": sum(per_class.values()), "per_class": per_class,
           "batched_images_per_s": n_total / t_batched, "plain_images_per_s": n_total / t_plain,
           "plain_sample": f"{n_plain} instances per class, one muser_image call each"}
    del mix
    torch.cuda.empty_cache()
    return res


def steer_image_leg(m, wl, cell, cfg, stream, n=296, frames=4, cycles=20):
    """Alg. 1 with the paper's production clean: `frames` chunks of `n` instances of the MUSER-II
    batch through muser_image with Steer clean (clean_variant 1, `cycles` major cycles at clip
    0.9; restore from the model map; chunk c + 1 prepared while chunk c is cleaned): images/s."""
    import torch
    chans = list(range(min(n, wl.n_chan)))
    c = m.Config(**{**cfg.__dict__, "batch_chunk": len(chans), "max_iter": cycles, "clean_variant": 1,
                    "steer_clip": 0.9})
    im = m.Imager(wl.ant_enu, wl.pairs, wl.ha[:frames], wl.dec[:frames], wl.freq[chans], cell[chans],
                  wl.vis[:frames, chans], c, flags=wl.flags[:frames, chans])
    im.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = im.run()
    e1.record(stream)
    torch.cuda.synchronize()
    res = {"instances": im.B, "chunks": frames, "major_cycles": cycles,
           "images_per_s": im.B / (e0.elapsed_time(e1) / 1e3), "cycles_run_mean": float(out.n_comp.float().mean())}
    del im, out
    torch.cuda.empty_cache()
    return res


LARGE = {1280: (148, 80), 2560: (148, 74), 5120: (64, 32)}      # N: (instances, chunk)


def large_images(m, stream, sizes=(1280, 2560, 5120)):
    """Table 2's high-band image sides through muser_image (G = 4N, 1000 Hogbom iterations,
    streaming CLEAN): images/s with inputs on the device, and the CLEAN bytes rate (read and
    write the residual and read one beam window per iteration: 12 N^2)."""
    import numpy as np
    import torch
    import synth
    res = {}
    for N in sizes:
        B, chunk = LARGE[N]
        n_band = int(((synth.muser2_channels() >= synth.LARGE_BANDS[N][0]) &
                      (synth.muser2_channels() <= synth.LARGE_BANDS[N][1])).sum())
        nf = -(-B // n_band)
        wl = synth.muser2_large_band(N, n_frame=nf, chans=list(range(min(B, n_band))))
        cfg = m.Config(N=N, G=4 * N, W=wl.W, os=wl.OS, max_iter=1000, gain=wl.gain, lat_rad=wl.lat, batch_chunk=chunk)
        cell = m.pixel_size(wl.freq, wl.bmax, N, wl.fov_min)
        warm = m.Imager(wl.ant_enu, wl.pairs, wl.ha[:1], wl.dec[:1], wl.freq[:1], cell[:1], wl.vis[:1, :1],
                        m.Config(**{**cfg.__dict__, "max_iter": 5, "batch_chunk": 0}), flags=wl.flags[:1, :1])
        warm.run()
        torch.cuda.synchronize()
        del warm
        im = m.Imager(wl.ant_enu, wl.pairs, wl.ha, wl.dec, wl.freq, cell, wl.vis, cfg, flags=wl.flags)
        im.ws.get(im.ws_bytes)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = im.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        Bt = wl.n_inst
        iters = float(out.n_comp.double().sum())
        res[f"N{N}"] = {"instances": Bt, "chunk": chunk, "ms": ms, "images_per_s": Bt / (ms / 1e3),
                        "clean_iterations": iters, "algorithmic_GBps_clean_bytes": 12.0 * N * N * iters / (ms / 1e3) / 1e9}
        del im, out
        torch.cuda.empty_cache()
    return res


def fft_vs_cufft(m, wl, cell, cfg, stream, n=32):
    """The dirty-map transform (muser_dirty: pruned column + row passes with the grid-correction
    epilogue) against cuFFT's full complex inverse 2-D FFT of the same grids (torch.fft)."""
    import torch
    rec, _, st = m.uvw(wl.ant_enu, wl.pairs, wl.ha[:1], wl.dec[:1], wl.freq[:n], cell[:n], wl.vis[:1, :n], cfg,
                       flags=wl.flags[:1, :n])
    off = torch.arange(n + 1, dtype=torch.int64, device="cuda") * wl.n_bl
    ws = m.Workspace()
    Z, st = m.grid(rec, off, cfg, status=st, ws=ws)
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for _ in range(2):
        m.dirty(Z, cfg, ws=ws)
        torch.fft.ifft2(Z)
    torch.cuda.synchronize()
    e[0].record(stream)
    for _ in range(3):
        D, Bm, _ = m.dirty(Z, cfg, ws=ws)
    e[1].record(stream)
    e[2].record(stream)
    for _ in range(3):
        F = torch.fft.ifft2(Z)
    e[3].record(stream)
    torch.cuda.synchronize()
    del F, D, Bm, Z
    return {"dirty_ms_per_instance": e[0].elapsed_time(e[1]) / 3 / n,
            "cufft_ifft2_ms_per_instance": e[2].elapsed_time(e[3]) / 3 / n,
            "fft_comparison": f"{n} MUSER-II grids of {cfg.G}^2: muser_dirty (pruned, with epilogue) vs "
                              "torch.fft.ifft2 (cuFFT, full transform, no epilogue)"}


if __name__ == "__main__":
    main()
