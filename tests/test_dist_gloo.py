"""Multi-rank host logic on CPU (gloo, two processes): frame/channel blocks cover every item
once, and per-rank chi-square gradients over channel blocks, summed over ranks, equal the
gradient of the whole visibility set (FP64 oracle operator on each rank's share)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1712_06913_b300 import dist as D


def test_blocks_partition_items():
    for n in (0, 1, 5, 7, 64, 528):
        for world in (1, 2, 3, 4, 8):
            got = []
            sizes = []
            for r in range(world):
                s = D.block(n, r, world)
                got.extend(range(n)[s])
                sizes.append(s.stop - s.start)
            assert got == list(range(n))
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.block(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    import synth
    from oracle import geometry
    wl = synth.small_workload(n_ant=6, N=16, config_id=241, bmax=120.0, freq=np.linspace(1.0e9, 1.6e9, 5))
    G = 2 * wl.N
    cell = np.full(wl.n_chan, 60 * synth.ARCMIN / wl.N)
    uvw = geometry.uvw(wl.ant_enu, wl.pairs, wl.lat, wl.ha, wl.dec, wl.freq)
    ro = geometry.grid_records(uvw, wl.vis, wl.flags, cell, G, 7)
    x = np.random.default_rng(5).normal(size=(wl.N, wl.N))
    return wl, G, ro, x


def _sub(ro, sl):
    return {k: v[sl] for k, v in ro.items()}


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from oracle import operator, pipeline
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert D.rank_world() == (rank, world)
        wl, G, ro, x = _case()
        ker = pipeline.spheroidal(7, 1024)
        ch = D.block(wl.n_chan, rank, world)          # this rank's channels (one frame)
        sl = slice(ch.start * wl.n_bl, ch.stop * wl.n_bl)
        mine = _sub(ro, sl)
        chi2, grad = operator.chi2_grad(x, mine, mine["vis"], 0.5, wl.N, G, ker)
        t = torch.tensor(np.concatenate([[chi2], grad.ravel()]), dtype=torch.float64)
        D.all_sum_(t)
        slowest = D.all_max(float(rank + 1))
        if rank == 0:
            chi2_all, grad_all = operator.chi2_grad(x, ro, ro["vis"], 0.5, wl.N, G, ker)
            err_c = abs(t[0].item() - chi2_all) / abs(chi2_all)
            err_g = np.abs(t[1:].numpy() - grad_all.ravel()).max() / np.abs(grad_all).max()
            q.put((err_c, err_g, slowest))
    finally:
        dist.destroy_process_group()


def test_gradient_sum_over_channel_blocks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=240)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    err_c, err_g, slowest = q.get()
    assert err_c < 1e-12 and err_g < 1e-12
    assert slowest == 2.0
