"""Multi-rank host logic on CPU (gloo, world size 2): disjoint hub shards of
one catalogue summed with an exact all-reduce reproduce the single-process
counts bit for bit, and the timing reduction takes the max over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import catalogs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2607_06604_gb300 import dist as gdist
        L = 80.0
        box_u = int(L * 1024)
        X = oracle.quantize(catalogs.neyman_scott(6000, L, seed=3, sigma=1.5), box_u, True)
        edges = catalogs.bin_edges_u(0.0, 8.0, 5)
        g = oracle.Graph(X, box_u, edges, nthreads=2)
        ptr, _, _ = g.export()
        lo, hi = gdist.shard_bounds(ptr, world)[rank]
        part = torch.from_numpy(g.count_3pcf(hub_lo=lo, hub_hi=hi).astype(np.int64))
        total = gdist.reduce_counts(part)
        ms, work = gdist.reduce_timing(10.0 * (rank + 1), float(part.sum()))
        if rank == 0:
            out.put((total.numpy(), g.count_3pcf().astype(np.int64), ms, work))
    finally:
        dist.destroy_process_group()


def test_hub_shards_sum_exactly_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    total, full, ms, work = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert np.array_equal(total, full)
    assert ms == 20.0 and work == float(full.sum())


def test_shard_bounds_cover_everything():
    from paper_2607_06604_gb300 import dist as gdist
    prefix = np.cumsum(np.r_[0, np.random.default_rng(1).integers(0, 50, 1000)])
    for k in (1, 2, 3, 7):
        b = gdist.shard_bounds(prefix, k)
        assert b[0][0] == 0 and b[-1][1] == 1000
        assert all(b[i][1] == b[i + 1][0] for i in range(k - 1))
