"""Multi-process host logic on CPU (gloo, world size 2): source shards cover
every source once, and the all-reduced partial gradients equal the full
gradient (computed here by the oracle, standing in for each rank's GPU)."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_09882_gb300.shard import source_range


def test_source_range_partition():
    for n in (0, 1, 7, 32, 1000, 134217728):
        for w in (1, 2, 3, 8):
            rs = [source_range(n, r, w) for r in range(w)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(rs[i][1] == rs[i + 1][0] for i in range(w - 1))
            sizes = [b - a for a, b in rs]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import oracle
    from paper_2605_09882_gb300.shard import sharded_gradient
    from tinytrees import random_octree
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(9)
    keys, lev, _ = random_octree(rng, 1, 4, 0.4)
    src = rng.random((37, 3))
    dirs = oracle.healpix(1)
    g = rng.standard_normal((37, 12, 2))

    def local(s0, s1):
        return torch.from_numpy(oracle.adjoint(keys, lev, 2, src[s0:s1], dirs, g[s0:s1], nthreads=1))

    tot = sharded_gradient(37, local)
    full = oracle.adjoint(keys, lev, 2, src, dirs, g, nthreads=1)
    q.put((rank, float(np.abs(tot.numpy() - full).max()), float(np.abs(full).max())))
    dist.destroy_process_group()


def test_sharded_gradient_gloo_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, scale in res:
        assert err <= 1e-12 * scale, (rank, err)
