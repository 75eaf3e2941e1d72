"""The N > 1 path on CPU with gloo ranks (world size 2).

Sharding points across ranks (no exchange during the sum) and gathering the
shards by host copy reproduces the unsharded result bit for bit; the per-rank
field evaluation is stood in for by the oracle, since this test has no GPU.
The benchmark's timing reductions (barrier, max and sum over ranks) run over
the same process group.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1609_08146_gb300.sharding import gather_points, shard_range


def test_shard_range_covers_and_balances():
    for n in (0, 1, 5, 17, 4160):
        for world in (1, 2, 3, 8):
            ranges = [shard_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(ranges[i][1] == ranges[i + 1][0] for i in range(world - 1))
            sizes = [e - b for b, e in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    import bench
    from paper_1609_08146_gb300 import workloads as wl

    w = wl.sweep(1e3, 16, n_points=37)
    m, b = wl.oracle_args(w)
    om = w["omegas"][::32]
    lo, hi = shard_range(len(w["points"]), rank, world)
    E, B = oracle.field(m, b, om, w["points"][lo:hi], threads=1)
    Eg = gather_points(torch.from_numpy(E), len(w["points"]), dim=1)
    # timing reductions of bench.py over the same group
    bench.barrier(dist)
    mx = bench.max_over_ranks(dist, float(rank + 1))
    sm = bench.sum_over_ranks(dist, float(rank + 1))
    if rank == 0:
        E0, _ = oracle.field(m, b, om, w["points"], threads=1)
        np.save(out_path, np.stack([Eg.numpy().ravel(), E0.ravel()]))
        with open(out_path + ".txt", "w") as f:
            f.write("%g %g" % (mx, sm))
    dist.destroy_process_group()


def test_sharded_equals_unsharded_over_gloo(tmp_path):
    out = str(tmp_path / "gathered.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    a = np.load(out)
    assert np.array_equal(a[0], a[1])
    mx, sm = map(float, open(out + ".txt").read().split())
    assert mx == 2.0 and sm == 3.0
