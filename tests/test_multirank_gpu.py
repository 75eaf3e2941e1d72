"""The sharded N > 1 path with the CUDA library as each rank's evaluator.

Two gloo ranks (spawned processes on the one GPU of this machine; their
kernels never wait on each other) each evaluate their contiguous shard of the
points through the C-ABI, and rank 0 gathers the shards by host copy
(sharding.gather_points).  With a fixed node split length
(SC_OPT_NODES_PER_SPLIT) every point's sum runs in the same order whatever the
partition, so the gathered field equals the unsharded one bit for bit; with
the autotuned splits it agrees to the FP32 gate.
"""
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_path, split_nodes):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import paper_1609_08146_gb300 as sc
    from paper_1609_08146_gb300 import workloads as wl
    from paper_1609_08146_gb300.sharding import gather_points, shard_range

    w = wl.sweep(1e4, 64, n_points=333)
    mc = w["mirror"]
    ctx = sc.Context(0)
    if split_nodes:
        ctx.set_option(sc.SC_OPT_NODES_PER_SPLIT, split_nodes)
    m = ctx.mirror(mc["f"], mc["r_min"], mc["r_max"], mc["n_r"], mc["n_theta"])
    inc = ctx.incident(profile="gauss", w0=w["beam"]["w0"], spectrum=w["spectrum"])
    om = w["omegas"][:100]
    pts = torch.tensor(w["points"], device="cuda")
    lo, hi = shard_range(pts.shape[0], rank, world)
    E, B = ctx.eval(m, inc, om, pts[lo:hi])
    torch.cuda.synchronize()
    Eg = gather_points(torch.view_as_real(E), pts.shape[0], dim=1)
    if rank == 0:
        E0, _ = ctx.eval(m, inc, om, pts)
        torch.cuda.synchronize()
        np.save(out_path, np.stack([Eg.numpy().ravel(), torch.view_as_real(E0).cpu().numpy().ravel()]))
    ctx.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("split_nodes", [1024, 0])
def test_sharded_cuda_path_equals_unsharded(tmp_path, split_nodes):
    out = str(tmp_path / "gathered.npy")
    mp.spawn(_worker, args=(2, _free_port(), out, split_nodes), nprocs=2, join=True)
    a = np.load(out)
    if split_nodes:
        assert np.array_equal(a[0], a[1])
    else:
        g = a[0].reshape(100, 333, 3, 2)
        r = a[1].reshape(100, 333, 3, 2)
        num = np.sqrt(np.mean(np.sum((g - r) ** 2, axis=(2, 3)), axis=1))
        den = np.max(np.sqrt(np.sum(r ** 2, axis=(2, 3))), axis=1)
        assert np.max(num / den) <= 1e-5
