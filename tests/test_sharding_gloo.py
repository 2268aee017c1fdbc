"""The multi-GPU split of the point sum, checked with two gloo ranks on CPU:
each rank transforms its shard with the oracle, the partial a_lm are summed by
the same all-reduce helper the benchmark uses, and the result equals the
single-process transform (Eq. alm_def is linear in the point set)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2312_12285_gb300.sharding import allreduce_sum, shard_array, shard_bounds  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rng = np.random.default_rng(5)
    L = 24
    x, phi, w = rng.uniform(-1, 1, 1001), rng.uniform(0, 6.3, 1001), rng.uniform(0.5, 1.5, 1001)
    part = oracle.alm(shard_array(x, rank, world), shard_array(phi, rank, world), shard_array(w, rank, world), L)
    t = torch.from_numpy(part.copy())
    n = torch.tensor([float(np.sum(shard_array(w, rank, world) ** 2))], dtype=torch.float64)
    allreduce_sum([t, n])
    if rank == 0:
        full = oracle.alm(x, phi, w, L)
        out.put((float(np.max(np.abs(t.numpy() - full))), float(np.max(np.abs(full))),
                 abs(float(n[0]) - float(np.sum(w ** 2)))))
    dist.barrier()
    dist.destroy_process_group()


def test_shard_bounds_partition():
    for n in (0, 1, 7, 1000, 1001):
        for world in (1, 2, 3, 8):
            b = [shard_bounds(n, r, world) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == n
            assert all(b[i][1] == b[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in b) - min(h - l for l, h in b) <= 1


def test_two_rank_point_sharding_matches_single_transform():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    err, scale, nerr = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert err <= 1e-12 * scale
    assert nerr <= 1e-9
