"""The N > 1 path on CPU ranks (gloo, world size 2): sharding and timing logic.

Each rank computes its row panel of C (numpy stands in for the GPU kernel: only
the partition, the gather and the max-over-ranks timing are under test), the
panels are gathered on rank 0 and must reproduce the oracle's product, and the
LPT partition of grouped problems must cover every problem once.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1803_04014_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, result_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import synth
        from oracle import gemm as og
        m, n, k = 600, 96, 64
        A = synth.uniform((m, k), seed=1)
        B = synth.uniform((k, n), seed=2)
        start, stop = shard.row_panels(m, world, granule=128)[rank]
        # this rank's panel (same rounding as the product it stands in for)
        panel = og.gemm_mixed("f16", A[start:stop], B).astype(np.float32)
        pad = np.zeros((m, n), np.float32)
        pad[start:stop] = panel
        t = torch.from_numpy(pad)
        gathered = [torch.zeros_like(t) for _ in range(world)]
        dist.all_gather(gathered, t)
        # slowest rank decides the step time
        slow = shard.max_over_ranks(1.0 + rank, dist)
        # grouped problems spread by LPT
        sizes = synth.group_sizes(101, seed=3)
        parts, loads = shard.lpt_partition(shard.gemm_costs([tuple(s) for s in sizes]), world)
        mine = torch.tensor(sorted(parts[rank]) + [-1] * (101 - len(parts[rank])), dtype=torch.int64)
        allparts = [torch.zeros_like(mine) for _ in range(world)]
        dist.all_gather(allparts, mine)
        if rank == 0:
            C = sum(g.numpy() for g in gathered)
            ref = og.gemm_mixed("f16", A, B)
            ids = sorted(int(x) for p in allparts for x in p.tolist() if x >= 0)
            np.savez(result_path, max_dev=float(np.max(np.abs(C - ref))), slow=slow, ids=np.array(ids),
                     imbalance=max(loads) / (sum(loads) / world))
    finally:
        dist.destroy_process_group()


def test_two_cpu_ranks_shard_gather_and_time(tmp_path):
    world = 2
    out = str(tmp_path / "res.npz")
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    res = np.load(out)
    assert float(res["max_dev"]) < 1e-5          # panels gathered into the full product
    assert float(res["slow"]) == 2.0             # max over ranks
    assert list(res["ids"]) == list(range(101))  # every grouped problem exactly once
    assert float(res["imbalance"]) < 1.05


@pytest.mark.parametrize("m,world", [(8192, 1), (8192, 2), (8192, 8), (300, 4), (1, 3), (0, 2)])
def test_row_panels_cover_once(m, world):
    panels = shard.row_panels(m, world)
    assert len(panels) == world
    covered = []
    for (a, b) in panels:
        assert 0 <= a <= b <= m
        covered.extend(range(a, b))
    assert covered == list(range(m))


def test_lpt_is_balanced_and_complete():
    costs = [float(c) for c in np.random.default_rng(0).integers(1, 1000, size=500)]
    parts, loads = shard.lpt_partition(costs, 8)
    assert sorted(i for p in parts for i in p) == list(range(500))
    assert max(loads) <= sum(loads) / 8 + max(costs)   # the LPT bound
    assert shard.weak_scaling_throughput(10.0, 4, 2.0) == 20.0
