"""Host-side logic of runs on several GPUs (one process per GPU).

The GEMM path shards without any exchange in its data path:

* a single GEMM splits C into row panels: rank r computes rows
  [start_r, stop_r) of C from its rows of A and all of B, and only an
  optional gather assembles C on one rank;
* grouped problems and served requests are independent units: they are
  spread over ranks by longest-processing-time-first on their cost (2mnk);
* the benchmark runs one independent replica of the workload per rank
  (weak scaling) and reports the work of all ranks over the slowest rank's
  time.

Nothing here launches kernels; collectives are used only for timing
(barrier, max over ranks) and for the optional gather.
"""
from __future__ import annotations

import heapq


def row_panels(m: int, world: int, granule: int = 256):
    """[(start, stop)] per rank: contiguous row panels of C, balanced in units of `granule` rows
    (the tile height), covering [0, m) exactly once.  Ranks beyond the work get empty panels."""
    if world < 1:
        raise ValueError("world must be >= 1")
    units = (m + granule - 1) // granule
    base, extra = divmod(units, world)
    out, u = [], 0
    for r in range(world):
        take = base + (1 if r < extra else 0)
        start = min(m, u * granule)
        stop = min(m, (u + take) * granule)
        out.append((start, stop))
        u += take
    return out


def lpt_partition(costs, world: int):
    """Assign units to ranks, largest cost first, each to the currently least-loaded rank.
    Returns (lists of unit indices per rank, load per rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    loads = [0.0] * world
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        loads[r] = load + costs[i]
        heapq.heappush(heap, (loads[r], r))
    return parts, loads


def gemm_costs(sizes):
    """2mnk per (m, n, k)."""
    return [2.0 * m * n * k for (m, n, k) in sizes]


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` of all ranks (the slowest rank decides a step's time)."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_scaling_throughput(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Work of all ranks divided by the slowest rank's time."""
    return world * units_per_rank / seconds_max
