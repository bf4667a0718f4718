"""Host logic of multi-process runs (one process per GPU, torch.distributed).

A single grid does not shard without an all-to-all transpose per axis change,
so a grid runs as independent replicas: each rank advances its own copy, the
ranks meet at a barrier around the timed region, the time is the maximum over
ranks and the throughput counts the cells of all replicas.  Independent
problems (the instances of a parameter scan, the trajectories of a training
set) are partitioned across ranks instead, balanced by their cost, with no
collective on the data path: only the timing and the per-instance results are
gathered at the end.  Data-parallel training of the surrogate has the one real
exchange: the gradients are averaged over the ranks before each Adam step.

Every function works with any process-group backend (nccl for CUDA tensors,
gloo for CPU tensors), so the logic is tested with gloo ranks on the CPU.
"""
from __future__ import annotations

import heapq
import math
from typing import List, Sequence


def world() -> int:
    import torch.distributed as dist
    return dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1


def rank() -> int:
    import torch.distributed as dist
    return dist.get_rank() if dist.is_available() and dist.is_initialized() else 0


def _device():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def max_over_ranks(x: float) -> float:
    """The largest x of all ranks (x itself without a process group)."""
    if world() == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    if world() == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def average_gradients(buf) -> None:
    """Data-parallel training: replace buf (a tensor on this backend's device)
    by its mean over the ranks, in place, with one all-reduce.  Training the
    surrogate is the one exchange step of the path: each rank computes the
    gradients of its own minibatch, and every rank then applies the same mean
    gradient, so the replicas' parameters stay identical."""
    n = world()
    if n == 1:
        return
    import torch.distributed as dist
    dist.all_reduce(buf, op=dist.ReduceOp.SUM)
    buf.div_(n)


def barrier() -> None:
    if world() > 1:
        import torch.distributed as dist
        dist.barrier()


def scan_cost(n: int) -> float:
    """Relative cost of one step of an n x n instance: n^2 log2 n (FFT passes)."""
    return float(n) * n * math.log2(max(n, 2))


def partition_by_cost(costs: Sequence[float], nparts: int) -> List[List[int]]:
    """Split item indices into nparts lists of nearly equal total cost: the
    largest item first onto the least-loaded part (ties by part index), each
    list in increasing index order.  Deterministic, so every rank computes the
    same partition without communicating."""
    if nparts < 1:
        raise ValueError("nparts must be >= 1")
    parts: List[List[int]] = [[] for _ in range(nparts)]
    heap = [(0.0, p) for p in range(nparts)]
    for i in sorted(range(len(costs)), key=lambda i: (-costs[i], i)):
        load, p = heapq.heappop(heap)
        parts[p].append(i)
        heapq.heappush(heap, (load + float(costs[i]), p))
    return [sorted(p) for p in parts]


def gather_objects(obj) -> list:
    """obj of every rank, in rank order."""
    if world() == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world()
    dist.all_gather_object(out, obj)
    return out


def replica_throughput(cells: int, steps: int, seconds: float) -> float:
    """Whole-job cell-steps/s of replicated grids: every rank's cells over the
    slowest rank's time."""
    return world() * cells * steps / max_over_ranks(seconds)


def sharded_throughput(local_cell_steps: float, seconds: float) -> float:
    """Whole-job cell-steps/s of partitioned independent problems."""
    return sum_over_ranks(local_cell_steps) / max_over_ranks(seconds)
