"""Replica sharding across GPUs (one process per GPU).

Replicas of NMFA runs are independent (Algorithm 1 draws every replica from its own
noise stream), so N GPUs simply run N batches: rank k anneals its batch on noise
stream id `base_stream + k` and no data crosses GPUs while annealing.  The only
collectives are host-side bookkeeping after a run: a gather of every rank's
energies (and optionally signs) to rank 0, and a max-reduction of elapsed times
for whole-job throughput.  Works with the nccl (GPU tensors) and gloo (CPU tensors)
backends of torch.distributed.
"""
from __future__ import annotations


def init_ranks(backend: str, timeout_s: float = 120.0, device_id=None, rank=None, world_size=None):
    """torch.distributed.init_process_group with a finite timeout: a rank that never
    joins, or that dies between steps, ends the other ranks' rendezvous or next
    collective with an error after `timeout_s` instead of a hang.  Rank and world
    size come from the environment (torchrun) unless given."""
    import datetime

    import torch.distributed as dist

    kw = {"timeout": datetime.timedelta(seconds=float(timeout_s))}
    if device_id is not None:
        kw["device_id"] = device_id
    if rank is not None:
        kw["rank"] = int(rank)
        kw["world_size"] = int(world_size)
    dist.init_process_group(backend, **kw)


def rank_stream(rank: int, base_stream: int = 0) -> int:
    """Noise stream id of rank `rank`'s replica batch."""
    return base_stream + rank


def gather_to_rank0(tensor):
    """All ranks pass an equally shaped tensor; rank 0 receives [world, *shape]
    (other ranks get None).  Uses all_gather so that it also works on gloo."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size()
    parts = [torch.empty_like(tensor) for _ in range(world)]
    dist.all_gather(parts, tensor.contiguous())
    return torch.stack(parts) if dist.get_rank() == 0 else None


def max_over_ranks(value: float, device=None) -> float:
    """The largest of the ranks' values (whole-job time of a weakly scaled step)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
