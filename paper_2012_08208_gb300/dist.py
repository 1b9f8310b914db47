"""Host-side helpers for runs over several GPUs of one node (one process per GPU).

The single-problem path does not shard (one GPU per problem: ranks run
independent replicas).  Batches of independent problems shard by instance:
each rank solves its own instances, and no data crosses ranks.  The only
collectives are host-side bookkeeping: the barrier around the timed region and
the maximum of the ranks' times.
"""
from __future__ import annotations

import os


def env():
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(weights, world, rank):
    """Indices of the units that `rank` owns: longest-processing-time greedy on
    `weights` (e.g. node counts of batch instances), ties to the lower rank,
    then sorted.  Every unit goes to exactly one rank."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("need 0 <= rank < world")
    load = [0.0] * world
    owner = [0] * len(weights)
    for i in sorted(range(len(weights)), key=lambda k: (-float(weights[k]), k)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += float(weights[i])
    return [i for i in range(len(weights)) if owner[i] == rank]


def max_over_ranks(values, group=None):
    """Element-wise maximum of a list of floats over all ranks (identity for one
    process).  Uses the default process group's backend (NCCL on GPUs, gloo on
    CPU)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return [float(v) for v in values]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return [float(v) for v in t.cpu()]


def sum_over_ranks(values, group=None):
    """Element-wise sum over all ranks (identity for one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size(group) == 1:
        return [float(v) for v in values]
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return [float(v) for v in t.cpu()]


def throughput(units_per_rank, seconds_per_rank):
    """Whole-job throughput: the units of all ranks over the slowest rank's time."""
    return float(sum(units_per_rank)) / float(max(seconds_per_rank))
