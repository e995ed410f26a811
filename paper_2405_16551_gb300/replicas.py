"""Independent replicas across GPUs: the multi-GPU form of the DE step.

A single DE generation needs donors from the whole population, so it does not
shard across GPUs without an exchange of the population every generation.
Independent runs do partition.  One process per GPU (torch.distributed) runs
its own replica of the workload, with the Philox stream id run_id = base +
rank, so that no two ranks draw the same numbers.  There is no collective on
the data path.  The job's time is the maximum of the ranks' times, and the
job's throughput is all ranks' units over that time (weak scaling).

This module holds only that host-side bookkeeping; it works with any
torch.distributed backend (NCCL on GPUs, gloo in the CPU tests).
"""
from __future__ import annotations

RUN_ID_LIMIT = 1 << 20  # the Philox counter keeps 20 bits for the run id


def replica_run_id(base_run_id: int, rank: int) -> int:
    """Philox stream id of rank `rank`'s replica."""
    rid = int(base_run_id) + int(rank)
    if not 0 <= rid < RUN_ID_LIMIT:
        raise ValueError(f"run_id {rid} out of range [0, {RUN_ID_LIMIT})")
    return rid


def max_over_ranks(values, dist=None, device=None):
    """Element-wise maximum of a list of floats over all ranks (the values
    themselves when there is no process group)."""
    vals = [float(v) for v in values]
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return vals
    import torch

    t = torch.tensor(vals, dtype=torch.float64, device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    if seconds_max <= 0:
        raise ValueError("seconds_max must be positive")
    return world * float(units_per_rank) / float(seconds_max)
