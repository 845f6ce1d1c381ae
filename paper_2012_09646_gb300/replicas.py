"""Replicas on several GPUs of one node: the DAG scheduler runs one program
on one device (the paper leaves multi-GPU scheduling to future work), so N
GPUs run N independent replicas of the workload, one process each, with no
data exchanged.  What the ranks share is the measurement: a barrier around
the timed region, the job time as the maximum over the ranks, the whole-job
throughput as every rank's units over that time (weak scaling), and one
report printed by rank 0.  Works with any torch.distributed backend (NCCL on
GPUs, gloo on the CPU)."""
from __future__ import annotations

import os


def rank_env():
    """(rank, world size, local rank) of this process, from the launcher's
    environment (1 process when unset)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def job_time_ms(dist, ms_local, device="cpu"):
    """The job's time: the slowest rank's (max over ranks); the local time
    when there is no process group."""
    if dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms):
    """Whole-job throughput in units per second: every rank processed
    `units_per_rank` units in the job time `ms`."""
    return world * units_per_rank * 1e3 / ms


def reports(rank):
    """Only rank 0 prints the job's report."""
    return rank == 0
