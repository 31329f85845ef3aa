"""Host logic of the multi-GPU bench: independent replicas, one per rank.

A smoothing problem of these workloads fits one GB300 many times over and the
method has no exchange step across problems, so N GPUs run N independent
solves (weak scaling, no collective on the data path).  The only collective is
the timing reduction: every rank's wall time of its own K solves is reduced
with MAX, and the job's rate is all ranks' solves divided by the slowest
rank's time.
"""
from __future__ import annotations


def job_rate(units_per_rank: float, seconds: float, world: int, device=None) -> tuple:
    """(rate, max_seconds): world * units_per_rank / max over ranks of seconds.

    With world == 1 no process group is needed.  `device` is where the
    reduction tensor lives ("cpu" for gloo, a CUDA device for NCCL)."""
    if world <= 1:
        return units_per_rank / seconds, seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    worst = float(t.item())
    return world * units_per_rank / worst, worst
