"""Whole-job throughput of independent replicas (one solve per GPU, no collective on the
data path): the units all ranks processed over the slowest rank's time."""
from __future__ import annotations


def replica_throughput(units: float, seconds: float):
    """Returns (units per second of the whole job, slowest rank's seconds, total units).

    Works without torch.distributed (one process) and with any initialised backend; the
    reduction tensors live on the GPU for NCCL and on the CPU otherwise."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return units / seconds, seconds, units
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return u.item() / t.item(), t.item(), u.item()
