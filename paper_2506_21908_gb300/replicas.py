"""Whole-job throughput of independent replicas (one process per GPU, no data exchange).

The propagation step does not shard across GPUs in this library (each process owns a complete
system on its own GPU), so a multi-GPU run is N independent replicas.  The only cross-rank
operations are for timing: the processed units are summed and the elapsed time is the maximum
over ranks, so the job throughput is sum(units) / max(seconds).
"""
import torch
import torch.distributed as dist


def aggregate(units, seconds, device=None):
    """Return (total units over ranks, max seconds over ranks); works without a process group."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(units), float(seconds)
    dev = device if device is not None else ("cuda" if dist.get_backend() == "nccl" else "cpu")
    u = torch.tensor([float(units)], dtype=torch.float64, device=dev)
    s = torch.tensor([float(seconds)], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(s, op=dist.ReduceOp.MAX)
    return float(u.item()), float(s.item())


def throughput(units, seconds, device=None):
    total, tmax = aggregate(units, seconds, device)
    return total / tmax
