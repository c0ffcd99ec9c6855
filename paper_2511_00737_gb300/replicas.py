"""Whole-job throughput of independent replicas (one process per GPU).

The client path has no exchange step, so ranks never communicate on the data path;
the only collectives are the timing barrier and the max over ranks of the timed
region, which make the reported throughput that of the slowest replica.
"""
import torch


def max_over_ranks(value, group=None, device=None):
    """Maximum of a float over all ranks (the value itself without a process group)."""
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized():
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def job_throughput(queries_per_rank, local_ms, world, group=None, device=None):
    """(queries/s of the whole job, ms of the slowest rank): every rank processed
    queries_per_rank queries in local_ms milliseconds."""
    ms = max_over_ranks(local_ms, group, device)
    return world * queries_per_rank / (ms / 1000.0), ms
