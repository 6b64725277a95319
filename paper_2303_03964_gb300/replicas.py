"""Multi-GPU form of the layout iteration: independent replicas, one process per GPU.

One graph's iteration runs on one GPU; the library has no step that exchanges data
between GPUs. Several GPUs either run the same workload side by side (weak scaling:
per-GPU work fixed) or split a list of independent graphs among themselves (`shard`).
The only collectives are host-side: barriers around a timed region and the reduction
of the per-rank times (max) and counts (sum). They run on whatever process group is
initialised: NCCL with CUDA tensors, gloo with CPU tensors.
"""
import os


def world():
    """(world_size, rank, local_rank) from the launcher's environment (1, 0, 0 alone)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def _group():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        return dist
    return None


def _tensor(x):
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    return torch.tensor([float(x)], dtype=torch.float64, device=dev)


def barrier():
    dist = _group()
    if dist is not None:
        dist.barrier()


def max_over_ranks(x):
    """Largest x over all ranks (x itself without a process group)."""
    dist = _group()
    if dist is None:
        return float(x)
    t = _tensor(x)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x):
    """Sum of x over all ranks (x itself without a process group)."""
    dist = _group()
    if dist is None:
        return float(x)
    t = _tensor(x)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard(count, rank, world_size):
    """Contiguous share [lo, hi) of `count` independent items for `rank`: the shares of
    all ranks partition range(count) and differ in size by at most one."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("rank %d outside world of %d" % (rank, world_size))
    return range(count * rank // world_size, count * (rank + 1) // world_size)


def throughput(units_per_rank, seconds_per_rank):
    """Whole-job rate: units processed by all ranks over the slowest rank's time."""
    units = sum_over_ranks(units_per_rank)
    return units / max_over_ranks(seconds_per_rank)
