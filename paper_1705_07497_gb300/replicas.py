"""Replica bookkeeping for running independent reconstructions on several
GPUs, one process per GPU.

Slices are independent problems, so the data path has no collective: every
rank reconstructs its own slices.  The only communication is timing: a
barrier before and after the timed region and the maximum of the ranks'
times, so that the job's throughput is the work of all ranks divided by the
slowest rank's time.  Works with any torch.distributed backend (NCCL on GPUs,
gloo on CPUs).
"""

import os


def rank_info():
    """(rank, world size, local rank) from the launcher's environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rank_seed(base_seed, rank):
    """Seed of the slice a rank reconstructs: each rank gets its own data."""
    return int(base_seed) + int(rank)


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(value, world, device=None):
    """Maximum of a per-rank float over all ranks (the value itself when world == 1)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_rank, seconds):
    """Units processed by all ranks per second of the slowest rank."""
    return world * units_per_rank / seconds
