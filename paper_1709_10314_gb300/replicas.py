"""Multi-GPU replicas: realisations are independent, so N GPUs run N independent copies of
the sampler on disjoint Philox keys and the job's throughput is the points of all ranks
over the slowest rank's time.  No collective touches the data path; torch.distributed is
used only for the barrier and the max-reduction of the timing."""


def rank_seed(seed, rank, per_rank):
    """First Philox key of `rank`: ranks draw the disjoint key ranges
    [seed + rank * per_rank, seed + (rank + 1) * per_rank)."""
    return (seed + rank * per_rank) & (2**64 - 1)


def max_over_ranks(values, device=None):
    """Element-wise max of a list of floats over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(v) for v in values]
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_throughput(points_per_rank, world, seconds_max):
    return world * points_per_rank / seconds_max
