"""Host-side helpers for running independent solves on several GPUs (one
process per GPU).

The waveform-relaxation path has no exchange step between GPUs: every GPU runs
whole, independent solves (replicas of one problem, or a shard of a batch or
request stream), so ranks never communicate on the data path.  The only
collectives are the barrier around a timed region and the max-reduction of its
duration (the job is as slow as its slowest rank)."""


def shard(sizes, rank, world):
    """Indices of the units (batch members, requests) that `rank` of `world` runs.

    Longest-processing-time-first assignment by size (ties to the lower rank),
    deterministic on every rank, so the shards partition range(len(sizes)) and
    their total sizes differ by at most the largest unit."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    load = [0] * world
    owner = [0] * len(sizes)
    for i in sorted(range(len(sizes)), key=lambda j: (-sizes[j], j)):
        r = min(range(world), key=lambda q: (load[q], q))
        owner[i] = r
        load[r] += sizes[i]
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(value, dist=None, device=None):
    """The largest `value` over all ranks (returns `value` without a process group)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, dist=None, device=None):
    """The sum of `value` over all ranks (units processed by the whole job)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
