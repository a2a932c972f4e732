"""Host-side multi-process plumbing: one process per GPU.

The single-grid solve does not shard (both Toeplitz directions couple the
whole grid), so N processes run N replicas. A batch of independent problems
does shard: each rank takes a disjoint subset of the problems and steps it
with no data-path collective. The only collectives are on the host's timing
scalars (max of the per-rank times, sum of the units processed).
"""


def shard(costs, rank, world):
    """Indices of the problems rank `rank` of `world` owns: longest processing
    time first over the per-problem cost estimates, so the per-rank sums of
    cost stay close. Every index lands on exactly one rank."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    owner = [0] * len(costs)
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        load[r] += costs[i]
        owner[i] = r
    return [i for i in range(len(costs)) if owner[i] == rank]


def problem_cost(n1, n2):
    """Work estimate of one CN step on an n2 x n1 grid: N log N (FFT applies)."""
    import math
    N = n1 * n2
    return N * math.log2(N + 2)


def _reduce(value, dist, op):
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(value, dist):
    """Largest per-rank value (the job's time is its slowest rank's)."""
    if dist is None:
        return float(value)
    return _reduce(value, dist, dist.ReduceOp.MAX)


def sum_over_ranks(value, dist):
    if dist is None:
        return float(value)
    return _reduce(value, dist, dist.ReduceOp.SUM)
