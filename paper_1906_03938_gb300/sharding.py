"""Host-side partition of independent projection problems over ranks (one GPU per rank).

The projections of different problems share nothing (Section 3: each problem has its own
mesh, contour and basis), so a multi-GPU run splits the problem list with no collective on
the data path; only the timings are reduced (max over ranks). The split balances the work
n^2 N of each problem by the longest-processing-time rule: problems in decreasing work,
each to the rank with the least work so far (ties to the lower rank), which is within 4/3
of the optimal makespan.
"""


def shard_by_cost(costs, world):
    """Index lists, one per rank, for problems of the given costs."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        shards[r].append(i)
        load[r] += costs[i]
    return [sorted(s) for s in shards]


def rank_share(costs, rank, world):
    """The problem indices of one rank."""
    return shard_by_cost(costs, world)[rank]
