"""Whole-grid assignment of a batch of independent grids to ranks.

The paper scales its design by splitting the problem into independent
compute units, each owning part of the domain and exchanging nothing with
the others while they compute (Sec. 5).  Across GPUs the units here are
whole grids: every rank computes the same assignment from the grid sizes
alone (no communication), marches its own grids in one batched launch, and
the job is timed by the slowest rank.  There is no data-path collective,
because the grids share no cells.
"""


def assign_grids(sizes, world):
    """Indices of the grids each of `world` ranks takes, balancing cells.

    sizes: cells (or any work measure) per grid.  Longest-processing-time
    order: grids by decreasing size (ties by index), each to the rank with
    the least work so far (ties by rank).  Deterministic, so every rank
    derives the same lists.  The largest load exceeds the mean by at most one
    grid's size.  Each rank's list is in increasing grid order.
    """
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0] * world
    out = [[] for _ in range(world)]
    for q in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        out[r].append(q)
        load[r] += sizes[q]
    return [sorted(x) for x in out]
