"""Assignment of evaluation points to ranks (one process per GPU).

The images b_t for different t are independent (paper Sect. 2.3: the T
evaluations share only the monomial values), so ranks take disjoint blocks
of consecutive points and need no exchange on the data path.

  weak_block(T, t0, rank)            every rank evaluates T points of its own:
                                     t0 + rank*T .. t0 + (rank+1)*T - 1
  strong_block(T, t0, rank, world)   the T points t0..t0+T-1 split into
                                     world contiguous blocks (sizes differ by
                                     at most one point)
  group_split(group_off, world)      contiguous ranges of (x1, x2) groups per
                                     rank with about equal numbers of terms:
                                     each rank owns whole output columns, so
                                     again nothing is exchanged
  job_split(costs, world)            independent jobs (a batch, a server's
                                     requests) to ranks, largest first onto
                                     the least loaded rank
"""
from typing import List, Sequence, Tuple


def weak_block(T: int, t0: int, rank: int) -> Tuple[int, int]:
    """(first point, number of points) of `rank` when each rank does T points."""
    if T < 0 or rank < 0:
        raise ValueError("T and rank must be non-negative")
    return t0 + rank * T, T


def strong_block(T: int, t0: int, rank: int, world: int) -> Tuple[int, int]:
    """(first point, number of points) of `rank` in a split of T points over `world` ranks."""
    if world < 1 or not 0 <= rank < world or T < 0:
        raise ValueError("need 0 <= rank < world and T >= 0")
    base, extra = divmod(T, world)
    first = rank * base + min(rank, extra)
    return t0 + first, base + (1 if rank < extra else 0)


def group_split(group_off: Sequence[int], world: int) -> List[Tuple[int, int]]:
    """[(first group, end group)] per rank: contiguous group ranges whose term
    counts are as even as whole groups allow (rank r ends at the first group
    boundary at or past r+1 world-th of the terms)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    G = len(group_off) - 1
    s = int(group_off[-1]) if G >= 0 else 0
    bounds, g = [0], 0
    for r in range(1, world):
        target = s * r // world
        while g < G and int(group_off[g]) < target:
            g += 1
        bounds.append(max(g, bounds[-1]))
    bounds.append(max(G, bounds[-1]))
    return [(bounds[r], bounds[r + 1]) for r in range(world)]


def job_split(costs: Sequence[float], world: int) -> List[List[int]]:
    """Job indices per rank: longest-processing-time-first greedy, which keeps
    the largest load within 4/3 of the best possible."""
    if world < 1:
        raise ValueError("world must be >= 1")
    load = [0.0] * world
    out: List[List[int]] = [[] for _ in range(world)]
    for j in sorted(range(len(costs)), key=lambda j: -costs[j]):
        r = min(range(world), key=lambda r: load[r])
        out[r].append(j)
        load[r] += costs[j]
    return out
