"""Assignment of evaluation points to ranks (one process per GPU).

The images b_t for different t are independent (paper Sect. 2.3: the T
evaluations share only the monomial values), so ranks take disjoint blocks
of consecutive points and need no exchange on the data path.

  weak_block(T, t0, rank)            every rank evaluates T points of its own:
                                     t0 + rank*T .. t0 + (rank+1)*T - 1
  strong_block(T, t0, rank, world)   the T points t0..t0+T-1 split into
                                     world contiguous blocks (sizes differ by
                                     at most one point)
"""
from typing import Tuple


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
