"""Splitting the boxes of one run across GPUs (host logic only).

The boxes of an sCOLA run never communicate after the initial conditions
(Sec. 3.2, "perfectly parallel"), so a run shards by giving each rank a
contiguous range of boxes: each rank builds the full-box initial conditions
itself, evolves only its boxes (``box_first``/``box_count`` in the problem
statement) and writes only its tiles' particles.  There is no collective on
the data path; merging the ranks' outputs is a disjoint union.
"""


def box_cost(nsc, ng):
    """Relative cost of one box: particle work plus the mesh work of the Poisson solve."""
    return nsc**3 + ng**3


def box_ranges(costs, world):
    """Contiguous (first, count) per rank with near-equal total cost; every box assigned once."""
    n = len(costs)
    if world < 1 or n < world:
        raise ValueError("need at least one box per rank")
    total = float(sum(costs))
    ranges, start, acc = [], 0, 0.0
    for r in range(world):
        if r == world - 1:
            ranges.append((start, n - start))
            break
        target = total * (r + 1) / world
        end = start + 1
        acc += costs[start]
        # leave at least one box for every remaining rank
        while end < n - (world - 1 - r) and acc + costs[end] / 2.0 <= target:
            acc += costs[end]
            end += 1
        ranges.append((start, end - start))
        start = end
    return ranges


def plan(params, world):
    """The library's native plan (scola_shard_ranges) for a problem statement: the same
    cost model and split as ``box_ranges`` over the tiling's boxes."""
    from . import binding
    return binding.scola_shard_ranges(params, world)


def merge_disjoint(parts, fill_value):
    """Union of per-rank arrays in which each rank filled only its own entries."""
    import numpy as np
    out = np.array(parts[0], copy=True)
    for p in parts[1:]:
        mask = ~np.isnan(p) if np.isnan(fill_value) else (p != fill_value)
        out[mask] = p[mask]
    return out
