"""Receiver sharding of one scenario over several ranks (design of the multi-GPU step).

Every block of the FDP=H operator has its receivers in one cluster of the tree, and clusters are
contiguous ranges of the internal (tree) order.  Splitting the internal order into contiguous
ranges therefore gives every rank whole receiver rows of the operator: rank r owns the blocks
(admissible and inadmissible) whose receivers fall in its range and evaluates T_n for those
receivers only.  Sources are global, so the one exchange per step is an allgather of the step's
slip rate D_n (N values); in dynamic rupture each rank first solves the friction law for its own
receivers and then the solved D_n is gathered.  Rings and accumulators stay with the block's
owner.

This module holds the host side of that design: the partition (from the library's tree export)
and the exchange; the tests run it with the gloo backend on CPU ranks.
"""
import numpy as np


def receiver_ranges(perm, world):
    """Split the internal order of `perm` (internal -> geometry index, from the tree export) into
    `world` contiguous ranges of (nearly) equal size; returns the geometry indices per rank."""
    n = len(perm)
    cuts = [(n * r) // world for r in range(world + 1)]
    return [np.asarray(perm[cuts[r]:cuts[r + 1]], dtype=np.int64) for r in range(world)]


def allgather_rows(values, owners, n):
    """The full length-n vector from every rank's values for its receivers `owners[rank]`
    (the one collective of a step; ranges may differ in length by one, so they are padded)."""
    import torch
    import torch.distributed as dist
    sizes = [len(o) for o in owners]
    m = max(sizes)
    mine = torch.zeros(m, dtype=torch.float64)
    mine[:len(values)] = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64))
    bufs = [torch.empty(m, dtype=torch.float64) for _ in sizes]
    dist.all_gather(bufs, mine)
    out = np.empty(n)
    for r, o in enumerate(owners):
        out[o] = bufs[r].numpy()[:sizes[r]]
    return out
