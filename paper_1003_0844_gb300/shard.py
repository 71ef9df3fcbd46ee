"""Host-side sharding of a template grid over processes (one GPU each).

Templates (sky position, spindown) are independent, so the search shards with
no data-path exchange: rank r of W takes every W-th point of a sky lattice of
W * nsky points (each rank keeps whole skies, so its per-sky demodulation is
shared by all of its spindowns); a fixed template set such as a lattice patch is
dealt out by sky rows instead.  The only cross-rank steps are the timing
reduction of a benchmark and, in a real search, merging the candidate lists.
"""
from __future__ import annotations

import numpy as np


def sky_shard(n_per_rank: int, rank: int, world: int) -> np.ndarray:
    """Indices into a lattice of n_per_rank * world sky points owned by `rank`."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside world %d" % (rank, world))
    return np.arange(rank, n_per_rank * world, world, dtype=np.int64)


def row_shard(nrows: int, rank: int, world: int) -> np.ndarray:
    """Rows of a fixed template set (the sky rows of a lattice patch, each with its
    spindown nodes) owned by `rank`: every world-th row, so the ranks split one
    search (strong scaling) with nearly equal shares."""
    if not 0 <= rank < world:
        raise ValueError("rank %d outside world %d" % (rank, world))
    return np.arange(rank, nrows, world, dtype=np.int64)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank value over the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_candidates(sky, spin, bins, F, sky_index):
    """Merge every rank's candidates on all ranks: global sky index, spindown, bin, F,
    sorted by (sky, spindown, bin).  `sky_index` maps a rank's local sky to the lattice."""
    import torch.distributed as dist
    local = np.stack([np.asarray(sky_index)[np.asarray(sky, dtype=np.int64)], np.asarray(spin, dtype=np.int64),
                      np.asarray(bins, dtype=np.int64), np.asarray(F, dtype=np.float64).view(np.int64)], axis=1)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, local)
        allc = np.concatenate(parts, axis=0)
    else:
        allc = local
    order = np.lexsort((allc[:, 2], allc[:, 1], allc[:, 0]))
    allc = allc[order]
    return allc[:, 0], allc[:, 1], allc[:, 2], allc[:, 3].copy().view(np.float64)
