"""Two processes over gloo (CPU): the sky sharding partitions the lattice, the row
dealing of a fixed lattice patch, the benchmark's max-over-ranks timing reduction,
and the candidate merge that is the only cross-rank exchange of a sharded search."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1003_0844_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n_per_rank = 7
        idx = shard.sky_shard(n_per_rank, rank, world)
        parts = [None] * world
        dist.all_gather_object(parts, idx.tolist())
        # this rank's "candidates": local sky index, spindown, bin, F
        rng = np.random.default_rng(rank)
        k = 5 + rank
        sky = rng.integers(0, n_per_rank, k)
        spin = rng.integers(0, 3, k)
        bins = rng.integers(0, 1000, k)
        F = rng.uniform(20, 40, k)
        gs, gm, gb, gF = shard.gather_candidates(sky, spin, bins, F, idx)
        t = shard.max_over_ranks(10.0 + rank)
        # a fixed lattice patch of 11 sky rows dealt out by rows; candidates merge by row index
        rows = shard.row_shard(11, rank, world)
        rparts = [None] * world
        dist.all_gather_object(rparts, rows.tolist())
        lsky = np.arange(rows.size)
        rs, _, _, _ = shard.gather_candidates(lsky, np.zeros(rows.size), np.zeros(rows.size), np.ones(rows.size),
                                              rows)
        out[rank] = (parts, (gs.tolist(), gm.tolist(), gb.tolist(), gF.tolist()), t, rparts, rs.tolist())
    finally:
        dist.destroy_process_group()


def test_two_rank_sharding_timing_and_candidate_merge():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    parts0 = res[0][0]
    allidx = sorted(parts0[0] + parts0[1])
    assert allidx == list(range(7 * world))          # complete
    assert not set(parts0[0]) & set(parts0[1])        # disjoint
    assert res[0][2] == res[1][2] == 11.0             # max over ranks
    rparts = res[0][3]
    assert sorted(rparts[0] + rparts[1]) == list(range(11)) and not set(rparts[0]) & set(rparts[1])
    assert abs(len(rparts[0]) - len(rparts[1])) <= 1  # nearly equal shares
    assert res[0][4] == res[1][4] == list(range(11))  # one candidate per row, merged in row order
    assert res[0][1] == res[1][1]                     # every rank holds the same merged list
    gs, gm, gb, gF = res[0][1]
    assert len(gs) == 5 + 6
    keys = list(zip(gs, gm, gb))
    assert keys == sorted(keys)
    # each candidate's global sky index belongs to the rank that produced it
    for r in range(world):
        rng = np.random.default_rng(r)
        k = 5 + r
        sky = rng.integers(0, 7, k)
        spin = rng.integers(0, 3, k)
        bins = rng.integers(0, 1000, k)
        F = rng.uniform(20, 40, k)
        for a, b, c, f in zip(np.array(parts0[r])[sky], spin, bins, F):
            assert (int(a), int(b), int(c)) in set(keys)
            assert f in gF


def test_single_process_shard_is_identity():
    assert shard.sky_shard(5, 0, 1).tolist() == list(range(5))
    assert shard.max_over_ranks(3.5) == 3.5
    with pytest.raises(ValueError):
        shard.sky_shard(5, 2, 2)
    assert shard.row_shard(5, 0, 1).tolist() == list(range(5))
    with pytest.raises(ValueError):
        shard.row_shard(5, -1, 2)
