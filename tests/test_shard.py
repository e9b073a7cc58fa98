"""One energy split over ranks (host logic, CPU): the triplet partition, the
rank-local compensated pair and the rank-order combination, with two gloo
ranks exchanging their pairs through paper_2512_01055_gb300.shard.

Without a GPU each rank's triplet contributions come from the oracle; the
partition, the pair and the combination are the library's own host code
(tc_shard_range, tc_sum_parts, tc_combine_parts), the same that
tc_energy_shard_dev uses on a device.
"""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
import paper_2512_01055_gb300 as tc
from paper_2512_01055_gb300 import build, shard


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    tc.load()


def _triplets(o):
    return [t for t in oracle.triplet_list(o) if t[0] != t[2]]


@pytest.mark.parametrize("o,world", [(1, 1), (1, 3), (2, 2), (5, 2), (7, 3), (20, 8), (40, 7), (3, 16)])
def test_ranges_cover_every_triplet_once(o, world):
    n = len(_triplets(o))
    nxt = 0
    for r in range(world):
        first, count = tc.tc_shard_range(o, r, world)
        assert first == nxt and count >= 0
        assert abs(count - n / world) < 1.0          # equal shares: every triplet costs the same
        nxt = first + count
    assert nxt == n


def test_invalid_shards_are_rejected():
    for args in ((0, 0, 1), (4, 2, 2), (4, -1, 2), (4, 0, 0)):
        with pytest.raises(tc.TcError):
            tc.tc_shard_range(*args)


def test_pairs_and_combination_are_compensated():
    rng = np.random.default_rng(5)
    x = rng.standard_normal(1000) * 10.0 ** rng.integers(-8, 8, 1000)
    s, c = tc.tc_sum_parts(x)
    assert abs((s + c) - math.fsum(x)) <= 4e-16 * np.abs(x).sum()
    parts = [tc.tc_sum_parts(x[a:a + 250]) for a in range(0, 1000, 250)]
    e = tc.tc_combine_parts(parts)
    assert abs(e - math.fsum(x)) <= 4e-16 * np.abs(x).sum()
    assert tc.tc_sum_parts([]) == (0.0, 0.0)
    assert tc.tc_combine_parts([(1.0, 0.0), (2.0 ** -60, 0.0), (-1.0, 0.0)]) == 2.0 ** -60


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, o, v, seed, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        tc.load()
        job = synth.make_job(o, v, seed)
        first, count = tc.tc_shard_range(o, rank, world)
        mine = _triplets(o)[first:first + count]
        part = tc.tc_sum_parts([oracle.triplet_energy(job, *t) for t in mine])
        parts = shard.gather_parts(part)
        out[rank] = (tc.tc_combine_parts(parts), parts, [tuple(t) for t in mine])
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_give_one_energy(world):
    o, v, seed = 5, 14, 77
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), o, v, seed, out), nprocs=world, join=True)
    e = [out[r][0] for r in range(world)]
    assert len(set(e)) == 1                          # the same bits on every rank
    covered = sorted(t for r in range(world) for t in out[r][2])
    assert covered == sorted(_triplets(o))
    ref = oracle.energy_by_triplets(synth.make_job(o, v, seed))
    assert abs(e[0] - ref) <= 1e-14 * abs(ref)
