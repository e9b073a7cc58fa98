"""tc_energy_shard_dev on one GPU: the ranks of a split energy run one after
another in one process (no collective, nothing waits on another rank), and
their pairs, combined in rank order, give the whole energy."""
import numpy as np
import pytest

import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,s", [(tc.TC_FP64, 0), (tc.TC_SPLIT_BF16, 3)])
@pytest.mark.parametrize("world", [2, 3, 64])
def test_shards_combine_to_the_whole_energy(prec, s, world):
    job = synth.make_job(5, 40, 91)
    d = gpu_util.to_device(job)
    r, e_ijk = gpu_util.energy_dev(job, prec=prec, slices=s, want_trip=True, dev=d)
    ctx = gpu_util.context()
    parts = []
    for rank in range(world):
        part, res = tc.tc_energy_shard_dev(ctx, job.o, job.v, d["eps"], d["t1"], d["t2"], d["ovvv"], d["ovoo"],
                                           d["ovov"], rank, world, prec=prec, slices=s)
        first, count = tc.tc_shard_range(job.o, rank, world)
        assert res.e_t == part[0] + part[1]
        if count == 0:
            assert part == (0.0, 0.0)
        parts.append(part)
    e = tc.tc_combine_parts(parts)
    print(f"world={world} prec={prec} E={e:.15e} whole={r.e_t:.15e}")
    assert abs(e - r.e_t) <= 1e-13 * np.abs(e_ijk).sum()
