"""Full-size workloads (o=40 v=400, o=50 v=450): sampled occupied triplets against the oracle.

The whole oracle energy at these sizes would take days on the host, so the
check is element by element on a sample of triplet contributions -- distinct
indices, i = j, j = k, first and last occupied orbitals -- computed by both GPU
precisions through tc_triplets_dev in the launch configuration of a full run
(same tiles, same work items per triplet).
"""
import numpy as np
import pytest

import oracle
import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util

pytestmark = pytest.mark.gpu


def sample_triplets(o):
    return [(o - 1, o - 2, 0), (o // 2, o // 3, o // 5), (o - 1, o - 1, 1), (o // 2, 2, 2), (1, 0, 0),
            (o - 1, o // 2, o // 2 - 1)]


@pytest.mark.parametrize("name", ["precision_o40_v400", "large_o50_v450"])
def test_sampled_triplets_full_size(name):
    import torch
    o, v = synth.WORKLOADS[name]
    amp = synth.make_amplitudes(o, v, synth.WORKLOAD_SEEDS[name])
    dev = synth.device_job(amp)
    trip = sample_triplets(o)
    occ = sorted({x for t in trip for x in t})
    slices = {x: synth.ovvv_slice(amp, x) for x in occ}
    for x in occ:                                  # device and host integrals are the same bits
        assert torch.equal(dev["ovvv"][x].cpu(), torch.from_numpy(slices[x]))
    hjob = synth.Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2, ovvv=None,
                     ovoo=synth.ovoo(amp), ovov=synth.ovov(amp))
    assert torch.equal(dev["ovoo"].cpu(), torch.from_numpy(hjob.ovoo))
    ref = np.array([oracle.triplet_energy(hjob, *t, ovvv_slices=slices) for t in trip])
    scale = np.abs(ref).max()
    ctx = gpu_util.context()
    args = (ctx, o, v, dev["eps"], dev["t1"], dev["t2"], dev["ovvv"], dev["ovoo"], dev["ovov"], trip)
    e64, r64 = tc.tc_triplets_dev(*args, prec=tc.TC_FP64)
    print(name, "fp64 max rel", np.abs(e64 - ref).max() / scale)
    assert np.all(np.abs(e64 - ref) <= 1e-9 * scale)
    for s in (2, 3):
        es, rs = tc.tc_triplets_dev(*args, prec=tc.TC_SPLIT_BF16, slices=s)
        print(name, f"split s={s} max rel", np.abs(es - ref).max() / scale, "per-triplet rel",
              np.abs(es - ref) / np.abs(ref))
        assert np.all(np.abs(es - ref) <= 1e-6 * scale)


def test_subset_equals_full_run_contributions():
    job = synth.make_job(6, 40, 31)
    ctx = gpu_util.context()
    d = gpu_util.to_device(job)
    for prec, s in ((tc.TC_FP64, 0), (tc.TC_SPLIT_BF16, 3)):
        r, e_ijk = gpu_util.energy_dev(job, prec=prec, slices=s, want_trip=True, dev=d)
        trip = [(5, 3, 1), (4, 4, 0), (2, 1, 1), (3, 3, 3), (5, 3, 1)]
        e, rr = tc.tc_triplets_dev(ctx, job.o, job.v, d["eps"], d["t1"], d["t2"], d["ovvv"], d["ovoo"], d["ovov"],
                                   trip, prec=prec, slices=s)
        for m, t in enumerate(trip):
            assert abs(e[m] - e_ijk[t]) <= 1e-12 * np.abs(e_ijk).max()
        assert e[3] == 0.0
        assert rr.e_t == pytest.approx(e.sum(), rel=1e-12)


def test_subset_rejects_bad_triplets():
    job = synth.make_job(4, 10, 3)
    ctx = gpu_util.context()
    d = gpu_util.to_device(job)
    for bad in ([(1, 2, 0)], [(4, 1, 0)], [(2, 1, -1)]):
        with pytest.raises(tc.TcError) as ei:
            tc.tc_triplets_dev(ctx, job.o, job.v, d["eps"], d["t1"], d["t2"], d["ovvv"], d["ovoo"], d["ovov"], bad)
        assert ei.value.status == tc.TC_EINVAL
