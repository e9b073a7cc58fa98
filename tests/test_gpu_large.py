"""Full-size workloads (o=40 v=400, o=50 v=450): sampled occupied triplets against the oracle.

The whole oracle energy at these sizes would take days on the host, so the
check is element by element on a fixed sample of triplet contributions --
distinct indices, i = j, j = k, first and last occupied orbitals, and seeded
random triplets -- whose oracle values tests/golden/make_golden.py --sampled
stored.  Both GPU precisions compute them through tc_triplets_dev in the
launch configuration of a full run (same tiles, same work items per triplet).

Physical-scale twin: t1 and t2 scaled by mu = 2^-17 (exact in binary
floating point) put |E_T| near 0.1 Eh; the oracle's contributions scale by
exactly mu^2 (pinned on the oracle), so the literal 1e-6 Eh bound is checked
on the whole energy projected from the sample: n_trip x the mean |dE| per
sampled triplet, which bounds the total error if every triplet erred alike.
"""
import json
import os

import numpy as np
import pytest

import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util
from tests.split_bounds import split_rel_bound

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
MU = 2.0 ** -17


def _golden(name):
    rec = json.load(open(os.path.join(GOLDEN, f"sampled_{name}.json")))
    return [tuple(t[:3]) for t in rec["triplets"]], np.array([t[3] for t in rec["triplets"]])


@pytest.mark.parametrize("name", ["precision_o40_v400", "large_o50_v450"])
def test_sampled_triplets_full_size(name):
    import torch
    o, v = synth.WORKLOADS[name]
    trip, ref = _golden(name)
    amp = synth.make_amplitudes(o, v, synth.WORKLOAD_SEEDS[name])
    dev = synth.device_job(amp)
    for x in sorted({x for t in trip for x in t})[:4]:   # device and host integrals are the same bits
        assert torch.equal(dev["ovvv"][x].cpu(), torch.from_numpy(synth.ovvv_slice(amp, x)))
    assert torch.equal(dev["ovoo"].cpu(), torch.from_numpy(synth.ovoo(amp)))
    scale = np.abs(ref).max()
    n_trip = o * (o + 1) * (o + 2) // 6 - o
    ctx = gpu_util.context()

    def run(t1, t2, prec, s=0):
        e, _ = tc.tc_triplets_dev(ctx, o, v, dev["eps"], t1, t2, dev["ovvv"], dev["ovoo"], dev["ovov"], trip,
                                  prec=prec, slices=s)
        return e

    e64 = run(dev["t1"], dev["t2"], tc.TC_FP64)
    print(name, "fp64 max rel", np.abs(e64 - ref).max() / scale)
    assert np.all(np.abs(e64 - ref) <= 1e-9 * scale)
    for s in (2, 3, 4):
        es = run(dev["t1"], dev["t2"], tc.TC_SPLIT_BF16, s)
        rel = np.abs(es - ref).max() / scale
        print(name, f"split s={s} max rel {rel:.3e}, sample-sum rel {abs(es.sum() - ref.sum()) / abs(ref.sum()):.3e}")
        assert rel <= split_rel_bound(s, o, v)
    t1m, t2m = dev["t1"] * MU, dev["t2"] * MU
    ref_tw = ref * MU * MU
    e_tw_total = n_trip * ref_tw.mean()
    assert 0.01 < abs(e_tw_total) < 1.0, e_tw_total
    for s in (3, 4):
        et = run(t1m, t2m, tc.TC_SPLIT_BF16, s)
        proj = n_trip * np.abs(et - ref_tw).mean()
        print(name, f"twin s={s}: projected E_T {e_tw_total:.4f} Eh, projected |dE| <= {proj:.2e} Eh")
        assert proj <= 1e-6


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
