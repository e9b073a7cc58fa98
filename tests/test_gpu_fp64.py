"""FP64 path through the C ABI against the CPU oracle (element by element per triplet)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
RTOL = 1e-9          # |dE| / |E_T| bound of the FP64 path


def check_triplets(job, e_ijk, rtol=RTOL):
    ref = {t: oracle.triplet_energy(job, *t) for t in oracle.triplet_list(job.o)}
    scale = max(abs(x) for x in ref.values()) or 1.0
    for (i, j, k), x in ref.items():
        assert abs(e_ijk[i, j, k] - x) <= rtol * scale, ((i, j, k), e_ijk[i, j, k], x)
    mask = np.ones(e_ijk.shape, bool)
    for t in ref:
        mask[t] = False
    assert np.all(e_ijk[mask] == 0.0)
    return math.fsum(ref.values())


def term_magnitude(job):
    """sum over all points of |W + V| (4|W| + |W_jki| + |W_kij| + 2|W_jik| + 2|W_ikj| + 2|W_kji|) / |D|."""
    tot = 0.0
    for a in range(job.v):
        for b in range(job.v):
            for c in range(job.v):
                W = oracle.w_ijk_all(job, a, b, c)
                V = oracle.v_ijk_all(job, a, b, c)
                D = oracle.d_ijk_all(job, a, b, c)
                A = np.abs(W)
                br = (4 * A + np.einsum("jki->ijk", A) + np.einsum("kij->ijk", A) + 2 * np.einsum("jik->ijk", A)
                      + 2 * np.einsum("ikj->ijk", A) + 2 * np.einsum("kji->ijk", A))
                tot += float(np.sum(np.abs(W + V) * br / np.abs(D)))
    return tot


def test_tiny_workload_matches_oracle_and_golden():
    job = synth.workload_job("tiny_o6_v36")
    r, e_ijk = gpu_util.energy_dev(job, want_trip=True)
    e_ref = check_triplets(job, e_ijk)
    gold = json.load(open(os.path.join(GOLDEN, "tiny_o6_v36.json")))
    assert abs(r.e_t - e_ref) <= RTOL * abs(e_ref)
    assert abs(r.e_t - gold["e_t"]) <= RTOL * abs(gold["e_t"])
    assert r.prec == tc.TC_FP64 and r.slices == 0


@pytest.mark.parametrize("o,v,seed", [(3, 5, 1), (4, 9, 2), (5, 17, 3), (2, 24, 4), (7, 13, 5), (3, 40, 6)])
def test_ragged_shapes_match_oracle(o, v, seed):
    """Several tiles, a ragged last tile, coincident-tile orbits, i=j / j=k triplets."""
    job = synth.make_job(o, v, seed)
    r, e_ijk = gpu_util.energy_dev(job, want_trip=True)
    e_ref = check_triplets(job, e_ijk)
    assert abs(r.e_t - e_ref) <= RTOL * abs(e_ref)
    assert abs(r.e_t - oracle.energy_eq1(job)) <= RTOL * abs(e_ref)


@pytest.mark.parametrize("o,v", [(1, 7), (3, 1), (1, 1)])
def test_degenerate_shapes(o, v):
    job = synth.make_job(o, v, 77)
    r, _ = gpu_util.energy_dev(job)
    ref = oracle.energy_eq1(job)
    assert abs(r.e_t - ref) <= 1e-12 * term_magnitude(job)


def test_zero_amplitudes_exact_zero():
    job = synth.make_job(4, 11, 8)
    job.t1[:] = 0.0
    job.t2[:] = 0.0
    r, _ = gpu_util.energy_dev(job)
    assert r.e_t == 0.0


def test_host_entry_equals_device_entry_bitwise():
    job = synth.make_job(5, 21, 9)
    rd, ed = gpu_util.energy_dev(job, want_trip=True)
    rh, eh = gpu_util.energy_host(job, want_trip=True)
    assert rd.e_t == rh.e_t
    np.testing.assert_array_equal(ed, eh)
    rd2, _ = gpu_util.energy_dev(job)
    assert rd2.e_t == rd.e_t                    # deterministic


def test_power_of_two_scaling_exact_on_gpu():
    job = synth.make_job(4, 19, 10)
    job.t1[:] = 0.0
    r1, _ = gpu_util.energy_dev(job)
    job.ovvv *= 2.0; job.ovoo *= 2.0; job.ovov *= 2.0; job.t2 *= 0.25
    r2, _ = gpu_util.energy_dev(job)
    assert r2.e_t == r1.e_t * (2.0 * 0.25) ** 2


def test_invalid_arguments():
    ctx = gpu_util.context()
    job = synth.make_job(2, 3, 1)
    with pytest.raises(tc.TcError) as ei:
        tc.tc_energy(ctx, 0, 3, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov)
    assert ei.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TcError) as ei:
        tc.tc_energy(ctx, 2, 3, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov, prec=7)
    assert ei.value.status == tc.TC_EINVAL


def test_budget_admission_refuses_before_work():
    import paper_2512_01055_gb300 as t
    ctx = t.tc_init(0, hbm_budget_bytes=1 << 16)
    try:
        job = synth.make_job(6, 36, 2)
        with pytest.raises(t.TcError) as ei:
            t.tc_energy(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov)
        assert ei.value.status == t.TC_ENOMEM
    finally:
        t.tc_finalize(ctx)


@pytest.mark.skipif(not os.path.exists(os.path.join(GOLDEN, "single_o20_v200.json")), reason="golden not generated")
def test_single_o20_v200_full_energy_and_triplets():
    """The o=20, v=200 workload: E_T and all 1540 triplet contributions vs the stored oracle values."""
    gold = json.load(open(os.path.join(GOLDEN, "single_o20_v200.json")))
    job = synth.workload_job("single_o20_v200")
    r, e_ijk = gpu_util.energy_dev(job, want_trip=True)
    scale = max(abs(t[3]) for t in gold["triplets"])
    for i, j, k, x in gold["triplets"]:
        assert abs(e_ijk[i, j, k] - x) <= RTOL * scale
    assert abs(r.e_t - gold["e_t"]) <= RTOL * abs(gold["e_t"])
