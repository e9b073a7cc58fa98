"""E[5]_ST, the part of E_(T) from the V factor of Eq. 1, against the oracle (both precisions)."""
import dataclasses

import numpy as np
import pytest

import oracle
import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util

pytestmark = pytest.mark.gpu
SPLIT = tc.TC_SPLIT_BF16


@pytest.mark.parametrize("o,v,seed", [(4, 9, 31), (5, 17, 32), (3, 40, 33)])
@pytest.mark.parametrize("prec,slices", [(tc.TC_FP64, 0), (SPLIT, 3)])
def test_e5_matches_oracle(o, v, seed, prec, slices):
    job = synth.make_job(o, v, seed)
    r, _ = gpu_util.energy_dev(job, prec=prec, slices=slices)
    e4, e5 = oracle.energy_parts_eq1(job)
    if prec == tc.TC_FP64:
        tol = 1e-9 * (abs(e4) + abs(e5))
    else:
        tol = 1e-6 * max(1.0, abs(e4 + e5))
    assert abs(r.e_t5 - e5) <= tol, (r.e_t5, e5)
    assert abs((r.e_t - r.e_t5) - e4) <= tol, (r.e_t - r.e_t5, e4)


@pytest.mark.parametrize("prec,slices", [(tc.TC_FP64, 0), (SPLIT, 3)])
def test_e5_zero_without_t1_and_odd_in_t1(prec, slices):
    job = synth.make_job(5, 21, 34)
    r, _ = gpu_util.energy_dev(job, prec=prec, slices=slices)
    r0, _ = gpu_util.energy_dev(dataclasses.replace(job, t1=np.zeros_like(job.t1)), prec=prec, slices=slices)
    rm, _ = gpu_util.energy_dev(dataclasses.replace(job, t1=-job.t1), prec=prec, slices=slices)
    assert r0.e_t5 == 0.0
    assert r.e_t5 != 0.0 and rm.e_t5 == -r.e_t5
