"""Serving: continuous batching of uneven (o, v) jobs, mixed precision, on one device.

Faults are made on the host (an injected allocation failure, a paused
scheduler); nothing is faulted on the GPU.
"""
import time

import numpy as np
import pytest

import oracle
import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util

pytestmark = pytest.mark.gpu
SPLIT = tc.TC_SPLIT_BF16

MIX = [  # (o, v, seed, prec, slices)
    (6, 40, 101, tc.TC_FP64, 0), (8, 50, 102, SPLIT, 3), (5, 33, 103, SPLIT, 2), (10, 64, 104, SPLIT, 3),
    (7, 45, 105, tc.TC_FP64, 0), (4, 24, 106, SPLIT, 4), (9, 58, 107, SPLIT, 3), (12, 80, 108, SPLIT, 2),
    (6, 60, 109, tc.TC_FP64, 0), (3, 18, 110, SPLIT, 3), (1, 20, 111, SPLIT, 3), (11, 70, 112, SPLIT, 3),
]


def alone(job, prec, s):
    r, _ = gpu_util.energy_dev(job, prec=prec, slices=s)
    return r.e_t


def submit_all(ctx, jobs, device=False, devs=None):
    tickets = []
    for n, (job, prec, s) in enumerate(jobs):
        if device:
            d = devs[n]
            tickets.append(tc.tc_submit(ctx, job.o, job.v, d["eps"], d["t1"], d["t2"], d["ovvv"], d["ovoo"],
                                        d["ovov"], prec=prec, slices=s, device_inputs=True))
        else:
            tickets.append(tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov,
                                        prec=prec, slices=s))
    return tickets


def test_results_alone_equal_results_in_the_mix():
    jobs = [(synth.make_job(o, v, seed), prec, s) for (o, v, seed, prec, s) in MIX]
    ref = [alone(j, p, s) for (j, p, s) in jobs]
    ctx = tc.tc_init(0, max_inflight=8, iteration_ms=5)
    try:
        tickets = submit_all(ctx, jobs)
        for n, t in enumerate(tickets):
            st, res = tc.tc_wait(ctx, t, 120000)
            assert st == tc.TC_OK, (n, tc.status_str(st))
            assert res.e_t == ref[n], (n, res.e_t, ref[n])        # same bits alone and in the mix
            assert res.seconds >= res.queue_seconds >= 0.0
        stats = tc.tc_serve_stats_get(ctx)
        assert stats.completed == len(jobs) and stats.failed == 0
        assert stats.graph_launches == stats.iterations > 0
        assert stats.batched_jobs > stats.iterations               # launches carried several jobs
        assert stats.reserved_bytes == 0 and stats.inflight == 0
    finally:
        tc.tc_finalize(ctx)
    # and the mix agrees with the oracle
    for n in (0, 1, 2):
        j, p, s = jobs[n]
        e = oracle.energy_by_triplets(j)
        assert abs(ref[n] - e) <= (1e-9 if p == tc.TC_FP64 else 1e-6) * abs(e)


def test_wide_and_narrow_n_chunks_in_one_batch():
    """A batch runs on one W-term kernel instance: the one with eight drain
    groups as soon as one of its jobs has an N chunk wider than 224 columns
    (v = 240, 250), which then also serves the narrow jobs; each result is the
    same bits as alone."""
    spec = [(3, 240, 121, 3), (6, 40, 122, 3), (8, 50, 123, 3), (4, 250, 124, 2), (5, 33, 125, 2)]
    jobs = [(synth.make_job(o, v, seed), SPLIT, s) for (o, v, seed, s) in spec]
    ref = [alone(j, p, s) for (j, p, s) in jobs]
    ctx = tc.tc_init(0, max_inflight=8, iteration_ms=5)
    try:
        tickets = submit_all(ctx, jobs)
        for n, t in enumerate(tickets):
            st, res = tc.tc_wait(ctx, t, 120000)
            assert st == tc.TC_OK, (n, tc.status_str(st))
            assert res.e_t == ref[n], (n, res.e_t, ref[n])
        stats = tc.tc_serve_stats_get(ctx)
        assert stats.completed == len(jobs) and stats.failed == 0
        assert stats.batched_jobs > stats.iterations
    finally:
        tc.tc_finalize(ctx)


def test_device_resident_inputs():
    jobs = [(synth.make_job(o, v, seed), prec, s) for (o, v, seed, prec, s) in MIX[:6]]
    devs = [gpu_util.to_device(j) for (j, _, _) in jobs]
    ref = [alone(j, p, s) for (j, p, s) in jobs]
    ctx = tc.tc_init(0)
    try:
        tickets = submit_all(ctx, jobs, device=True, devs=devs)
        for n, t in enumerate(tickets):
            st, res = tc.tc_wait(ctx, t, 120000)
            assert st == tc.TC_OK and res.e_t == ref[n]
    finally:
        tc.tc_finalize(ctx)


def test_admission_by_hbm_footprint():
    jobs = [(synth.make_job(8, 60, 200 + n), SPLIT, 3) for n in range(6)]
    j0 = jobs[0][0]
    inputs = sum(getattr(j0, k).nbytes for k in ("eps", "t1", "t2", "ovvv", "ovoo", "ovov"))
    one = (inputs + 255) // 256 * 256 + tc.tc_workspace_bytes(8, 60, SPLIT, 3)   # one job's footprint
    ctx = tc.tc_init(0, hbm_budget_bytes=int(1.5 * one), max_inflight=8, iteration_ms=5)
    try:
        ref = [alone(j, p, s) for (j, p, s) in jobs]
        # hold the scheduler so the first admitted job keeps its memory while
        # the others are submitted (each job alone finishes in milliseconds)
        assert tc.tc_inject_fault(ctx, tc.TC_FAULT_STALL, 500) == tc.TC_OK
        tickets = submit_all(ctx, jobs)
        seen_queue = False
        for _ in range(200):
            st = tc.tc_serve_stats_get(ctx)
            assert st.reserved_bytes <= int(1.5 * one)
            seen_queue |= st.queued > 0
            if st.completed == len(jobs):
                break
            time.sleep(0.005)
        assert seen_queue                                     # jobs waited for room on the device
        for n, t in enumerate(tickets):
            st, res = tc.tc_wait(ctx, t, 120000)
            assert st == tc.TC_OK and res.e_t == ref[n]
        big = synth.make_job(20, 120, 7)
        with pytest.raises(tc.TcError) as ei:
            tc.tc_submit(ctx, big.o, big.v, big.eps, big.t1, big.t2, big.ovvv, big.ovoo, big.ovov, prec=SPLIT, slices=3)
        assert ei.value.status == tc.TC_ENOMEM
    finally:
        tc.tc_finalize(ctx)


def test_wait_timeout_cancel_and_queue_limit_with_a_paused_scheduler():
    job = synth.make_job(5, 30, 9)
    ctx = tc.tc_init(0, max_inflight=1, max_queue=2)
    try:
        assert tc.tc_inject_fault(ctx, tc.TC_FAULT_STALL, 1500) == tc.TC_OK
        t0 = tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov, prec=SPLIT, slices=3)
        time.sleep(0.2)                                       # t0 is admitted; the next ones wait
        t1 = tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov, prec=SPLIT, slices=3)
        t2 = tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov, prec=SPLIT, slices=3)
        with pytest.raises(tc.TcError) as ei:
            tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov)
        assert ei.value.status == tc.TC_EBUSY
        st, _ = tc.tc_wait(ctx, t0, 100)
        assert st == tc.TC_ETIMEOUT                           # still pending: the ticket stays valid
        assert tc.tc_poll(ctx, t0)[0] == tc.TC_ENOTREADY
        assert tc.tc_cancel(ctx, t2) == tc.TC_OK
        assert tc.tc_cancel(ctx, t0) == tc.TC_EBUSY           # already admitted
        st, res0 = tc.tc_wait(ctx, t0, 60000)
        assert st == tc.TC_OK
        st, res1 = tc.tc_wait(ctx, t1, 60000)
        assert st == tc.TC_OK and res1.e_t == res0.e_t
        assert tc.tc_poll(ctx, t2)[0] == tc.TC_ECANCELLED
        assert tc.tc_poll(ctx, t2)[0] == tc.TC_EINVAL         # released
    finally:
        tc.tc_finalize(ctx)


def test_injected_allocation_failure_fails_one_job_only():
    jobs = [(synth.make_job(6, 40, 300 + n), SPLIT, 3) for n in range(3)]
    ctx = tc.tc_init(0, max_inflight=1)
    try:
        assert tc.tc_inject_fault(ctx, tc.TC_FAULT_ALLOC) == tc.TC_OK
        tickets = submit_all(ctx, jobs)
        status = [tc.tc_wait(ctx, t, 60000)[0] for t in tickets]
        assert status[0] == tc.TC_ENOMEM
        assert status[1] == tc.TC_OK and status[2] == tc.TC_OK
        st = tc.tc_serve_stats_get(ctx)
        assert st.failed == 1 and st.completed == 2 and st.reserved_bytes == 0
    finally:
        tc.tc_finalize(ctx)


def test_invalid_submissions():
    job = synth.make_job(3, 10, 1)
    ctx = tc.tc_init(0)
    try:
        for kw in (dict(prec=5), dict(prec=SPLIT, slices=7)):
            with pytest.raises(tc.TcError) as ei:
                tc.tc_submit(ctx, job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov, **kw)
            assert ei.value.status == tc.TC_EINVAL
        assert tc.tc_poll(ctx, 987654)[0] == tc.TC_EINVAL
    finally:
        tc.tc_finalize(ctx)


def test_factor_jobs_assembled_by_the_service_equal_integral_jobs():
    """Jobs given as DF factors (the service assembles the integrals on admission)
    give the bits of the same jobs given as integral arrays, host or device
    inputs, alone and mixed with integral jobs."""
    import torch
    specs = [(6, 40, 121, tc.TC_FP64, 0), (8, 50, 122, SPLIT, 3), (5, 33, 123, SPLIT, 2), (7, 44, 124, SPLIT, 3)]
    amps = [synth.make_amplitudes(o, v, seed) for (o, v, seed, _, _) in specs]
    jobs = [synth.Job(o=a.o, v=a.v, eps=a.eps, t1=a.t1, t2=a.t2, ovvv=synth.ovvv(a), ovoo=synth.ovoo(a),
                      ovov=synth.ovov(a)) for a in amps]
    ref = [alone(j, p, s) for j, (_, _, _, p, s) in zip(jobs, specs)]
    ctx = tc.tc_init(0, max_inflight=8, iteration_ms=5)
    f = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to("cuda")
    keep = []                      # device inputs stay valid until their jobs complete
    try:
        tickets = []
        for n, (a, (o, v, _, p, s)) in enumerate(zip(amps, specs)):
            if n % 2:
                d = [f(a.eps), f(a.t1), f(a.t2), f(a.B)]
                keep.append(d)
                tickets.append(tc.tc_submit(ctx, o, v, d[0], d[1], d[2], prec=p, slices=s,
                                            device_inputs=True, B=d[3]))
            else:
                tickets.append(tc.tc_submit(ctx, o, v, a.eps, a.t1, a.t2, prec=p, slices=s,
                                            B=np.ascontiguousarray(a.B)))
            tickets.append(tc.tc_submit(ctx, o, v, jobs[n].eps, jobs[n].t1, jobs[n].t2, jobs[n].ovvv, jobs[n].ovoo,
                                        jobs[n].ovov, prec=p, slices=s))
        for n, t in enumerate(tickets):
            st, res = tc.tc_wait(ctx, t, 120000)
            assert st == tc.TC_OK, (n, tc.status_str(st))
            assert res.e_t == ref[n // 2], (n, res.e_t, ref[n // 2])
            if n % 2 == 0:
                assert 1 <= res.df_digits <= 3
        stats = tc.tc_serve_stats_get(ctx)
        assert stats.failed == 0 and stats.reserved_bytes == 0
    finally:
        tc.tc_finalize(ctx)
