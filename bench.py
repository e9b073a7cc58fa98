#!/usr/bin/env python
"""Benchmark of the (T) correction: (T) TFLOP/s and seconds per energy.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--prec split|fp64] [--slices S]

A step is one full (T) energy -- every hot-path stage: BF16 slicing into
tensor-core images (split path), work tables, the W-term GEMM and orbit-energy
kernels (split path; the FP64 path has one fused W/V/energy kernel), the
compensated reduction and the read-back of E_T -- on one seeded synthetic job
whose inputs are resident in HBM before timing starts.  The inputs (ovvv
alone is 20.5 GB at o=40, v=400) exceed the 129 MB L2, so no L2 flush is
needed between steps.

Headline ("value"): the split-precision path (BF16 slices, s = --slices) on
the precision workload o=40, v=400 (Q = 1320).  Beside it: one energy at each
other slice count (2, 3, 4); the FP64 tensor-core path and every slice count
on a fixed sample of occupied triplets (tc_triplets_dev, the launch
configuration of a full run) against the oracle's stored values for the same
triplets, with the FP64 seconds per energy projected from the sample (one
full FP64 energy takes about an hour at this size; --fp64-full times one);
and the same energy end to end through the host entry point.

With N > 1 (torchrun) every rank solves its own copy of the job (independent
problems, no collective on the data path): weak scaling, value = total
energies' FLOPs / max-over-ranks time.

--impl reference times the CPU oracle (the tests' ground truth) on one seeded
occupied triplet per step of the same workload, on this host's cores, and
projects it to the whole energy.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

FP64_NOMINAL_TF = 1.25          # GB300 nominal dense FP64 (TFLOP/s)
BF16_NOMINAL_TF = 2250.0        # GB300 nominal dense BF16 (TFLOP/s)
FALLBACK_BF16_TF = 1900.0
FALLBACK_HBM = 6800.0


def alg_flops(o, v):
    return 2.0 * (o ** 3 * v ** 4 + o ** 4 * v ** 3)


def max_over_ranks(x, dist, device):
    """The job's time is the slowest rank's: MAX all-reduce of one float (x itself when dist is None)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        m = json.load(open(p))
        return (m.get("bf16_tflops", FALLBACK_BF16_TF), m.get("bf16_tflops_sustained"),
                m.get("hbm_gbs", FALLBACK_HBM), "measured")
    return FALLBACK_BF16_TF, None, FALLBACK_HBM, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()

    def summary(self):
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def kernel_source_hash(prec):
    """Hash of the kernel source with comments and blank lines removed (a comment edit keeps it)."""
    import re
    names = ["tc_fp64.cu"] if prec == "fp64" else ["tc_split.cu", "tc_ptx.cuh"]
    paths = [os.path.join(ROOT, "paper_2512_01055_gb300", "csrc", n) for n in names]
    if not all(os.path.exists(p) for p in paths):
        return None
    src = re.sub(r"/\*.*?\*/", "", "".join(open(p).read() for p in paths), flags=re.S)
    src = "\n".join(line.split("//")[0].rstrip() for line in src.splitlines())
    src = "\n".join(line for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def recorded_traffic(kernel, workload, prec):
    """DRAM bytes per launch from a committed ncu summary, if taken on the current kernel source."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    rec = json.load(open(p)).get(f"{kernel}:{workload}")
    if not rec or rec.get("source_sha") != kernel_source_hash(prec):
        return None
    return rec.get("dram_bytes_per_launch")


def golden_sample(name):
    """(triplets, oracle contributions, source) of the stored sample of a workload, or None.

    The values were written by tests/golden/make_golden.py from the oracle only:
    a fixed sample of occupied triplets for the full-size workloads, every
    triplet for the o=20 v=200 one (of which the same kind of sample is taken).
    """
    g = os.path.join(ROOT, "tests", "golden")
    p = os.path.join(g, f"sampled_{name}.json")
    if os.path.exists(p):
        rec = json.load(open(p))
        return [tuple(t[:3]) for t in rec["triplets"]], np.array([t[3] for t in rec["triplets"]]), os.path.basename(p)
    p = os.path.join(g, f"{name}.json")
    if os.path.exists(p):
        rec = json.load(open(p))
        o = rec["o"]
        want = [(o - 1, o - 2, 0), (o // 2, o // 3, o // 5), (o - 1, o - 1, 1), (o // 2, 2, 2), (1, 0, 0),
                (o - 1, o // 2, o // 2 - 1)]
        val = {tuple(t[:3]): t[3] for t in rec["triplets"]}
        return want, np.array([val[t] for t in want]), os.path.basename(p)
    return None


class CpuMeter:
    """Wall time and the process's CPU time (all threads) over a region: cores actually used = cpu / wall."""

    def __enter__(self):
        self.w0, self.c0 = time.perf_counter(), os.times()
        return self

    def __exit__(self, *a):
        c1 = os.times()
        self.wall = time.perf_counter() - self.w0
        self.cpu = (c1.user - self.c0.user) + (c1.system - self.c0.system)

    @property
    def cores_used(self):
        return self.cpu / max(self.wall, 1e-9)


def host_job(name, amp=None):
    """The workload's oracle inputs on the host without the o v^3 array: (amp, job); ovvv slices come per triplet."""
    o, v = synth.WORKLOADS[name]
    if amp is None:
        amp = synth.make_amplitudes(o, v, synth.WORKLOAD_SEEDS[name])
    job = synth.Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2, ovvv=None, ovoo=synth.ovoo(amp), ovov=synth.ovov(amp))
    return amp, job


def oracle_triplet_seconds(amp, job, trip):
    """Time oracle.triplet_energy on one triplet (its ovvv slices are formed before the clock starts)."""
    import oracle
    sl = {x: synth.ovvv_slice(amp, x) for x in set(trip)}
    with CpuMeter() as m:
        e = oracle.triplet_energy(job, *trip, ovvv_slices=sl)
    return e, m


def oracle_sample(amp, job, budget_s, seed=4242):
    """Time the oracle on seeded triplets until budget_s is spent: (projected s/energy, cores used, sample text)."""
    import oracle
    trip = [t for t in oracle.triplet_list(job.o) if t[0] != t[2]]
    order = np.random.default_rng(seed).permutation(len(trip))
    wall = cpu = 0.0
    done = 0
    while done < len(order) and (done == 0 or wall < budget_s):
        _, m = oracle_triplet_seconds(amp, job, trip[order[done]])
        wall += m.wall
        cpu += m.cpu
        done += 1
    proj = wall / done * len(trip)
    return proj, cpu / wall, (f"{done} of {len(trip)} occupied triplets (oracle.triplet_energy), {wall:.1f} s, "
                              f"projected to all")


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def workload_config(name, args):
    o, v = synth.WORKLOADS[name]
    return {"workload": name, "o": o, "v": v, "Q": 3 * (o + v), "prec": args.prec, "slices": args.slices,
            "l2": ("inputs larger than L2 (ovvv %.2f GB): no flush needed" if 8.0 * o * v ** 3 > 129e6
                   else "inputs fit in L2 (ovvv %.2f GB): small workload, not timed for a bench line")
                  % (8.0 * o * v ** 3 / 1e9)}


def reference_arm(args, name, o, v, flops, metric):
    """The oracle as it stands, one sampled occupied triplet per step, projected to the whole energy."""
    import oracle
    amp, job = host_job(name)
    trip = [t for t in oracle.triplet_list(o) if t[0] != t[2]]
    order = np.random.default_rng(4242).permutation(len(trip))
    walls, used = [], []
    for s in range(args.warmup + args.steps):
        _, m = oracle_triplet_seconds(amp, job, trip[order[s % len(order)]])
        if s >= args.warmup:
            walls.append(m.wall)
            used.append(m.cores_used)
    per_trip = statistics.mean(walls)
    val = flops / (per_trip * len(trip)) / 1e12
    sample = (f"one seeded occupied triplet per step (oracle.triplet_energy), {args.steps} timed steps, "
              f"mean {per_trip:.2f} s per triplet, projected to all {len(trip)} triplets")
    cfg = workload_config(name, args)
    print(json.dumps({
        "impl": "reference", "metric": metric, "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * per_trip,
        "step": "one sampled occupied triplet", "projected": True,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": round(statistics.mean(used), 1),
                         "cores_available": cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}))


def serving_requests(n, fp64_share, slices):
    """The seeded request stream: (o, v, seed, prec, slices) per request and Poisson arrival offsets (s, rate 1)."""
    reqs = []
    for r in range(n):
        o, v = synth.serving_request_shape(r)
        u = float(synth.uniform(synth.SERVING_SEED_BASE + r, 98, 0, 1)[0])
        fp64 = u < fp64_share
        reqs.append((o, v, synth.SERVING_SEED_BASE + r, 0 if fp64 else 1, 0 if fp64 else slices))
    gaps = -np.log1p(-synth.uniform(synth.SERVING_ARRIVAL_SEED, 1, 0, n))
    return reqs, np.cumsum(gaps)


def serving(args):
    """Continuous-batching service on one GPU: p50/p99 latency and jobs/s at a stated arrival rate.

    The seeded stream: request r has o ~ U{6..32}, v = round(o U[6,12]),
    Q = 3 (o + v), its own seed, and arrives at a Poisson time.  A client
    thread draws each request's inputs on the device (the seeded generator's
    device twin: orbital energies, amplitudes and the density-fitting factor)
    shortly before its arrival, with at most --lookahead-gb of drawn but
    unfinished inputs; at the arrival time the request is submitted with its
    device arrays and its factor (TC_JOB_DEVICE_INPUTS, nq = Q: the service
    assembles the integrals on admission), and its arrays are released once it
    completes.  Latency = completion - the scheduled arrival (so any client
    delay counts against the service).
    """
    import threading
    import torch
    import paper_2512_01055_gb300 as tc
    from paper_2512_01055_gb300 import build as tcbuild
    if int(os.environ.get("RANK", "0")) != 0:
        return
    torch.cuda.set_device(0)
    tcbuild.build()
    reqs, offs = serving_requests(args.requests, args.fp64_share, args.slices)
    flops = [alg_flops(o, v) for (o, v, _, _, _) in reqs]
    # service-time model for the arrival rate: FP64 ~0.9 TF/s; split 130 TF/s at s = 3 (the
    # service's aggregate rate over the mix of sizes; large jobs alone reach ~200), scaled by the
    # slice pairs, plus a fixed 30 ms per job (tables, images, reduction)
    est = [f / (0.9e12 if p == 0 else 130e12 * 6.0 / (s * (s + 1) / 2)) + 0.03
           for f, (_, _, _, p, s) in zip(flops, reqs)]
    capacity = 1.0 / max(1e-9, float(np.mean(est)))
    rate = args.rate if args.rate > 0 else args.load * capacity
    arrivals = offs / rate
    free0, total_mem = torch.cuda.mem_get_info()
    budget = int(args.budget_frac * free0)
    ctx = tc.tc_init(0, hbm_budget_bytes=budget, max_inflight=16, iteration_ms=50)
    n = len(reqs)
    devs = [None] * n
    ready = [threading.Event() for _ in range(n)]
    tickets = [None] * n
    submit_t = [None] * n
    results = [None] * n
    pending_bytes = [0]
    cv = threading.Condition()
    done = threading.Event()
    gen_s = [0.0]
    lookahead = args.lookahead_gb * 1e9

    def nbytes(o, v):
        return 8.0 * (3 * (o + v) ** 3 + o * o * v * v + o * v + o + v)

    def generator():
        st = torch.cuda.Stream()
        for r, (o, v, seed, _, _) in enumerate(reqs):
            with cv:
                cv.wait_for(lambda: pending_bytes[0] + nbytes(o, v) <= lookahead or pending_bytes[0] == 0)
                pending_bytes[0] += nbytes(o, v)
            t0 = time.perf_counter()
            with torch.cuda.stream(st):
                d = synth.make_amplitudes_device(o, v, seed, "cuda")
            st.synchronize()
            gen_s[0] += time.perf_counter() - t0
            devs[r] = d
            ready[r].set()

    def collector():
        # poll every submitted request, so a finished small job releases its
        # inputs while a large one still runs
        nxt, outstanding, left = 0, [], n
        while left:
            while nxt < n and tickets[nxt] is not None:
                outstanding.append(nxt)
                nxt += 1
            still = []
            for r in outstanding:
                st_, res = tc.tc_poll(ctx, tickets[r])
                if st_ == tc.TC_ENOTREADY:
                    still.append(r)
                    continue
                results[r] = (st_, res.seconds, res.queue_seconds, res.e_t)
                devs[r] = None
                left -= 1
                with cv:
                    pending_bytes[0] -= nbytes(reqs[r][0], reqs[r][1])
                    cv.notify_all()
            outstanding = still
            time.sleep(0.005)
        done.set()

    gth = threading.Thread(target=generator, daemon=True)
    cth = threading.Thread(target=collector, daemon=True)
    gth.start()
    cth.start()
    late = []
    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        for r, (o, v, _, prec, s) in enumerate(reqs):
            delay = arrivals[r] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            ready[r].wait()
            submit_t[r] = time.perf_counter() - t0
            late.append(submit_t[r] - arrivals[r])
            d = devs[r]
            tickets[r] = tc.tc_submit(ctx, o, v, d["eps"], d["t1"], d["t2"], prec=prec, slices=s,
                                      device_inputs=True, B=d["B"])
        done.wait()
        makespan = time.perf_counter() - t0
    stats = tc.tc_serve_stats_get(ctx)
    tc.tc_finalize(ctx)
    ok = [r for r in range(n) if results[r][0] == tc.TC_OK]
    lat = np.array([late[r] + results[r][1] for r in ok])
    que = np.array([results[r][2] for r in ok])

    def pct(x):
        return ({"n": int(len(x)), "p50_s": float(np.percentile(x, 50)), "p99_s": float(np.percentile(x, 99)),
                 "mean_s": float(np.mean(x))} if len(x) else {"n": 0})

    by_prec = {}
    for name, p in (("fp64", 0), ("split", 1)):
        by_prec[name] = pct(np.array([late[r] + results[r][1] for r in ok if reqs[r][3] == p]))
    buckets = {}
    for name, lo, hi in (("small <1e13 flop", 0, 1e13), ("medium 1e13-1e14", 1e13, 1e14), ("large >=1e14", 1e14, 1e99)):
        buckets[name] = pct(np.array([late[r] + results[r][1] for r in ok if lo <= flops[r] < hi]))
    out = {
        "metric": "serving latency", "unit": "s", "higher_is_better": False, "n_gpus": 1,
        "value": float(np.percentile(lat, 99)), "p50_s": float(np.percentile(lat, 50)),
        "p99_s": float(np.percentile(lat, 99)), "mean_s": float(lat.mean()),
        "queue_p50_s": float(np.percentile(que, 50)), "queue_p99_s": float(np.percentile(que, 99)),
        "client_late_p99_s": float(np.percentile(late, 99)),
        "jobs_per_s": len(ok) / makespan, "tflops_aggregate": sum(flops[r] for r in ok) / makespan / 1e12,
        "rate_per_s": rate, "offered_load": rate / capacity, "capacity_model_jobs_per_s": capacity,
        "requests": n, "completed": len(ok), "fp64_requests": int(sum(1 for q in reqs if q[3] == 0)),
        "by_precision": by_prec, "by_size": buckets,
        "makespan_s": makespan, "input_generation_s": gen_s[0],
        "iterations": stats.iterations, "graph_launches": stats.graph_launches,
        "mean_jobs_per_launch": stats.batched_jobs / max(1, stats.iterations),
        "hbm_budget_gb": budget / 1e9,
        "clocks": clk.summary(),
        "data": "synthetic (seeded request stream drawn on the device; DF factors, integrals assembled by the service)",
        "config": {"workload": "serving", "o": "U{6..32}", "v": "round(o*U[6,12])", "Q": "3(o+v)",
                   "fp64_share": args.fp64_share, "slices": args.slices, "prefix_of_stream": args.requests,
                   "arrivals": "Poisson (seeded)"},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="precision_o40_v400", choices=sorted(synth.WORKLOADS) + ["serving"])
    ap.add_argument("--prec", default="split", choices=["split", "fp64"])
    ap.add_argument("--slices", type=int, default=3)
    ap.add_argument("--fp64-full", action="store_true",
                    help="also time one full FP64 energy (default only when it takes under a minute)")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--cpu-baseline-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=24, help="serving: requests of the seeded stream to run")
    ap.add_argument("--rate", type=float, default=0.0, help="serving: arrivals per second (0: --load x capacity)")
    ap.add_argument("--load", type=float, default=0.5, help="serving: offered load relative to estimated capacity")
    ap.add_argument("--fp64-share", type=float, default=0.5, help="serving: fraction of FP64 requests")
    ap.add_argument("--budget-frac", type=float, default=0.55,
                    help="serving: the library's HBM budget as a fraction of free device memory")
    ap.add_argument("--lookahead-gb", type=float, default=40.0,
                    help="serving: device memory for drawn but unfinished request inputs")
    args = ap.parse_args()
    if args.workload == "serving":
        return serving(args)
    if args.prec == "fp64":
        args.slices = 0

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    name = args.workload
    o, v = synth.WORKLOADS[name]
    flops = alg_flops(o, v)
    metric = "(T) TFLOP/s"

    if args.impl == "reference":
        if rank == 0:
            reference_arm(args, name, o, v, flops, metric)
        return

    import torch
    import paper_2512_01055_gb300 as tc
    from paper_2512_01055_gb300 import build as tcbuild

    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
        if rank == 0:
            tcbuild.build()
        dist.barrier()
    else:
        torch.cuda.set_device(0)
        tcbuild.build()
    dev_id = torch.cuda.current_device()
    device = f"cuda:{dev_id}"

    head_prec = tc.TC_FP64 if args.prec == "fp64" else tc.TC_SPLIT_BF16
    head_slices = args.slices
    # inputs: the seeded DF factor and amplitudes drawn on the host, the integral
    # blocks formed from them on the device (exact: B sits on a 2^-20 grid)
    t_gen = time.perf_counter()
    amp = synth.make_amplitudes(o, v, synth.WORKLOAD_SEEDS[name])
    dev = synth.device_job(amp, device)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t_gen
    names = ("eps", "t1", "t2", "ovvv", "ovoo", "ovov")
    ctx = tc.tc_init(dev_id)
    stream = torch.cuda.current_stream()

    def step(prec, slices):
        return tc.tc_energy_dev(ctx, o, v, dev["eps"], dev["t1"], dev["t2"], dev["ovvv"], dev["ovoo"], dev["ovov"],
                                prec=prec, slices=slices, stream=stream)

    def timed(prec, slices, warmup, steps, sample_clocks):
        r = None
        for _ in range(warmup):
            r = step(prec, slices)
        e_ref = r.e_t if r is not None else None
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        kern, wterm, prep, launches = [], [], [], 0
        clk = ClockSampler(dev_id) if sample_clocks else None
        if clk:
            clk.__enter__()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            r = step(prec, slices)
            kern.append(r.kernel_seconds)
            wterm.append(r.wterm_seconds)
            prep.append(r.prep_seconds)
            launches += r.launches
            assert e_ref is None or r.e_t == e_ref, "energy changed between steps"
            e_ref = r.e_t
        ev1.record(stream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        if clk:
            clk.__exit__()
        t = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dist, device)
        return {"sec": t / steps, "e_t": e_ref, "e_t5": r.e_t5, "kernel": statistics.mean(kern),
                "wterm": statistics.mean(wterm), "prep": statistics.mean(prep), "launches": launches,
                "clocks": clk.summary() if clk else None}

    split_counts = (2, 3, 4) if head_prec == tc.TC_SPLIT_BF16 else ()
    if split_counts:
        step(head_prec, max(split_counts))      # the largest workspace first: later calls reuse it
    head = timed(head_prec, head_slices, args.warmup, args.steps, True)
    # the other slice counts: one energy each, same device-side timing
    per_slices = {}
    for s in split_counts:
        r = head if s == head_slices else timed(head_prec, s, 0, 1, False)
        per_slices[str(s)] = {"s_per_energy": r["sec"], "e_t": r["e_t"], "wterm_ms": 1e3 * r["wterm"],
                              "tflops": flops / r["sec"] / 1e12}

    # sampled occupied triplets through tc_triplets_dev (the launch configuration of
    # a full run) against the oracle's stored values for the same triplets
    sampled = None
    gs = golden_sample(name)
    n_trip_all = o * (o + 1) * (o + 2) // 6 - o
    if gs is not None:
        trip, ref, src = gs
        scale = float(np.abs(ref).max())
        args_t = (ctx, o, v, dev["eps"], dev["t1"], dev["t2"], dev["ovvv"], dev["ovoo"], dev["ovov"], trip)
        e64, r64 = tc.tc_triplets_dev(*args_t, prec=tc.TC_FP64, stream=stream)
        sampled = {"triplets": len(trip), "source": src, "oracle_sum": float(ref.sum()),
                   "fp64": {"max_abs": float(np.abs(e64 - ref).max()),
                            "max_rel": float(np.abs(e64 - ref).max() / scale),
                            "s_per_energy_projected": r64.kernel_seconds * n_trip_all / len(trip)}}
        for s in split_counts:
            es, _ = tc.tc_triplets_dev(*args_t, prec=head_prec, slices=s, stream=stream)
            sampled[f"split_s{s}"] = {"max_abs": float(np.abs(es - ref).max()),
                                      "max_rel": float(np.abs(es - ref).max() / scale),
                                      "abs_dE_sample_sum": float(abs(es.sum() - ref.sum())),
                                      "rel_dE_sample_sum": float(abs(es.sum() - ref.sum()) / abs(ref.sum())),
                                      "abs_dE_vs_fp64_sample_sum": float(abs(es.sum() - e64.sum()))}

    # end to end through the host entry point: pinned host inputs -> E_T on the host
    host = {}
    for k in names:
        pt = torch.empty(dev[k].shape, dtype=torch.float64, pin_memory=True)
        pt.copy_(dev[k])
        host[k] = pt.numpy()
    h2d = sum(host[k].nbytes for k in names)

    def host_step():
        return tc.tc_energy(ctx, o, v, host["eps"], host["t1"], host["t2"], host["ovvv"], host["ovoo"], host["ovov"],
                            prec=head_prec, slices=head_slices)

    host_step()
    if dist:
        dist.barrier()
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        re = host_step()
        assert re.e_t == head["e_t"], (re.e_t, head["e_t"])
    te = max_over_ranks((time.perf_counter() - t0) / e2e_steps, dist, device)
    del host

    # the same energy from the DF factor (tc_energy_df_dev: the integral blocks
    # assembled on the device as exact digit products on the tensor cores)
    Bdev = torch.from_numpy(np.ascontiguousarray(amp.B)).to(device)
    rdf = tc.tc_energy_df_dev(ctx, o, v, Bdev, dev["eps"], dev["t1"], dev["t2"], prec=head_prec, slices=head_slices,
                              stream=stream)
    df_line = {"entry": "tc_energy_df_dev", "df_seconds": rdf.df_seconds, "digits": rdf.df_digits,
               "kernel_seconds": rdf.kernel_seconds, "df_over_kernel": rdf.df_seconds / rdf.kernel_seconds,
               "s_per_energy": rdf.seconds, "same_e_t": rdf.e_t == head["e_t"]}
    del Bdev

    fp64 = None
    if head_prec != tc.TC_FP64 and (args.fp64_full or flops < 5e13):
        fp64 = timed(tc.TC_FP64, 0, 1, 1, False)

    bf16_peak, bf16_sus, hbm, src = peaks()
    # the dominant kernel: the fused kernel (FP64) or the W-term GEMMs (split), its own
    # CUDA-event time summed over its launches inside the timed steps.  Its launches run
    # back to back for the whole energy, so the sustained (power-capped) peak applies.
    peak_bf16 = bf16_sus or bf16_peak
    which = "sustained" if bf16_sus else "burst"
    if head_prec == tc.TC_FP64:
        kname, pairs = "tc_fp64_kernel", 1
        peak = peak_bf16 * FP64_NOMINAL_TF / BF16_NOMINAL_TF
        peak_note = f"FP64 tensor (DMMA) peak = {src} bf16 {which} x nominal FP64/BF16 ratio 1.25/2250"
    else:
        kname, pairs = "tc_wterm_kernel", head_slices * (head_slices + 1) // 2
        peak = peak_bf16
        peak_note = (f"BF16 dense {src} {which} peak (the kernel's launches run back to back through the energy); "
                     f"achieved counts the s(s+1)/2 = {pairs} slice-pair products of the 2(o^3 v^4 + o^4 v^3) "
                     f"flop that form W (padding to tiles not counted)")
    achieved = flops * pairs / head["wterm"] / 1e12
    if rank == 0:
        cfg = workload_config(name, args)
        cfg.update({"s_per_energy": head["sec"], "e_t": head["e_t"], "e_t5": head["e_t5"],
                    "prep_ms": 1e3 * head["prep"], "kernels_ms": 1e3 * head["kernel"],
                    "wterm_ms": 1e3 * head["wterm"], "input_generation_s": t_gen})
        if head_prec == tc.TC_FP64:
            dtype = "f64 (DMMA) throughout"
        else:
            dtype = (f"bf16x{head_slices} slices -> f32 tensor-core accumulation; epilogue (D, 1/D, quotients, "
                     f"sums over an item) in float pairs; per-triplet f64; compensated f64 total")
        out = {
            "metric": metric, "value": world * flops / head["sec"] / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * head["sec"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic (seeded DF factor and amplitudes, integrals formed on the device)",
            "config": cfg,
            "clocks": head["clocks"],
            "e2e": {"value": world * flops / te / 1e12, "unit": "TFLOP/s", "s_per_energy": te, "steps": e2e_steps,
                    "entry": "tc_energy (host arrays, pinned)", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": 8},
            "gpu_launches": head["launches"],
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak,
                         "traffic": recorded_traffic(kname, name, "fp64" if pairs == 1 else "split"),
                         "kernel": kname, "kernel_ms": 1e3 * head["wterm"], "peak_source": peak_note},
        }
        out["df"] = df_line
        if per_slices:
            out["slices"] = per_slices
        if sampled:
            out["sampled"] = sampled
            fp_s = sampled["fp64"]["s_per_energy_projected"]
            out["fp64"] = {"s_per_energy": fp_s, "projected": True, "value": flops / fp_s / 1e12, "unit": "TFLOP/s",
                           "how": "tc_triplets_dev kernel time on the sampled triplets x all triplets / sampled"}
            out["config"]["speedup_split_vs_fp64"] = fp_s / head["sec"]
        if fp64 is not None:
            fpeak = peak_bf16 * FP64_NOMINAL_TF / BF16_NOMINAL_TF
            fach = flops / fp64["kernel"] / 1e12
            out["fp64"] = {"value": world * flops / fp64["sec"] / 1e12, "unit": "TFLOP/s", "s_per_energy": fp64["sec"],
                           "steps": 1, "warmup": 1, "e_t": fp64["e_t"], "projected": False,
                           "roofline": {"bound": "tensor", "achieved": fach, "peak": fpeak, "frac": fach / fpeak,
                                        "kernel": "tc_fp64_kernel"}}
            out["config"]["abs_dE_split_vs_fp64"] = abs(head["e_t"] - fp64["e_t"])
            out["config"]["rel_dE_split_vs_fp64"] = abs(head["e_t"] - fp64["e_t"]) / abs(fp64["e_t"])
            out["config"]["speedup_split_vs_fp64"] = fp64["sec"] / head["sec"]
        if world == 1 and not args.no_cpu_baseline:
            _, hjob = host_job(name, amp)
            proj, used, info = oracle_sample(amp, hjob, args.cpu_baseline_seconds)
            out["cpu_baseline"] = {"value": flops / proj / 1e12, "unit": "TFLOP/s", "cores": round(used, 1),
                                   "cores_available": cores(), "kind": "oracle", "sample": info, "projected": True}
        print(json.dumps(out))
    tc.tc_finalize(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
