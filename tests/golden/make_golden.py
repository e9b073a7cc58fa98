"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py [workload ...]
    python tests/golden/make_golden.py --sampled [workload ...]

For each named synthetic workload it stores E_(T) (oracle.energy_by_triplets,
cross-checked against oracle.energy_eq1 when that is affordable) and the
weighted contribution of every occupied triplet i >= j >= k.

With --sampled (the full-size workloads, whose whole oracle energy would take
days on a host) it stores the weighted contributions of a fixed sample of
occupied triplets instead: edge cases (first and last orbitals, i = j, j = k)
and seeded random triplets, in sampled_<workload>.json.
"""
import json
import math
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def main(names):
    for name in names:
        t0 = time.time()
        job = synth.workload_job(name)
        trip = oracle.triplet_list(job.o)
        per = [oracle.triplet_energy(job, i, j, k) for (i, j, k) in trip]
        e = math.fsum(per)
        rec = {"workload": name, "o": job.o, "v": job.v, "seed": synth.WORKLOAD_SEEDS[name],
               "e_t": e, "triplets": [[i, j, k, x] for (i, j, k), x in zip(trip, per)],
               "source": "oracle.triplet_energy summed with math.fsum",
               "seconds": None}
        if job.o * job.v <= 300:
            rec["e_t_eq1"] = oracle.energy_eq1(job)
        rec["seconds"] = time.time() - t0
        with open(os.path.join(HERE, f"{name}.json"), "w") as f:
            json.dump(rec, f, indent=0)
        print(name, repr(e), f"{rec['seconds']:.1f}s", flush=True)


def sample_triplets(o, n_random=6, seed=777):
    """Edge-case triplets plus n_random seeded ones (distinct, i >= j >= k, not all equal)."""
    fixed = [(o - 1, o - 2, 0), (o // 2, o // 3, o // 5), (o - 1, o - 1, 1), (o // 2, 2, 2), (1, 0, 0),
             (o - 1, o // 2, o // 2 - 1)]
    allt = [t for t in oracle.triplet_list(o) if t[0] != t[2] and t not in fixed]
    u = synth.uniform(seed, 7, 0, 4 * n_random)
    picked = []
    for x in u:
        t = allt[int(x * len(allt))]
        if t not in picked:
            picked.append(t)
        if len(picked) == n_random:
            break
    return fixed + picked


def main_sampled(names):
    for name in names:
        t0 = time.time()
        o, v = synth.WORKLOADS[name]
        amp = synth.make_amplitudes(o, v, synth.WORKLOAD_SEEDS[name])
        job = synth.Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2, ovvv=None,
                        ovoo=synth.ovoo(amp), ovov=synth.ovov(amp))
        trip = sample_triplets(o)
        per = []
        for (i, j, k) in trip:
            sl = {x: synth.ovvv_slice(amp, x) for x in {i, j, k}}
            per.append(oracle.triplet_energy(job, i, j, k, ovvv_slices=sl))
            print(name, (i, j, k), repr(per[-1]), f"{time.time() - t0:.0f}s", flush=True)
        rec = {"workload": name, "o": o, "v": v, "seed": synth.WORKLOAD_SEEDS[name],
               "triplets": [[i, j, k, x] for (i, j, k), x in zip(trip, per)],
               "source": "oracle.triplet_energy on a fixed sample of occupied triplets (integral slices from synth)",
               "seconds": time.time() - t0}
        with open(os.path.join(HERE, f"sampled_{name}.json"), "w") as f:
            json.dump(rec, f, indent=0)


if __name__ == "__main__":
    args = sys.argv[1:]
    if args and args[0] == "--sampled":
        main_sampled(args[1:] or ["precision_o40_v400", "large_o50_v450"])
    else:
        main(args or ["tiny_o6_v36"])
