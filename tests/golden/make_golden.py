"""Writes the stored expected values under tests/golden/ from the CPU oracle only.

    python tests/golden/make_golden.py [workload ...]

For each named synthetic workload it stores E_(T) (oracle.energy_by_triplets,
cross-checked against oracle.energy_eq1 when that is affordable) and the
weighted contribution of every occupied triplet i >= j >= k.
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


if __name__ == "__main__":
    main(sys.argv[1:] or ["tiny_o6_v36"])
