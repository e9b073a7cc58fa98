"""Helpers shared by the GPU tests: build the library once, move jobs to the device."""
import functools

import numpy as np

import paper_2512_01055_gb300 as tc
from paper_2512_01055_gb300 import build


@functools.lru_cache(maxsize=1)
def context():
    build.build()
    return tc.tc_init(0)


def to_device(job):
    import torch
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    return dict(eps=f(job.eps), t1=f(job.t1), t2=f(job.t2), ovvv=f(job.ovvv), ovoo=f(job.ovoo), ovov=f(job.ovov))


def energy_dev(job, prec=tc.TC_FP64, slices=0, want_trip=False, dev=None):
    import torch
    dev = dev or to_device(job)
    e_ijk = torch.zeros((job.o,) * 3, dtype=torch.float64, device="cuda") if want_trip else None
    r = tc.tc_energy_dev(context(), job.o, job.v, dev["eps"], dev["t1"], dev["t2"], dev["ovvv"], dev["ovoo"],
                         dev["ovov"], prec=prec, slices=slices, e_ijk=e_ijk)
    return r, (e_ijk.cpu().numpy() if want_trip else None)


def energy_host(job, prec=tc.TC_FP64, slices=0, want_trip=False):
    e_ijk = np.zeros((job.o,) * 3) if want_trip else None
    r = tc.tc_energy(context(), job.o, job.v, job.eps, job.t1, job.t2, job.ovvv, job.ovoo, job.ovov,
                     prec=prec, slices=slices, e_ijk=e_ijk)
    return r, e_ijk
