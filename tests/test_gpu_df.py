"""Integrals assembled on the device from density-fitting factors (Eq. 6).

tc_energy_df_dev takes B[Q][p][q] with (pq|rs) = sum_Q B[Q][p][q] B[Q][r][s]
and forms (ia|bd), (ia|jl), (ia|jb) itself, as exact base-256 digit products
on the tensor cores.  The synthetic factors sit on a 2^-20 grid, so every
integral is an exact sum in any order: the assembled integrals equal the
host-built ones bit for bit, and so must the energies and the per-triplet
contributions of both precisions.  The energies are also checked against the
oracle.  Factors off the grid (general FP64 values) take seven digits and
must agree with FP64 integrals to FP64 accuracy.
"""
import ctypes

import numpy as np
import pytest

import oracle
import synth
import paper_2512_01055_gb300 as tc
from tests import gpu_util
from tests.split_bounds import split_rel_bound

pytestmark = pytest.mark.gpu
FP64, SPLIT = tc.TC_FP64, tc.TC_SPLIT_BF16


def _run(amp, prec, s):
    import torch
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    o, v = amp.o, amp.v
    job = synth.Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2,
                    ovvv=synth.ovvv(amp), ovoo=synth.ovoo(amp), ovov=synth.ovov(amp))
    r_int, e_int = gpu_util.energy_dev(job, prec=prec, slices=s, want_trip=True)
    e_df = torch.zeros((o,) * 3, dtype=torch.float64, device="cuda")
    r_df = tc.tc_energy_df_dev(gpu_util.context(), o, v, f(amp.B), f(amp.eps), f(amp.t1), f(amp.t2),
                               prec=prec, slices=s, e_ijk=e_df)
    return job, r_int, e_int, r_df, e_df.cpu().numpy()


@pytest.mark.parametrize("o,v,seed,prec,s", [(4, 17, 41, FP64, 0), (5, 33, 42, SPLIT, 3), (3, 20, 43, SPLIT, 2),
                                             (6, 36, 44, FP64, 0), (6, 36, 44, SPLIT, 3)])
def test_df_input_equals_integral_input(o, v, seed, prec, s):
    amp = synth.make_amplitudes(o, v, seed)
    job, r_int, e_int, r_df, e_df = _run(amp, prec, s)
    print(f"o={o} v={v} prec={prec} s={s} E_df={r_df.e_t:.15e} E_int={r_int.e_t:.15e} df {r_df.df_seconds:.2e} s")
    assert r_df.e_t == r_int.e_t and r_df.e_t5 == r_int.e_t5
    assert np.array_equal(e_df, e_int)
    assert r_df.df_seconds > 0.0 and r_df.prec == prec
    assert 1 <= r_df.df_digits <= 3                 # factors on the 2^-20 grid: exact in three digits
    ref = oracle.energy_by_triplets(job)
    tol = 1e-9 * abs(ref) if prec == FP64 else split_rel_bound(s, o, v) * max(1.0, abs(ref))
    assert abs(r_df.e_t - ref) <= tol


@pytest.mark.parametrize("prec,s", [(FP64, 0), (SPLIT, 3)])
def test_df_general_factors_agree_to_fp64_accuracy(prec, s):
    """Factors with full 53-bit values: seven digits, energies as from FP64-rounded integrals."""
    import dataclasses
    amp = synth.make_amplitudes(5, 30, 47)
    rng = np.random.default_rng(11)
    noise = rng.standard_normal(amp.B.shape) * 1e-3
    B = amp.B + (noise + noise.transpose(0, 2, 1)) * 0.5          # symmetric, off the grid
    amp = dataclasses.replace(amp, B=B)
    job, r_int, e_int, r_df, e_df = _run(amp, prec, s)
    print(f"prec={prec} digits={r_df.df_digits} E_df={r_df.e_t:.15e} E_int={r_int.e_t:.15e}")
    assert r_df.df_digits == 7
    assert abs(r_df.e_t - r_int.e_t) <= 1e-12 * abs(r_int.e_t)
    assert np.all(np.abs(e_df - e_int) <= 1e-12 * np.abs(e_int).max())


def test_df_full_size_o20_v200():
    """The o=20, v=200 workload through the DF entry point: the same energy as from the integral arrays."""
    amp = synth.make_amplitudes(20, 200, synth.WORKLOAD_SEEDS["single_o20_v200"])
    _, r_int, e_int, r_df, e_df = _run(amp, SPLIT, 3)
    print(f"E_df={r_df.e_t:.12e} df assembly {r_df.df_seconds * 1e3:.2f} ms, energy kernels "
          f"{r_df.kernel_seconds * 1e3:.1f} ms")
    assert r_df.e_t == r_int.e_t
    assert np.array_equal(e_df, e_int)


@pytest.mark.parametrize("prec,s", [(FP64, 0), (SPLIT, 3)])
def test_df_host_entry_equals_device_entry(prec, s):
    """tc_energy_df (host arrays) gives the same bits as tc_energy_df_dev."""
    amp = synth.make_amplitudes(5, 28, 46)
    _, r_int, e_int, r_df, e_df = _run(amp, prec, s)
    e_h = np.zeros((5, 5, 5))
    r_h = tc.tc_energy_df(gpu_util.context(), 5, 28, np.ascontiguousarray(amp.B), amp.eps, amp.t1, amp.t2,
                          prec=prec, slices=s, e_ijk=e_h)
    assert r_h.e_t == r_df.e_t == r_int.e_t
    assert np.array_equal(e_h, e_df) and r_h.df_seconds > 0.0


def test_df_rejects_bad_arguments():
    import torch
    amp = synth.make_amplitudes(3, 8, 45)
    f = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to("cuda")
    lib = tc.load()
    res = tc.tc_result()
    ctx = gpu_util.context()
    eps, t1, t2, B = f(amp.eps), f(amp.t1), f(amp.t2), f(amp.B)
    for nq, bp in ((0, B.data_ptr()), (amp.Q, None)):
        s = lib.tc_energy_df_dev(ctx, 3, 8, nq, eps.data_ptr(), t1.data_ptr(), t2.data_ptr(), bp, FP64, 0, None,
                                 None, ctypes.byref(res))
        assert s == tc.TC_EINVAL
