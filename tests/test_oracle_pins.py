"""Pins of the CPU oracle against things other than itself (no GPU needed)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synth
from tests import pins


def small_job(o, v, seed, **scale):
    amp = synth.make_amplitudes(o, v, seed)
    job = synth.Job(o=o, v=v, eps=amp.eps, t1=amp.t1, t2=amp.t2,
                    ovvv=synth.ovvv(amp), ovoo=synth.ovoo(amp), ovov=synth.ovov(amp))
    return amp, job


def scaled(job, lam=1.0, mu=1.0, mu1=None, eps_shift=0.0, eps_scale=1.0):
    mu1 = mu if mu1 is None else mu1
    return dataclasses.replace(job, ovvv=job.ovvv * lam, ovoo=job.ovoo * lam, ovov=job.ovov * lam,
                               t1=job.t1 * mu1, t2=job.t2 * mu,
                               eps=(job.eps + eps_shift) * eps_scale)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 11), (3, 2, 12), (2, 4, 13), (3, 3, 14)])
def test_spin_orbital_textbook_formula(o, v, seed):
    """Closed-shell Eq. 1 equals the spin-orbital (T) of the CC literature."""
    amp, job = small_job(o, v, seed)
    e_cs = oracle.energy_eq1(job)
    e_so = pins.spin_orbital_energy(amp)
    assert abs(e_cs - e_so) <= 1e-12 * abs(e_so), (e_cs, e_so)
    # and with t1 = 0 (the E[4] part alone)
    amp0 = dataclasses.replace(amp, t1=np.zeros_like(amp.t1))
    job0 = dataclasses.replace(job, t1=np.zeros_like(job.t1))
    e0 = oracle.energy_eq1(job0)
    assert abs(e0 - pins.spin_orbital_energy(amp0)) <= 1e-12 * abs(e0)


@pytest.mark.parametrize("o,v,seed", [(2, 3, 21), (3, 2, 22), (3, 4, 23)])
def test_brute_force_unrestricted_sum(o, v, seed):
    """(1/3) sum over all (ijk, abc) with scalar loops equals the a>=b>=c form of Eq. 1."""
    _, job = small_job(o, v, seed)
    eb = pins.brute_force_energy(job)
    e1 = oracle.energy_eq1(job)
    assert abs(eb - e1) <= 1e-13 * abs(eb)


@pytest.mark.parametrize("o,v,seed", [(3, 4, 31), (4, 5, 32), (5, 3, 33), (6, 7, 34)])
def test_triplet_grouping_equals_eq1(o, v, seed):
    """The i>=j>=k grouping (the library's schedule) equals Eq. 1 as printed."""
    _, job = small_job(o, v, seed)
    e1 = oracle.energy_eq1(job)
    et = oracle.energy_by_triplets(job)
    assert abs(e1 - et) <= 1e-13 * abs(e1)


def test_w_permutational_symmetry():
    """W_ijk^abc = W_{s(ijk)}^{s(abc)} for the six simultaneous permutations (Eq. 5)."""
    _, job = small_job(4, 5, 41)
    perms = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]
    for (i, j, k) in [(3, 1, 0), (2, 2, 1), (3, 0, 2)]:
        W = oracle.w_abc_all(job, i, j, k)
        occ = (i, j, k)
        for s in perms:
            Ws = oracle.w_abc_all(job, occ[s[0]], occ[s[1]], occ[s[2]])
            # W_{s(ijk)}^{s(abc)}: virtual axes permuted the same way
            np.testing.assert_allclose(np.transpose(W, s), Ws, rtol=1e-13, atol=1e-15)
    # and the (a,b,c)-outer accessor agrees with the (i,j,k)-outer one
    Wa = oracle.w_ijk_all(job, 3, 1, 2)
    for (i, j, k) in [(3, 1, 0), (0, 2, 1)]:
        assert abs(Wa[i, j, k] - oracle.w_abc_all(job, i, j, k)[3, 1, 2]) <= 1e-13 * max(1e-30, abs(Wa[i, j, k]))


def test_zero_amplitudes_give_zero():
    _, job = small_job(3, 4, 51)
    z = scaled(job, mu=0.0)
    assert oracle.energy_eq1(z) == 0.0
    assert oracle.energy_by_triplets(z) == 0.0


@pytest.mark.parametrize("o,v", [(1, 5), (4, 1), (1, 1)])
def test_single_occupied_or_virtual_gives_zero(o, v):
    """With o = 1 (or v = 1) only totally symmetric W survive, which r3 annihilates."""
    _, job = small_job(o, v, 61)
    e = oracle.energy_eq1(job)
    scale = sum(abs(oracle.abc_contribution(job, a, b, c)) for a in range(v) for b in range(v) for c in range(v)) + 1.0
    assert abs(e) <= 1e-14 * scale


def test_power_of_two_scaling_is_exact():
    """E(lam G, mu t1, mu t2) = lam^2 mu^2 E; powers of two make it bit-exact."""
    _, job = small_job(3, 4, 71)
    e = oracle.energy_eq1(job)
    for lam, mu in [(2.0, 0.5), (4.0, 2.0), (0.25, 8.0)]:
        assert oracle.energy_eq1(scaled(job, lam=lam, mu=mu)) == lam ** 2 * mu ** 2 * e
    j0 = scaled(job, mu1=0.0)
    e0 = oracle.energy_eq1(j0)
    assert oracle.energy_by_triplets(scaled(j0, lam=2.0, mu=4.0, mu1=0.0)) == 64.0 * oracle.energy_by_triplets(j0)
    assert e0 != 0.0


def test_orbital_energy_shift_and_scale():
    _, job = small_job(3, 4, 81)
    e = oracle.energy_eq1(job)
    es = oracle.energy_eq1(scaled(job, eps_shift=0.37))
    assert abs(es - e) <= 1e-12 * abs(e)
    assert oracle.energy_eq1(scaled(job, eps_scale=2.0)) == e / 2.0


def test_linear_in_t1():
    """V is linear in t1 and W does not depend on it: E(t1) + E(-t1) = 2 E(0)."""
    _, job = small_job(3, 5, 91)
    ep = oracle.energy_eq1(job)
    em = oracle.energy_eq1(dataclasses.replace(job, t1=-job.t1))
    e0 = oracle.energy_eq1(dataclasses.replace(job, t1=np.zeros_like(job.t1)))
    assert abs(ep + em - 2 * e0) <= 1e-12 * abs(e0)
    assert ep != e0


@pytest.mark.parametrize("seed", [101, 102, 103])
def test_connected_part_is_stabilising(seed):
    """With t1 = 0 and D < 0, E_(T) <= 0 (r3 is positive semidefinite)."""
    _, job = small_job(3, 4, seed)
    j0 = dataclasses.replace(job, t1=np.zeros_like(job.t1))
    assert oracle.energy_eq1(j0) < 0.0
    for (i, j, k) in oracle.triplet_list(3):
        assert oracle.triplet_energy(j0, i, j, k) <= 1e-18


def test_equal_triplet_sum_vanishes():
    _, job = small_job(3, 4, 111)
    s = oracle.triplet_sum(job, 1, 1, 1)
    ref = abs(oracle.triplet_sum(job, 2, 1, 0))
    assert abs(s) <= 1e-14 * ref


def test_planted_mistakes_are_caught():
    """A plausible slip in Eq. 1's bracket or Eq. 3 is visible to the spin-orbital pin."""
    amp, job = small_job(2, 3, 121)
    e_so = pins.spin_orbital_energy(amp)
    orig = oracle.abc_contribution

    def wrong_bracket(job, a, b, c):   # sign of one permuted term flipped
        W = oracle.w_ijk_all(job, a, b, c)
        V = oracle.v_ijk_all(job, a, b, c)
        D = oracle.d_ijk_all(job, a, b, c)
        br = (4.0 * W + np.einsum("jki->ijk", W) - np.einsum("kij->ijk", W)
              - 2.0 * np.einsum("jik->ijk", W) - 2.0 * np.einsum("ikj->ijk", W)
              - 2.0 * np.einsum("kji->ijk", W))
        return float(np.sum((W + V) * br / D))

    def wrong_v(job, a, b, c):         # V with (ia|jb) -> (ib|ja)
        W = oracle.w_ijk_all(job, a, b, c)
        t1, g = job.t1, job.ovov
        V = (np.einsum("i,jk->ijk", t1[:, a], g[:, b, :, c]) + np.einsum("j,ik->ijk", t1[:, b], g[:, a, :, c])
             + np.einsum("k,ij->ijk", t1[:, c], g[:, b, :, a]))
        D = oracle.d_ijk_all(job, a, b, c)
        br = (4.0 * W + np.einsum("jki->ijk", W) + np.einsum("kij->ijk", W)
              - 2.0 * np.einsum("jik->ijk", W) - 2.0 * np.einsum("ikj->ijk", W) - 2.0 * np.einsum("kji->ijk", W))
        return float(np.sum((W + V) * br / D))

    try:
        for bad in (wrong_bracket, wrong_v):
            oracle.abc_contribution = bad
            e_bad = oracle.energy_eq1(job)
            assert abs(e_bad - e_so) > 1e-8 * abs(e_so)
    finally:
        oracle.abc_contribution = orig
    assert abs(oracle.energy_eq1(job) - e_so) <= 1e-12 * abs(e_so)


# ---------------------------------------------------------------------------
# E[4] and E[5]_ST: the W part and the V part of Eq. 1's factor (W + V).
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("o,v,seed", [(3, 5, 21), (4, 6, 22)])
def test_energy_parts_add_up(o, v, seed):
    job = synth.make_job(o, v, seed)
    e4, e5 = oracle.energy_parts_eq1(job)
    e = oracle.energy_eq1(job)
    assert abs((e4 + e5) - e) <= 1e-12 * (abs(e4) + abs(e5))


def test_e5_structure_in_t1():
    """V is linear in t1 and W does not depend on t1: E[5]_ST vanishes without t1
    and is odd in t1, E[4] is the same for t1, -t1 and 0 (all exactly)."""
    job = synth.make_job(4, 6, 23)
    e4, e5 = oracle.energy_parts_eq1(job)
    e4m, e5m = oracle.energy_parts_eq1(dataclasses.replace(job, t1=-job.t1))
    e40, e50 = oracle.energy_parts_eq1(dataclasses.replace(job, t1=np.zeros_like(job.t1)))
    assert e50 == 0.0
    assert e5m == -e5 and e5 != 0.0
    assert e4m == e4 == e40
