"""CPU oracle for the closed-shell, canonical-orbital (T) correction.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, FP64 statement of
what the GPU library computes.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import it; the library never does.  It
shares no code with the CUDA path.

Everything follows the "Implementation Details" section of Fajen, Kelly,
Hohenstein, Martinez, "Accelerating CCSD(T) on GPUs" (arXiv 2512.01055):

* Eq. 1  -- the energy, a >= b >= c restricted, weight (2 - d_ab - d_bc);
* Eq. 2  -- W = P[ sum_f G_if^ab t_kj^cf - sum_l G_ij^al t_lk^bc ];
* Eq. 3  -- V = t_i^a G_jk^bc + t_j^b G_ik^ac + t_k^c G_ij^ab;
* Eq. 4 / Fig. 4 -- the denominator, taken with the Fig. 4 sign
  D = e_i + e_j + e_k - e_a - e_b - e_c (negative; see the readings below);
* Eq. 5  -- P sums the six simultaneous permutations of (ia)(jb)(kc).

G_pq^rs is read as the Mulliken integral (pr|qs), so with the input layouts

    ovvv[i, a, b, d] = (ia|bd),  ovoo[i, a, j, l] = (ia|jl),  ovov[i, a, j, b] = (ia|jb)

the integrals of Eqs. 2-3 are G_if^ab = (ia|fb) = ovvv[i, a, f, b],
G_ij^al = (ia|jl) = ovoo[i, a, j, l], G_jk^bc = (jb|kc) = ovov[j, b, k, c],
G_ik^ac = (ia|kc), G_ij^ab = (ia|jb).

Two forms are provided:

* ``energy_eq1`` -- Eq. 1 as printed: loop a >= b >= c, W and V over all
  (i, j, k) for that (a, b, c);
* ``triplet_energy`` / ``energy_by_triplets`` -- the same sum regrouped by
  occupied triplets i >= j >= k with weight (2 - d_ij - d_jk) and a sum over
  all (a, b, c); the permutations of W's occupied indices in Eq. 1 become
  permutations of its virtual indices at fixed (i, j, k) (W is invariant under
  simultaneous permutations, Eq. 5).  This is the grouping the GPU library
  uses, so it is what sampled checks at full size compare per triplet.

Totals are summed with ``math.fsum`` (exactly rounded).
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["x_bracket_ijk", "w_ijk_all", "v_ijk_all", "d_ijk_all", "energy_eq1", "energy_parts_eq1",
           "w_abc_all", "triplet_energy", "energy_by_triplets", "triplet_weight"]


def _ev(job, a):
    return job.eps[job.o + a]


# ---------------------------------------------------------------------------
# Eq. 1 as printed: a >= b >= c outside, arrays over (i, j, k) inside.
# ---------------------------------------------------------------------------

def x_bracket_ijk(job, p: int, q: int, r: int) -> np.ndarray:
    """Bracket of Eq. 2 before P, X(xyz, pqr), for all occupied (x, y, z) at fixed (p, q, r).

    X(xyz, pqr) = sum_f G_xf^pq t_zy^rf - sum_l G_xy^pl t_lz^qr
    returned as an array indexed [x, y, z].
    """
    part = np.einsum("xf,zyf->xyz", job.ovvv[:, p, :, q], job.t2[:, :, r, :])   # G_xf^pq = (xp|fq)
    hole = np.einsum("xyl,lz->xyz", job.ovoo[:, p, :, :], job.t2[:, :, q, r])    # G_xy^pl = (xp|yl)
    return part - hole


def w_ijk_all(job, a: int, b: int, c: int) -> np.ndarray:
    """W_ijk^abc (Eqs. 2 and 5) for all (i, j, k) at fixed (a, b, c)."""
    W = x_bracket_ijk(job, a, b, c)                                   # X(ijk, abc)
    W = W + np.einsum("ikj->ijk", x_bracket_ijk(job, a, c, b))        # X(ikj, acb)
    W = W + np.einsum("jik->ijk", x_bracket_ijk(job, b, a, c))        # X(jik, bac)
    W = W + np.einsum("jki->ijk", x_bracket_ijk(job, b, c, a))        # X(jki, bca)
    W = W + np.einsum("kji->ijk", x_bracket_ijk(job, c, b, a))        # X(kji, cba)
    W = W + np.einsum("kij->ijk", x_bracket_ijk(job, c, a, b))        # X(kij, cab)
    return W


def v_ijk_all(job, a: int, b: int, c: int) -> np.ndarray:
    """V_ijk^abc (Eq. 3) for all (i, j, k) at fixed (a, b, c)."""
    t1, g = job.t1, job.ovov
    return (np.einsum("i,jk->ijk", t1[:, a], g[:, b, :, c])      # t_i^a (jb|kc)
            + np.einsum("j,ik->ijk", t1[:, b], g[:, a, :, c])    # t_j^b (ia|kc)
            + np.einsum("k,ij->ijk", t1[:, c], g[:, a, :, b]))   # t_k^c (ia|jb)


def d_ijk_all(job, a: int, b: int, c: int) -> np.ndarray:
    """D_ijk^abc = e_i + e_j + e_k - (e_a + e_b + e_c)   (Fig. 4 sign)."""
    eo = job.eps[:job.o]
    return (eo[:, None, None] + eo[None, :, None] + eo[None, None, :]) - (_ev(job, a) + _ev(job, b) + _ev(job, c))


def abc_contribution(job, a: int, b: int, c: int) -> float:
    """sum_ijk (W + V)(4W_ijk + W_jki + W_kij - 2W_jik - 2W_ikj - 2W_kji)/D at one (a, b, c)."""
    W = w_ijk_all(job, a, b, c)
    V = v_ijk_all(job, a, b, c)
    D = d_ijk_all(job, a, b, c)
    bracket = (4.0 * W + np.einsum("jki->ijk", W) + np.einsum("kij->ijk", W)
               - 2.0 * np.einsum("jik->ijk", W) - 2.0 * np.einsum("ikj->ijk", W)
               - 2.0 * np.einsum("kji->ijk", W))
    return float(np.sum((W + V) * bracket / D))


def abc_contribution_parts(job, a: int, b: int, c: int) -> tuple:
    """The two parts of abc_contribution: (sum_ijk W r3(W)/D, sum_ijk V r3(W)/D),
    r3(W) = 4W_ijk + W_jki + W_kij - 2W_jik - 2W_ikj - 2W_kji (the bracket of Eq. 1)."""
    W = w_ijk_all(job, a, b, c)
    V = v_ijk_all(job, a, b, c)
    D = d_ijk_all(job, a, b, c)
    bracket = (4.0 * W + np.einsum("jki->ijk", W) + np.einsum("kij->ijk", W)
               - 2.0 * np.einsum("jik->ijk", W) - 2.0 * np.einsum("ikj->ijk", W)
               - 2.0 * np.einsum("kji->ijk", W))
    return float(np.sum(W * bracket / D)), float(np.sum(V * bracket / D))


def energy_parts_eq1(job) -> tuple:
    """(E[4], E[5]_ST): Eq. 1 with its factor (W + V) split into the W part and
    the V part, same a >= b >= c weights; E_(T) = E[4] + E[5]_ST."""
    t4, t5 = [], []
    for a in range(job.v):
        for b in range(a + 1):
            for c in range(b + 1):
                wgt = 2 - (a == b) - (b == c)
                if wgt == 0:
                    continue
                e4, e5 = abc_contribution_parts(job, a, b, c)
                t4.append(wgt * e4)
                t5.append(wgt * e5)
    return math.fsum(t4), math.fsum(t5)


def energy_eq1(job) -> float:
    """E_(T) of Eq. 1, literally: a >= b >= c with weight (2 - d_ab - d_bc)."""
    terms = []
    for a in range(job.v):
        for b in range(a + 1):
            for c in range(b + 1):
                wgt = 2 - (a == b) - (b == c)
                if wgt == 0:
                    continue
                terms.append(wgt * abc_contribution(job, a, b, c))
    return math.fsum(terms)


# ---------------------------------------------------------------------------
# The same energy grouped by occupied triplets i >= j >= k.
# ---------------------------------------------------------------------------

def x_bracket_abc(job, x: int, y: int, z: int, ovvv_x=None) -> np.ndarray:
    """X(xyz, abc) of Eq. 2 (before P) for all (a, b, c) at fixed occupied (x, y, z).

    X(xyz, abc) = sum_f (xa|fb) t_zy^cf - sum_l (xa|yl) t_lz^bc,  indexed [a, b, c].
    ``ovvv_x`` may supply ovvv[x] when the full ovvv is not held in memory.
    """
    Gx = job.ovvv[x] if ovvv_x is None else ovvv_x                    # [a, f, b] = (xa|fb)
    part = np.einsum("afb,cf->abc", Gx, job.t2[z, y], optimize=True)
    hole = np.einsum("al,lbc->abc", job.ovoo[x, :, y, :], job.t2[:, z], optimize=True)
    return part - hole


def w_abc_all(job, i: int, j: int, k: int, ovvv_slices=None) -> np.ndarray:
    """W_ijk^abc (Eqs. 2 and 5) for all (a, b, c) at fixed (i, j, k), indexed [a, b, c]."""
    sl = (lambda x: None) if ovvv_slices is None else (lambda x: ovvv_slices[x])
    W = x_bracket_abc(job, i, j, k, sl(i))                                   # X(ijk, abc)
    W += np.einsum("acb->abc", x_bracket_abc(job, i, k, j, sl(i)))           # X(ikj, acb)
    W += np.einsum("bac->abc", x_bracket_abc(job, j, i, k, sl(j)))           # X(jik, bac)
    W += np.einsum("bca->abc", x_bracket_abc(job, j, k, i, sl(j)))           # X(jki, bca)
    W += np.einsum("cba->abc", x_bracket_abc(job, k, j, i, sl(k)))           # X(kji, cba)
    W += np.einsum("cab->abc", x_bracket_abc(job, k, i, j, sl(k)))           # X(kij, cab)
    return W


def v_abc_all(job, i: int, j: int, k: int) -> np.ndarray:
    """V_ijk^abc (Eq. 3) for all (a, b, c) at fixed (i, j, k)."""
    t1, g = job.t1, job.ovov
    return (np.einsum("a,bc->abc", t1[i], g[j, :, k, :])      # t_i^a (jb|kc)
            + np.einsum("b,ac->abc", t1[j], g[i, :, k, :])    # t_j^b (ia|kc)
            + np.einsum("c,ab->abc", t1[k], g[i, :, j, :]))   # t_k^c (ia|jb)


def d_abc_all(job, i: int, j: int, k: int) -> np.ndarray:
    ev = job.eps[job.o:]
    eijk = job.eps[i] + job.eps[j] + job.eps[k]
    return eijk - (ev[:, None, None] + ev[None, :, None] + ev[None, None, :])


def triplet_weight(i: int, j: int, k: int) -> int:
    """Weight of an ordered triplet i >= j >= k: 2 if distinct, 1 if two equal, 0 if all equal."""
    assert i >= j >= k
    return 2 - (i == j) - (j == k)


def triplet_sum(job, i: int, j: int, k: int, ovvv_slices=None) -> float:
    """sum over all (a, b, c) of (W + V) r3(W) / D at fixed (i, j, k), no weight.

    The occupied permutations of Eq. 1's bracket act at fixed (a, b, c); by the
    simultaneous-permutation symmetry of W they equal virtual permutations at
    fixed (i, j, k): W_jki^abc = W_ijk^cab, W_kij^abc = W_ijk^bca,
    W_jik^abc = W_ijk^bac, W_ikj^abc = W_ijk^acb, W_kji^abc = W_ijk^cba.
    """
    W = w_abc_all(job, i, j, k, ovvv_slices)
    V = v_abc_all(job, i, j, k)
    D = d_abc_all(job, i, j, k)
    Y = (4.0 * W + np.einsum("cab->abc", W) + np.einsum("bca->abc", W)
         - 2.0 * np.einsum("bac->abc", W) - 2.0 * np.einsum("acb->abc", W)
         - 2.0 * np.einsum("cba->abc", W))
    return float(np.sum((W + V) * Y / D))


def triplet_energy(job, i: int, j: int, k: int, ovvv_slices=None) -> float:
    """Weighted contribution of the occupied triplet i >= j >= k to E_(T).

    E_(T) = sum_{i>=j>=k} triplet_energy(i, j, k).  Equivalent to Eq. 1 because
    Eq. 1 equals one third of the unrestricted sum over all (i,j,k,a,b,c), and
    an unordered triplet with 3 distinct / 2 equal / 3 equal members has
    6 / 3 / 1 orderings (weights 2 / 1 / 0; the last sum vanishes: r3 annihilates
    a tensor symmetric in its three occupied indices).
    """
    w = triplet_weight(i, j, k)
    if w == 0:
        return 0.0
    return w * triplet_sum(job, i, j, k, ovvv_slices)


def energy_by_triplets(job) -> float:
    terms = [triplet_energy(job, i, j, k)
             for i in range(job.o) for j in range(i + 1) for k in range(j + 1)]
    return math.fsum(terms)


def triplet_list(o: int):
    """All i >= j >= k, in the order (i, j, k) lexicographic -- the library's triplet order."""
    return [(i, j, k) for i in range(o) for j in range(i + 1) for k in range(j + 1)]


def algorithmic_flops(o: int, v: int) -> float:
    """2 (o^3 v^4 + o^4 v^3): the particle and hole contractions of Eq. 2."""
    return 2.0 * (float(o) ** 3 * float(v) ** 4 + float(o) ** 4 * float(v) ** 3)
