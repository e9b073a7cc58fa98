"""Independent checks for the oracle (test-side only).

* ``brute_force_energy`` -- Eq. 1 with every tensor element formed by scalar
  loops (no array reshuffling), evaluated as one third of the unrestricted sum
  over all (i, j, k, a, b, c).  It pins the vectorised index bookkeeping of the
  oracle and the a >= b >= c weights of Eq. 1.

* ``spin_orbital_energy`` -- the textbook spin-orbital (T) expression
  (e.g. Crawford and Schaefer, Rev. Comput. Chem. 14, 33 (2000)):

      D t_ijk^abc(c) = P(i/jk) P(a/bc) [ sum_e t_jk^ae <ei||bc> - sum_m t_im^bc <ma||jk> ]
      D t_ijk^abc(d) = P(i/jk) P(a/bc) t_i^a <jk||bc>
      E_(T) = 1/36 sum t(c) D (t(c) + t(d)),    P(i/jk) f = f(ijk) - f(jik) - f(kji)

  built from the spatial density-fitting factor directly (not from the
  oracle's integral blocks) with the closed-shell spin adaptation
  t_{I J}^{A B} = t_ij^ab d(sI,sA) d(sJ,sB) - t_ij^ba d(sI,sB) d(sJ,sA).
  A different formula reaching the same number pins normalisation, signs and
  the pairing of integrals with amplitudes in the closed-shell Eq. 1.
"""
import math

import numpy as np


def brute_force_energy(job) -> float:
    o, v = job.o, job.v
    ovvv, ovoo, ovov, t1, t2, eps = job.ovvv, job.ovoo, job.ovov, job.t1, job.t2, job.eps

    def bracket(x, y, z, p, q, r):
        s = 0.0
        for f in range(v):
            s += ovvv[x, p, f, q] * t2[z, y, r, f]
        for l in range(o):
            s -= ovoo[x, p, y, l] * t2[l, z, q, r]
        return s

    Wt = np.zeros((o, o, o, v, v, v))
    for i in range(o):
        for j in range(o):
            for k in range(o):
                for a in range(v):
                    for b in range(v):
                        for c in range(v):
                            Wt[i, j, k, a, b, c] = (bracket(i, j, k, a, b, c) + bracket(i, k, j, a, c, b)
                                                    + bracket(j, i, k, b, a, c) + bracket(j, k, i, b, c, a)
                                                    + bracket(k, j, i, c, b, a) + bracket(k, i, j, c, a, b))
    terms = []
    for i in range(o):
        for j in range(o):
            for k in range(o):
                for a in range(v):
                    for b in range(v):
                        for c in range(v):
                            W = Wt[i, j, k, a, b, c]
                            V = (t1[i, a] * ovov[j, b, k, c] + t1[j, b] * ovov[i, a, k, c]
                                 + t1[k, c] * ovov[i, a, j, b])
                            D = eps[i] + eps[j] + eps[k] - eps[o + a] - eps[o + b] - eps[o + c]
                            r = (4 * W + Wt[j, k, i, a, b, c] + Wt[k, i, j, a, b, c]
                                 - 2 * Wt[j, i, k, a, b, c] - 2 * Wt[i, k, j, a, b, c] - 2 * Wt[k, j, i, a, b, c])
                            terms.append((W + V) * r / D)
    return math.fsum(terms) / 3.0


def spin_orbital_energy(amp) -> float:
    o, v = amp.o, amp.v
    N = o + v
    eri = np.einsum("Qpq,Qrs->pqrs", amp.B, amp.B)            # (pq|rs), spatial
    spat = np.array([I // 2 for I in range(2 * o)] + [o + A // 2 for A in range(2 * v)])
    spin = np.array([I % 2 for I in range(2 * o)] + [A % 2 for A in range(2 * v)])
    same = (spin[:, None] == spin[None, :]).astype(float)
    chem = eri[np.ix_(spat, spat, spat, spat)] * same[:, :, None, None] * same[None, None, :, :]
    phys = chem.transpose(0, 2, 1, 3)                          # <PQ|RS> = (PR|QS)
    g = phys - phys.transpose(0, 1, 3, 2)                      # <PQ||RS>
    O = slice(0, 2 * o)
    Vs = slice(2 * o, 2 * N)
    so, sv = spin[O], spin[Vs]
    io, av = spat[O], spat[Vs] - o
    t1 = amp.t1[np.ix_(io, av)] * (so[:, None] == sv[None, :])
    t2sp = amp.t2[np.ix_(io, io, av, av)]
    d = lambda x, y: (x[:, None] == y[None, :]).astype(float)
    t2 = (t2sp * d(so, sv)[:, None, :, None] * d(so, sv)[None, :, None, :]
          - amp.t2[np.ix_(io, io, av, av)].transpose(0, 1, 3, 2) * d(so, sv)[:, None, None, :] * d(so, sv)[None, :, :, None])
    eps = amp.eps[spat]
    eo, ev = eps[O], eps[Vs]

    def Pocc(X):
        return X - np.einsum("jikabc->ijkabc", X) - np.einsum("kjiabc->ijkabc", X)

    def Pvir(X):
        return X - np.einsum("ijkbac->ijkabc", X) - np.einsum("ijkcba->ijkabc", X)

    conn = (np.einsum("jkae,eibc->ijkabc", t2, g[Vs, O, Vs, Vs])
            - np.einsum("imbc,majk->ijkabc", t2, g[O, Vs, O, O]))
    conn = Pocc(Pvir(conn))
    disc = Pocc(Pvir(np.einsum("ia,jkbc->ijkabc", t1, g[O, O, Vs, Vs])))
    D = (eo[:, None, None, None, None, None] + eo[None, :, None, None, None, None]
         + eo[None, None, :, None, None, None] - ev[None, None, None, :, None, None]
         - ev[None, None, None, None, :, None] - ev[None, None, None, None, None, :])
    return float(np.sum(conn * (conn + disc) / D) / 36.0)
