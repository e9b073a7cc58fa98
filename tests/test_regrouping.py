"""The split path's regrouping of Eq. 5 into three GEMMs per triplet, checked on the CPU.

For one occupied triplet (i, j, k):
    W_abc = F(i,j,k)[ab, c] + F(i,k,j)[ac, b] + F(j,k,i)[bc, a]
    F(p,q,r)[xy, z] =   sum_f G_pf^xy t_rq^zf + sum_f G_qf^yx t_rp^zf
                      - sum_l t_lp^yx G_rq^zl - sum_l t_lq^xy G_rp^zl
with G_pq^rs = (pr|qs).  Written here with plain einsums and compared with the
oracle's W (Eqs. 2 and 5), element by element, for every triplet of small jobs.
"""
import numpy as np
import pytest

import oracle
import synth


def f_term(job, p, q, r):
    """F(p,q,r)[x, y, z] for all virtual x, y, z."""
    G = job.ovvv                       # G_pf^xy = (p x | f y) = ovvv[p][x][f][y]
    t2 = job.t2
    H = job.ovoo                       # G_rq^zl = (r z | q l) = ovoo[r][z][q][l]
    part = (np.einsum("xfy,zf->xyz", G[p], t2[r, q])
            + np.einsum("yfx,zf->xyz", G[q], t2[r, p]))
    hole = (np.einsum("lyx,zl->xyz", t2[:, p], H[r, :, q, :])
            + np.einsum("lxy,zl->xyz", t2[:, q], H[r, :, p, :]))
    return part - hole


@pytest.mark.parametrize("o,v,seed", [(3, 5, 11), (4, 9, 12), (5, 7, 13)])
def test_three_gemm_regrouping_reproduces_w(o, v, seed):
    job = synth.make_job(o, v, seed)
    ref = np.empty((o, o, o, v, v, v))
    for a in range(v):
        for b in range(v):
            for c in range(v):
                ref[:, :, :, a, b, c] = oracle.w_ijk_all(job, a, b, c)
    for i in range(o):
        for j in range(i + 1):
            for k in range(j + 1):
                f0 = f_term(job, i, j, k)                       # [a, b, c]
                f1 = np.einsum("acb->abc", f_term(job, i, k, j))   # F(i,k,j)[ac, b]
                f2 = np.einsum("bca->abc", f_term(job, j, k, i))   # F(j,k,i)[bc, a]
                w = f0 + f1 + f2
                scale = np.max(np.abs(ref[i, j, k])) + 1e-300
                assert np.max(np.abs(w - ref[i, j, k])) <= 1e-13 * scale, (i, j, k)
