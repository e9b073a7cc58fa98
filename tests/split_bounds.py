"""Error bounds of the split-precision path used by the parity tests.

s BF16 slices keep the slice-pair products p + q < s of each operand product.
For s >= 3 the dropped pairs are 2^-24 of the product or smaller, below the
FP32 accumulation error, and the bound is the stated 1e-6 relative
(|dE| <= 1e-6 max(1 Eh, |E_T|); literally 1e-6 Eh on the physical-scale twins).

For s = 2 the dropped pairs (x1 y1, x0 y2, x2 y0) are about 2^-16 of each
product, with random signs.  W sums K = 2v + 2o of them and E_T sums many
points, so the relative error of E_T falls as v grows: on the tiny
workloads (v < 64) it is bounded by S2_SMALL, from v = 64 on by 1e-6 like
s >= 3 (measured: within 2.4e-9 of s = 3 at o=20 v=200).
"""

S2_SMALL = 1e-4


def split_rel_bound(s, o, v):
    if s >= 3:
        return 1e-6
    return S2_SMALL if v < 64 else 1e-6
