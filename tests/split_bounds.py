"""Error bounds of the split-precision path used by the parity tests.

s BF16 slices keep the slice-pair products p + q < s of each operand product.
The dropped pairs are about 2^-8s of each product with random signs, and W
sums K = 2v + 2o products accumulated in FP32, whose rounding (about 2^-24
per addition, partly systematic) dominates the error of E_T for every s.
The bound is the stated 1e-6 relative, |dE| <= 1e-6 max(1 Eh, |E_T|), and
literally 1e-6 Eh on the physical-scale twins, for s = 2, 3 and 4 alike.
Measured relative errors of E_T: 1.8e-7 / 1.3e-7 / 1.3e-7 (s = 2 / 3 / 4,
o=6 v=36), 3.3e-7 for all s at o=20 v=200, 3.2e-7 to 3.3e-7 on the sampled
triplets at o=40 v=400 and 3.8e-7 to 3.9e-7 at o=50 v=450.
"""


def split_rel_bound(s, o, v):
    if s not in (2, 3, 4):
        raise ValueError("slice count must be 2, 3 or 4")
    return 1e-6
