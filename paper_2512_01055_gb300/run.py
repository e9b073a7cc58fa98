"""Run (T) energies on one seeded synthetic job through the C ABI.

    python -m paper_2512_01055_gb300.run --o 8 --v 128 [--prec fp64|split] [--slices 3] [--repeat 1] [--seed 7] [--df]

Prints one line per call: E_T, wall seconds, kernel seconds (all W/V/energy
kernels, and the W-forming kernels alone) and the algorithmic TFLOP/s.  With
--df the integrals are passed as the density-fitting factor and assembled by
the library (tc_energy_df_dev).  Used for quick runs and as the target of
profiler captures on small cases.
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--o", type=int, required=True)
    ap.add_argument("--v", type=int, required=True)
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--prec", default="fp64", choices=["fp64", "split"])
    ap.add_argument("--slices", type=int, default=3)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--df", action="store_true", help="pass the DF factor (tc_energy_df_dev)")
    a = ap.parse_args(argv)

    import torch
    import synth
    import paper_2512_01055_gb300 as tc
    from paper_2512_01055_gb300 import build

    build.build()
    # the seeded DF factor and amplitudes drawn on the host, the integral blocks
    # formed from them on the device (exact: the factor sits on a 2^-20 grid)
    amp = synth.make_amplitudes(a.o, a.v, a.seed)
    if a.df:
        f = lambda x: torch.from_numpy(x).to("cuda")
        dev = {"eps": f(amp.eps), "t1": f(amp.t1), "t2": f(amp.t2), "B": f(amp.B)}
    else:
        dev = synth.device_job(amp)
    ctx = tc.tc_init(0)
    prec = tc.TC_FP64 if a.prec == "fp64" else tc.TC_SPLIT_BF16
    try:
        for _ in range(a.repeat):
            if a.df:
                r = tc.tc_energy_df_dev(ctx, a.o, a.v, dev["B"], dev["eps"], dev["t1"], dev["t2"], prec=prec,
                                        slices=a.slices if prec else 0)
            else:
                r = tc.tc_energy_dev(ctx, a.o, a.v, dev["eps"], dev["t1"], dev["t2"], dev["ovvv"], dev["ovoo"],
                                     dev["ovov"], prec=prec, slices=a.slices if prec else 0)
            print(f"o={a.o} v={a.v} prec={a.prec} E_T={r.e_t:.15e} wall_s={r.seconds:.4f} "
                  f"kernel_s={r.kernel_seconds:.4f} wterm_s={r.wterm_seconds:.4f} prep_s={r.prep_seconds:.4f} "
                  f"df_s={r.df_seconds:.4f} digits={r.df_digits} TFLOP/s={r.tflops_alg:.3f}")
    finally:
        tc.tc_finalize(ctx)


if __name__ == "__main__":
    main()
