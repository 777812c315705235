"""Run the solver on a synthetic periodic box through the C ABI.

    python -m paper_1707_08900_gb300.run --n 256 --precision fp32 --form 55p --steps 10

Draws the k^-2 spectrum initial state (rms Mach 0.1, lnrho 1e-3, seed 1),
takes dt from CFL 0.4 once, advances `steps` RK3 steps, synchronises and
prints the diagnostics.  Also the program profiled when a single kernel is captured.
"""
import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--form", default="55p")
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--entropy-mode", type=int, default=1)
    ap.add_argument("--tile-config", type=int, default=-1)
    ap.add_argument("--simple", action="store_true", help="one-thread-per-point kernels")
    args = ap.parse_args()

    import torch

    from . import build, gbfd, inputs
    build.build()
    shape = (args.n,) * 3
    nf = 5 if args.entropy_mode else 4
    st = inputs.spectrum(shape, 1, p=-2.0, k1=1, k2=8, mach=0.1, lnrho_rms=1e-3, nfields=nf)
    s = gbfd.Solver(shape, precision=args.precision, form=args.form,
                    entropy_mode=args.entropy_mode, nu=5e-3)
    if args.simple:
        s.set_option(gbfd.GBFD_OPT_KERNEL_PATH, 1)
    s.set_option(gbfd.GBFD_OPT_TILE_CONFIG, args.tile_config)
    s.set_state(st if args.precision == "fp64" else st.astype(np.float32))
    dt = s.cfl_dt(0.4)
    torch.cuda.synchronize()
    t = time.perf_counter()
    s.rk3_step(dt, args.steps)
    s.sync()
    el = time.perf_counter() - t
    d = s.diagnostics()
    print(json.dumps({"n": args.n, "precision": args.precision, "form": args.form,
                      "steps": args.steps, "dt": dt, "seconds": el,
                      "updates_per_s": args.n ** 3 * args.steps / el,
                      "mass": d["mass"], "ekin": d["ekin"], "nonfinite": d["nonfinite"]}))
    s.close()


if __name__ == "__main__":
    main()
