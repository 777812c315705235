"""Run the solver on a synthetic periodic box through the C ABI.

    python -m paper_1707_08900_gb300.run --n 256 --precision fp32 --form 55p --steps 10

Draws the k^-2 spectrum initial state (rms Mach 0.1, lnrho 1e-3, seed 1),
takes dt from CFL 0.4 once, advances `steps` RK3 steps, synchronises and
prints the diagnostics.  Also the program profiled when a single kernel is captured.

    python -m paper_1707_08900_gb300.run --n 128 --batch-boxes 4 --batch-kernel 0 --steps 1

runs the batched form instead: that many n^3 boxes (seeds 100 + i, FP32),
one dataflow launch per call with the chosen column routine and z-chunk, no
graph (so each call is one launch of the dataflow kernel).
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
    ap.add_argument("--batch-boxes", type=int, default=0, help="run the batched form")
    ap.add_argument("--batch-kernel", type=int, default=0, help="column routine (batch)")
    ap.add_argument("--batch-zchunk", type=int, default=64, help="planes per work item (batch)")
    args = ap.parse_args()
    if args.batch_boxes:
        return run_batch(args)

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


def run_batch(args):
    import torch

    from . import build, gbfd, inputs
    build.build()
    nb, n = args.batch_boxes, args.n
    b = gbfd.Batch([n] * nb, [2 * np.pi] * nb, [5e-3] * nb)
    b.set_option(gbfd.GBFD_BATCH_OPT_GRAPH, 0)
    b.set_option(gbfd.GBFD_BATCH_OPT_DATAFLOW, 1)
    b.set_option(gbfd.GBFD_BATCH_OPT_KERNEL, args.batch_kernel)
    b.set_option(gbfd.GBFD_BATCH_OPT_ZCHUNK, args.batch_zchunk)
    for i in range(nb):
        st = inputs.spectrum((n,) * 3, 100 + i, p=-2.0, k1=1, k2=8, mach=0.1, lnrho_rms=1e-3)
        b.set_state(i, st.astype(np.float32))
    dts = [0.4 * (2 * np.pi / n) / (1.0 + b.diagnostics(i)["umax"]) for i in range(nb)]
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        b.step(dts, 1)
    b.sync()
    el = time.perf_counter() - t
    d = b.diagnostics(0)
    print(json.dumps({"boxes": nb, "n": n, "kernel": args.batch_kernel, "zchunk": args.batch_zchunk,
                      "steps": args.steps, "seconds": el,
                      "updates_per_s": nb * n ** 3 * args.steps / el,
                      "mass0": d["mass"], "nonfinite0": d["nonfinite"]}))
    b.close()


if __name__ == "__main__":
    main()
