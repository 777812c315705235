"""Precision study: FP32 storage and stencils with the RK3 update in FP32, in
FP64 registers (u-tilde stored in FP32 or FP64), or in float-float FP32
pairs, against an FP64 run of the same solver on the same state.  (The one-step check of this workload
against the FP64 oracle on 64^3 windows is a GPU test:
tests/test_gpu_parity.py::test_config3_window_against_oracle.)

Workload: 512^3 periodic box, k^-5/3 velocity spectrum over 1 <= k <= 16 at
rms Mach 0.3 (seed 2), lnrho perturbation 1e-2, nu 5e-3, 50 RK3 steps at CFL
0.4, 55-point form.

    python -m paper_1707_08900_gb300.precision --n 512 --steps 50 --out study.json

Errors per field: relative L2 ||x - x64|| / ||x64|| and max |x - x64| /
max |x64|; diagnostics (FP64 reductions) side by side.
"""
import argparse
import json
import time

import numpy as np

from . import gbfd, inputs

FORMS = ("fp32", "fp32_acc64", "fp32_acc64_w64", "fp32_accff")


def _errors(x, ref):
    out = []
    for f in range(ref.shape[0]):
        d = x[f] - ref[f]
        nr = np.linalg.norm(ref[f].ravel())
        mr = np.abs(ref[f]).max()
        out.append({"rel_l2": float(np.linalg.norm(d.ravel()) / nr) if nr > 0 else float(np.abs(d).max()),
                    "rel_max": float(np.abs(d).max() / mr) if mr > 0 else float(np.abs(d).max())})
    return out


def _timed(s, dt, steps):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s.rk3_step(dt, steps)
    s.sync()
    return time.perf_counter() - t0


def run(n=512, steps=50, seed=2, nu=5e-3):
    shape = (n, n, n)
    st = inputs.spectrum(shape, seed, p=-5.0 / 3.0, k1=1, k2=16, mach=0.3, lnrho_rms=1e-2)
    res = {"n": n, "steps": steps, "seed": seed, "nu": nu, "forms": {}}
    s64 = gbfd.Solver(shape, precision="fp64", nu=nu)
    s64.set_state(st)
    dt = s64.cfl_dt(0.4)
    res["dt"] = dt
    sec = _timed(s64, dt, steps)
    ref = s64.get_state()
    res["fp64"] = {"seconds": sec, "updates_per_s": n ** 3 * steps / sec,
                   "diagnostics": {k: v for k, v in s64.diagnostics().items()
                                   if k in ("mass", "ekin", "umax")}}
    s64.close()
    st32 = st.astype(np.float32)
    for prec in FORMS:
        s = gbfd.Solver(shape, precision=prec, nu=nu)
        s.set_state(st32)
        sec = _timed(s, dt, steps)
        x = s.get_state()
        d = s.diagnostics()
        res["forms"][prec] = {"seconds": sec, "updates_per_s": n ** 3 * steps / sec,
                              "errors": _errors(x, ref),
                              "diagnostics": {k: d[k] for k in ("mass", "ekin", "umax")}}
        s.close()
        del x
    # the FP32 rounding of the initial state alone, for scale
    res["initial_fp32_rounding"] = _errors(st32.astype(np.float64), st)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    res = run(a.n, a.steps)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(text)


if __name__ == "__main__":
    main()
