"""Parity bars shared by the GPU parity tests and the CPU test that shows the
element-wise bar is tight enough to catch planted mistakes.

FP64_TOL  per-field relative L2 ||g - o|| / ||o|| after the configured steps.
FP32_TOL  per-field relative L2 of one step from the oracle state rounded to
          FP32 (the FP32 output itself rounds at 2^-24 of the field).
INC_TOL   element-wise bar on the per-step increment, for FP32 storage:
          max |(g - b) - (o - b)| / max |o - b| per field, b the step's input,
          must stay within inc_bar = INC_TOL + FLOOR_ULPS 2^-24 max|o| / max|o - b|.
          The second term is the FP32 storage itself: the state is rounded to
          FP32 after each of the three substeps (half an ulp each, plus the
          rounding of u-tilde), so the output can sit a couple of ulps of the
          field's magnitude away from the FP64 oracle whatever the increment;
          where the step changes the field little (fine grids: 256^3, 512^3)
          this term dominates.  On the term-exposing state below it is about
          1e-5 and INC_TOL = 1e-4 dominates, with 10-50x headroom over what the
          FP32 kernels reach there; every planted mistake of the oracle mutant
          set moves some field's increment by more than 10 x inc_bar on that
          state (tests/test_oracle_mutants.py checks this on the CPU).
"""
import numpy as np

FP64_TOL = 1e-12
FP32_TOL = 1e-5
INC_TOL = 1e-4
FLOOR_ULPS = 4.0
EPS32 = 2.0 ** -24


def rel_l2(got, ref, abs_floor=1e-14):
    """Per-field relative L2 error (absolute floor where the oracle field is 0)."""
    out = []
    for g, o in zip(got, ref):
        no = np.linalg.norm(o.ravel())
        d = np.linalg.norm((g - o).ravel())
        out.append(d / no if no > 0 else (0.0 if d <= abs_floor * np.sqrt(o.size) else np.inf))
    return np.array(out)


def max_abs(got, ref):
    """Per-field maximum absolute error."""
    return np.array([np.abs(g - o).max() for g, o in zip(got, ref)])


def inc_err(got, ref, base):
    """Per-field element-wise error of the increment: max|(g-b)-(o-b)| / max|o-b|
    (0 for a field whose oracle increment is 0 and whose GPU increment is 0)."""
    out = []
    for g, o, b in zip(got, ref, base):
        do = o - b
        dg = g - b
        m = np.abs(do).max()
        e = np.abs(dg - do).max()
        out.append(e / m if m > 0 else (0.0 if e == 0 else np.inf))
    return np.array(out)


def inc_bar(ref, base):
    """Per-field bar on inc_err: INC_TOL plus the FP32 storage floor (0 for a
    field the oracle step leaves unchanged: the GPU must leave it unchanged
    too, since inc_err is then 0 or infinite)."""
    out = []
    for o, b in zip(ref, base):
        m = np.abs(o - b).max()
        out.append(INC_TOL + FLOOR_ULPS * EPS32 * np.abs(o).max() / m if m > 0 else 0.0)
    return np.array(out)


def term_exposing_state(shape, seed, inputs):
    """A state on which every term of Eqs. 1-3 moves the increment visibly:
    k^-2 velocity over 1 <= k <= 8 at rms Mach 0.3, lnrho perturbation 0.1
    (so the pressure and 2 nu S.grad(lnrho) terms matter), entropy 0.3 u_x.
    Used with nu = 0.02, c_s = 1, CFL 0.4.  Returned rounded to FP32 (as
    FP64 values)."""
    st = inputs.spectrum(shape, seed, p=-2.0, k1=1, k2=8, mach=0.3, lnrho_rms=0.1)
    st[4] = 0.3 * st[1]
    return st.astype(np.float32).astype(np.float64)


TERM_NU = 0.02
