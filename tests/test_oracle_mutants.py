"""Planted mistakes: each mutant is a copy of the C oracle with one
plausible error (dropped term, wrong sign, wrong index, wrong factor),
compiled to a temporary library.  The pins must reject every mutant; a
mutant that survives means the pins leave that part of the method
unchecked.  Mistakes are planted only in a CPU copy of the oracle."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import build_oracle, fd

MUTANTS = {
    "d1_sign": ("45.0 * s[4] - 9.0 * s[5]", "45.0 * s[4] + 9.0 * s[5]"),
    "d2_h_not_squared": ("(180.0 * h * h)", "(180.0 * h)"),
    "dmix_k2_sign": ("- 27.0 * k2", "+ 27.0 * k2"),
    "dmix_index": ("S(1, 1) - S(-1, 1) + S(-1, -1) - S(1, -1)",
                   "S(1, 1) - S(-1, 1) + S(-1, -1) - S(1, 1)"),
    "continuity_drops_div": ("rhs[0] = -adv_lnrho - divu;", "rhs[0] = -adv_lnrho;"),
    "strain_factor": ("ph->nu * (lap + 2.0 * sgl)", "ph->nu * (lap + sgl)"),
    "strain_trace": ("(2.0 / 3.0) * divu", "(1.0 / 3.0) * divu"),
    "strain_transpose": ("S[i][j] * glnrho[j]", "S[j][i] * glnrho[i]"),
    "advection_index": ("adv += uc[j] * gu[i][j];", "adv += uc[i] * gu[i][j];"),
    "pressure_sign": ("- ph->cs2 * glnrho[i]", "+ ph->cs2 * glnrho[i]"),
    "graddiv_third": ("(ph.nu / 3.0) * gd[i];", "(ph.nu / 2.0) * gd[i];"),
    "graddiv_axis": ("dmix(u[j], g, p, i, j)", "dmix(u[i], g, p, i, j)"),
    "rk3_alpha": ("-153.0 / 128.0", "-151.0 / 128.0"),
    "rk3_beta": ("15.0 / 16.0", "13.0 / 16.0"),
    "pass2_beta": ("out[(1 + i) * n + c] += RK3_BETA[s] *", "out[(1 + i) * n + c] += "),
    "entropy_sign": ("rhs[4] = -adv_s;", "rhs[4] = adv_s;"),
}


def _build_mutant(tmp, name, old, new):
    src = open(build_oracle.SRC).read()
    assert src.count(old) >= 1, name
    src = src.replace(old, new)
    path = os.path.join(tmp, name + ".c")
    with open(path, "w") as f:
        f.write(src)
    so = os.path.join(tmp, name + ".so")
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", so,
                    path, "-lm"], check=True, capture_output=True)
    return so


def _pin_suite():
    """A fast subset of the pins that between them cover every term."""
    import test_oracle_physics as P
    import test_oracle_stencils as S
    checks = [
        lambda: S.test_d1_exact_through_degree_6(3),
        lambda: S.test_d2_scales_with_h_squared(),
        lambda: S.test_dmix_xy_is_one(),
        lambda: S.test_dmix_modified_wavenumber(0, 1, 2, -3),
    ]
    for form in (0, 1):
        for q in (0, 2):
            checks.append(lambda form=form, q=q: P.test_rhs_longitudinal_closed_form(form, q, 1))
        checks.append(lambda form=form: P.test_rhs_transverse_closed_form(form, 0, 1))
        checks.append(lambda form=form: P.test_rhs_mixed_derivative_closed_form(form, 0, 1))
        checks.append(lambda form=form: P.test_linear_sound_wave(form))
        checks.append(lambda form=form: P.test_shear_wave_discrete_decay_exact(form))
    checks.append(P.test_rk3_third_order_on_nonlinear_problem)
    checks.append(P.test_rk3_coefficients_low_storage_third_order)
    return checks


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="oracle_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_reject_mutant(name, mutant_dir):
    old, new = MUTANTS[name]
    so = _build_mutant(mutant_dir, name, old, new)
    saved = fd._lib
    try:
        fd._lib = None
        real_build = build_oracle.build
        build_oracle.build = lambda force=False: so
        try:
            fd.lib()
        finally:
            build_oracle.build = real_build
        failures = 0
        for check in _pin_suite():
            try:
                check()
            except AssertionError:
                failures += 1
        assert failures > 0, f"mutant {name} survived every pin"
    finally:
        fd._lib = saved


def test_unmutated_oracle_passes_suite():
    for check in _pin_suite():
        check()


def test_increment_bar_catches_every_mutant(mutant_dir):
    """The GPU parity tests bound the element-wise error of the FP32
    per-step increment by bars.inc_bar on the term-exposing state.  That
    bar must be tight enough to catch a mistake anywhere in the right-hand
    side: each planted mutant's increment must differ from the oracle's by
    more than 10 x inc_bar in some field, in the 55-point or the 19-point
    form (the 19-point pass-2 mutant only shows in the latter)."""
    import bars
    from paper_1707_08900_gb300 import inputs
    shape = (20, 24, 32)
    nz, ny, nx = shape
    g = fd.Grid(nx, ny, nz)
    ph = fd.Physics(cs=1.0, nu=bars.TERM_NU, entropy_mode=1)
    base = bars.term_exposing_state(shape, 11, inputs)
    dt = fd.cfl_dt(base, g, ph, 0.4)
    refs = [fd.rk3_step(base, dt, g, ph, form) for form in (fd.FORM_55P, fd.FORM_19P)]
    saved = fd._lib
    for name, (old, new) in sorted(MUTANTS.items()):
        so = _build_mutant(mutant_dir, name, old, new)
        try:
            fd._lib = None
            real_build = build_oracle.build
            build_oracle.build = lambda force=False: so
            try:
                fd.lib()
            finally:
                build_oracle.build = real_build
            worst = max((bars.inc_err(fd.rk3_step(base, dt, g, ph, form), ref, base)
                         / bars.inc_bar(ref, base)).max()
                        for form, ref in zip((fd.FORM_55P, fd.FORM_19P), refs))
        finally:
            fd._lib = saved
        assert worst > 10, (name, worst)
