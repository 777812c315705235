"""Pins of the oracle's wall variant (z bounded by two free-slip,
impermeable walls through the grid points z = 0 and z = Lz; ghost zones
filled by mirror images, Sect. 4 / Algorithm 1's boundary step).

The exact reference: a mirror-symmetric state stays mirror-symmetric under
the periodic method, so the wall run on N_z planes must reproduce the
periodic run (pinned independently by the stencil and physics pins) on the
2 (N_z - 1) planes of the mirror-extended state, restricted to the interior.
Both sides read the same stencil values in the same order at every interior
point; they differ only because the periodic run's mirrored half is not
kept bit-for-bit symmetric (the stencil sums are not evaluated in a
symmetric order), so the agreement is to rounding."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from oracle import build_oracle, fd
from paper_1707_08900_gb300 import inputs

PAR = np.array(fd.WALL_PARITY)


def mirror_extend(st):
    """(nf, nz, ny, nx) -> (nf, 2 (nz - 1), ny, nx): planes nz .. 2 nz - 3 are
    the parity-scaled mirror images of planes nz - 2 .. 1."""
    nf, nz = st.shape[:2]
    back = st[:, nz - 2:0:-1] * PAR[:nf, None, None, None]
    return np.ascontiguousarray(np.concatenate([st, back], axis=1))


def wall_state(shape, seed, nf=5):
    """A smooth random state that satisfies the wall condition (u_z = 0 on
    both walls): even fields from cosines in z, u_z from sines."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z = np.arange(nz) * np.pi / (nz - 1)  # z / Lz * pi
    y = np.arange(ny) * 2 * np.pi / ny
    x = np.arange(nx) * 2 * np.pi / nx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    st = np.zeros((nf,) + shape)
    for f in range(nf):
        for _ in range(6):
            m, ky, kx = rng.integers(0, 4), rng.integers(0, 3), rng.integers(0, 3)
            amp = (0.02 if f == 0 else 0.05) * rng.standard_normal()
            ph = rng.uniform(0, 2 * np.pi)
            zf = np.sin(m * Z) if f == 3 else np.cos(m * Z)
            st[f] += amp * zf * np.cos(ky * Y + kx * X + ph)
    return st


def _grids(nz, ny, nx, lz=2.0):
    gw = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, lz)
    gp = fd.Grid(nx, ny, 2 * (nz - 1), 2 * np.pi, 2 * np.pi, 2 * lz)
    return gw, gp


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_wall_run_is_the_periodic_run_of_the_mirror_extension(form):
    nz, ny, nx = 12, 10, 16
    st = wall_state((nz, ny, nx), 3)
    gw, gp = _grids(nz, ny, nx)
    ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
    assert gw.lz / (gw.nz - 1) == pytest.approx(gp.lz / gp.nz)
    dt = fd.cfl_dt_wall(st, gw, ph, 0.4)
    got = fd.rk3_step_wall(st, dt, gw, ph, form, nsteps=3)
    ref = fd.rk3_step(mirror_extend(st), dt, gp, ph, form, nsteps=3)[:, :nz]
    scale = np.abs(ref).max(axis=(1, 2, 3))
    err = np.abs(got - ref).max(axis=(1, 2, 3)) / scale
    assert np.all(err < 1e-14), err
    # the state moved: the test is not comparing two copies of the input
    assert np.abs(got - st).max() > 1e-4


def test_ghost_fill_is_the_parity_mirror():
    rng = np.random.default_rng(1)
    nz = 9
    ext = rng.standard_normal((5, nz + 6, 4, 8))
    want = ext.copy()
    for k in range(1, 4):
        want[:, 3 - k] = PAR[:, None, None] * want[:, 3 + k]
        want[:, 3 + nz - 1 + k] = PAR[:, None, None] * want[:, 3 + nz - 1 - k]
    fd.fill_ghosts_z(ext)
    assert np.array_equal(ext, want)


def test_normal_velocity_stays_zero_on_the_walls():
    """u_z = 0 on both walls is kept to rounding: its right-hand side there is
    a sum of terms that vanish identically for mirror-symmetric data."""
    nz, ny, nx = 10, 8, 12
    st = wall_state((nz, ny, nx), 5)
    gw, _ = _grids(nz, ny, nx)
    ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
    dt = fd.cfl_dt_wall(st, gw, ph, 0.4)
    out = fd.rk3_step_wall(st, dt, gw, ph, nsteps=4)
    umax = np.abs(out[1:4]).max()
    assert np.abs(out[3, 0]).max() < 1e-14 * umax
    assert np.abs(out[3, -1]).max() < 1e-14 * umax
    assert np.abs(out[1:3, 0]).max() > 1e-3 * umax  # the tangential flow is free


# Planted mistakes in the wall code, each in a CPU copy of the oracle: the
# mirror-extension pin must reject every one.
WALL_MUTANTS = {
    "parity_ignored": ("a[-k * plane + c] = parity[f] * a[k * plane + c];",
                       "a[-k * plane + c] = a[k * plane + c];"),
    "mirror_off_by_one": ("a[(nz - 1 + k) * plane + c] = parity[f] * a[(nz - 1 - k) * plane + c];",
                          "a[(nz - 1 + k) * plane + c] = parity[f] * a[(nz - k) * plane + c];"),
    "spacing_periodic": ("g.h[2] = walls ? lz / (double)(nz - 1) : lz / (double)nz;",
                         "g.h[2] = lz / (double)nz;"),
    "divergence_ghosts_stale": ("        or_fill_ghosts_z(divf, nx, ny, nz, 1, &even);",
                                "        (void)even;"),
}


@pytest.fixture(scope="module")
def mutant_dir():
    d = tempfile.mkdtemp(prefix="oracle_wall_mutants_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("name", sorted(WALL_MUTANTS))
def test_mirror_pin_rejects_wall_mutant(name, mutant_dir):
    old, new = WALL_MUTANTS[name]
    src = open(build_oracle.SRC).read()
    assert src.count(old) == 1, name
    path = os.path.join(mutant_dir, name + ".c")
    with open(path, "w") as f:
        f.write(src.replace(old, new))
    so = os.path.join(mutant_dir, name + ".so")
    subprocess.run(["gcc", "-O1", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", "-o", so,
                    path, "-lm"], check=True, capture_output=True)
    saved = fd._lib
    try:
        fd._lib = None
        real_build = build_oracle.build
        build_oracle.build = lambda force=False: so
        try:
            fd.lib()
        finally:
            build_oracle.build = real_build
        failed = 0
        for form in (fd.FORM_55P, fd.FORM_19P):
            try:
                test_wall_run_is_the_periodic_run_of_the_mirror_extension(form)
            except AssertionError:
                failed += 1
        assert failed > 0, f"wall mutant {name} survived"
    finally:
        fd._lib = saved
