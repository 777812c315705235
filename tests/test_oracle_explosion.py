"""The radial-explosion symmetry test (Sect. 6, Eq. 19) on the CPU oracle.

Pins: the seven-axis integral is exact for a radial Gaussian (spacing h along
x, y, z and sqrt(3) h along a diagonal); and since Eqs. 1-3 and the stencils
of Eqs. 6-9 are covariant under the symmetries of the cube, a centred
spherical initial state keeps the x, y and z integrals equal, and the four
diagonal integrals equal, to rounding -- only axis against diagonal measures
the scheme's anisotropy."""
import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import explosion, inputs


def test_axis_integrals_of_a_radial_gaussian():
    n, L, sig = 64, 2 * np.pi, 0.3
    h = L / n
    ax = np.arange(n) * h - L / 2
    z, y, x = np.meshgrid(ax, ax, ax, indexing="ij")
    r2 = x * x + y * y + z * z
    st = np.zeros((5, n, n, n))
    st[0] = np.log1p(np.exp(-r2 / (2 * sig * sig)))  # rho - 1 = the Gaussian
    st[1] = np.exp(-r2 / (2 * sig * sig))             # |u| = the Gaussian
    ir, iu = explosion.axis_integrals(st)
    exact = sig * np.sqrt(2 * np.pi)
    np.testing.assert_allclose(ir, exact, rtol=1e-10)
    np.testing.assert_allclose(iu, exact, rtol=1e-10)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_explosion_keeps_the_cube_symmetries(form):
    n = 32
    g = fd.Grid(n, n, n)
    ph = fd.Physics(cs=1.0, nu=5e-3, entropy_mode=1)
    st = inputs.explosion((n, n, n))
    dt = fd.cfl_dt(st, g, ph, 0.4)
    out = fd.rk3_step(st, dt, g, ph, form=form, nsteps=12)
    ir, iu = explosion.axis_integrals(out)
    for v in (ir, iu):
        scale = np.abs(v).max()
        assert np.ptp(v[:3]) <= 1e-12 * scale, v
        assert np.ptp(v[3:]) <= 1e-12 * scale, v
    dr, du = explosion.asymmetry(out)
    # the density has moved and the measure sees only axis vs diagonal
    assert np.abs(ir).max() > 1e-4
    assert 0 < du < 0.2 and 0 < dr < 1.0


def test_reynolds_reading():
    assert explosion.reynolds(1e-3) == pytest.approx(200.0)
