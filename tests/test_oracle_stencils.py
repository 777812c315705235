"""Pins of the oracle's finite-difference operators (Eqs. 6-8) against
facts fixed by mathematics, not by the oracle's own code:

* polynomial exactness (Taylor): Eq. 6 is exact for degree <= 6, Eq. 7 for
  degree <= 7, Eq. 8 for total degree <= 7; the first failing degree misses
  by the textbook leading truncation term (h^6/140 f^(7) for Eq. 6,
  h^6/560 f^(8) for Eq. 7);
* modified wavenumbers: on a periodic grid a Fourier mode is an eigenvector
  of each stencil with a closed-form eigenvalue;
* sixth-order convergence of the periodic derivatives of a smooth mode.
"""
import math

import numpy as np
import pytest

from oracle import fd


def _poly_samples(coeffs, x0, h):
    xs = x0 + h * np.arange(-3, 4)
    return np.polyval(coeffs[::-1], xs)


def _deriv(coeffs, x0, order):
    c = np.polynomial.polynomial.polyder(coeffs, order)
    return np.polynomial.polynomial.polyval(x0, c)


@pytest.mark.parametrize("deg", range(0, 7))
def test_d1_exact_through_degree_6(deg):
    rng = np.random.default_rng(deg)
    coeffs = rng.uniform(-1, 1, deg + 1)
    x0, h = 0.37, 0.11
    got = fd.d1_point(_poly_samples(coeffs, x0, h), h)
    assert got == pytest.approx(_deriv(coeffs, x0, 1), rel=1e-11, abs=1e-11)


@pytest.mark.parametrize("deg", range(0, 8))
def test_d2_exact_through_degree_7(deg):
    rng = np.random.default_rng(100 + deg)
    coeffs = rng.uniform(-1, 1, deg + 1)
    x0, h = -0.21, 0.13
    got = fd.d2_point(_poly_samples(coeffs, x0, h), h)
    assert got == pytest.approx(_deriv(coeffs, x0, 2), rel=1e-9, abs=1e-9)


def test_d1_degree_7_leading_error():
    # f = x^7: D1 - f' = h^6 f^(7) / 140 = 36 h^6 exactly (odd moments)
    h = 0.1
    s = (h * np.arange(-3, 4)) ** 7
    assert fd.d1_point(s, h) == pytest.approx(5040.0 / 140.0 * h ** 6, rel=1e-10)


def test_d2_degree_8_leading_error():
    # f = x^8: D2 - f'' = h^6 f^(8) / 560 = 72 h^6 exactly (even moments)
    h = 0.1
    s = (h * np.arange(-3, 4)) ** 8
    assert fd.d2_point(s, h) == pytest.approx(40320.0 / 560.0 * h ** 6, rel=1e-10)


def test_d2_scales_with_h_squared():
    # The printed 1/(180 dx) in Eq. 7 would make D2(x^2) = 2 h, not 2.
    for h in (0.5, 0.1, 0.01):
        s = (h * np.arange(-3, 4)) ** 2
        assert fd.d2_point(s, h) == pytest.approx(2.0, rel=1e-12)


def test_dmix_xy_is_one():
    # the normalisation check 270*4 - 27*16 + 2*36 = 720
    ha, hb = 0.2, 0.3
    a = ha * np.arange(-3, 4)[:, None]
    b = hb * np.arange(-3, 4)[None, :]
    assert fd.dmix_point(a * b, ha, hb) == pytest.approx(1.0, rel=1e-13)


def test_dmix_exact_through_total_degree_7():
    rng = np.random.default_rng(7)
    ha, hb = 0.15, 0.25
    a0, b0 = 0.3, -0.4
    a = a0 + ha * np.arange(-3, 4)[:, None]
    b = b0 + hb * np.arange(-3, 4)[None, :]
    for i in range(8):
        for j in range(8 - i):
            c = rng.uniform(-1, 1)
            f = c * a ** i * b ** j
            exact = c * i * j * a0 ** max(i - 1, 0) * b0 ** max(j - 1, 0) if i and j else 0.0
            got = fd.dmix_point(f, ha, hb)
            assert got == pytest.approx(exact, rel=1e-9, abs=1e-10), (i, j)


def test_dmix_fails_at_total_degree_8():
    ha = hb = 0.1
    a = ha * np.arange(-3, 4)[:, None]
    b = hb * np.arange(-3, 4)[None, :]
    f = a ** 7 * b  # exact d2/dadb at 0 is 0; the diagonal stencils see t^8
    assert abs(fd.dmix_point(f, ha, hb)) > 1e-9


def test_dmix_ignores_axial_points():
    # only the diagonals enter: a function living on the axes gives 0
    patch = np.zeros((7, 7))
    patch[3, :] = np.arange(7.0) ** 3
    patch[:, 3] = np.arange(7.0) ** 2
    assert fd.dmix_point(patch, 0.1, 0.1) == 0.0


# ------------------------------------------------------------ Fourier pins

def K1(theta, h):
    return (45 * np.sin(theta) - 9 * np.sin(2 * theta) + np.sin(3 * theta)) / (30 * h)


def K2(theta, h):
    return (490 - 540 * np.cos(theta) + 54 * np.cos(2 * theta) - 4 * np.cos(3 * theta)) / (180 * h * h)


def MIX(ta, tb, ha, hb):
    c = (270.0, -27.0, 2.0)
    return sum(c[m - 1] * (np.cos(m * (ta + tb)) - np.cos(m * (ta - tb)))
               for m in (1, 2, 3)) / (360 * ha * hb)


GRID = fd.Grid(24, 20, 16, 2 * np.pi, 3.0, 5.0)


def _axis_coords(g):
    nz, ny, nx = g.shape
    hx, hy, hz = g.spacing
    return (np.arange(nx)[None, None, :] * hx, np.arange(ny)[None, :, None] * hy,
            np.arange(nz)[:, None, None] * hz)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 3, 5])
def test_d1_modified_wavenumber(axis, m):
    g = GRID
    L = (g.lx, g.ly, g.lz)[axis]
    h = g.spacing[axis]
    k = 2 * np.pi * m / L
    xs = _axis_coords(g)[axis]
    f = np.broadcast_to(np.sin(k * xs + 0.3), g.shape).copy()
    want = np.broadcast_to(K1(k * h, h) * np.cos(k * xs + 0.3), g.shape)
    np.testing.assert_allclose(fd.grid_d1(f, g, axis), want, rtol=0, atol=1e-12 * abs(K1(k * h, h)))


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("m", [1, 2, 6])
def test_d2_modified_wavenumber(axis, m):
    g = GRID
    L = (g.lx, g.ly, g.lz)[axis]
    h = g.spacing[axis]
    k = 2 * np.pi * m / L
    xs = _axis_coords(g)[axis]
    f = np.broadcast_to(np.sin(k * xs - 1.1), g.shape).copy()
    want = np.broadcast_to(-K2(k * h, h) * np.sin(k * xs - 1.1), g.shape)
    np.testing.assert_allclose(fd.grid_d2(f, g, axis), want, rtol=0, atol=1e-11 * K2(k * h, h))


@pytest.mark.parametrize("a,b", [(0, 1), (0, 2), (1, 2), (2, 0)])
@pytest.mark.parametrize("ma,mb", [(1, 1), (2, -3), (4, 1)])
def test_dmix_modified_wavenumber(a, b, ma, mb):
    g = GRID
    Ls = (g.lx, g.ly, g.lz)
    xs = _axis_coords(g)
    ka, kb = 2 * np.pi * ma / Ls[a], 2 * np.pi * mb / Ls[b]
    ha, hb = g.spacing[a], g.spacing[b]
    f = np.broadcast_to(np.sin(ka * xs[a] + kb * xs[b] + 0.7), g.shape).copy()
    lam = MIX(ka * ha, kb * hb, ha, hb)
    want = np.broadcast_to(lam * np.sin(ka * xs[a] + kb * xs[b] + 0.7), g.shape)
    np.testing.assert_allclose(fd.grid_dmix(f, g, a, b), want, rtol=0, atol=1e-11 * abs(lam))


def test_sixth_order_convergence():
    errs = []
    for n in (16, 32, 64, 128):
        g = fd.Grid(n, 1, 1)
        x = np.arange(n) * (2 * np.pi / n)
        f = np.sin(x + 0.2).reshape(g.shape)
        e1 = np.max(np.abs(fd.grid_d1(f, g, 0).ravel() - np.cos(x + 0.2)))
        e2 = np.max(np.abs(fd.grid_d2(f, g, 0).ravel() + np.sin(x + 0.2)))
        errs.append((e1, e2))
    for (a1, a2), (b1, b2) in zip(errs, errs[1:]):
        assert 56 < a1 / b1 < 68
        assert 56 < a2 / b2 < 68
