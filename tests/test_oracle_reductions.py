"""Pins of the oracle's FP64 diagnostics, time-step helper and box filter
against values that follow directly from their definitions on states where
the answer is known in closed form."""
import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import inputs


def test_diagnostics_uniform_state():
    g = fd.Grid(8, 6, 4, 2.0, 3.0, 5.0)
    ph = fd.Physics(entropy_mode=1)
    st = np.zeros((5,) + g.shape)
    st[0] = np.log(2.0)
    st[1], st[2], st[3] = 0.3, -0.4, 0.0
    st[4] = -0.25
    d = fd.diagnostics(st, g, ph)
    vol = 2.0 * 3.0 * 5.0
    assert d["mass"] == pytest.approx(2.0 * vol, rel=1e-14)
    assert d["ekin"] == pytest.approx(0.5 * 2.0 * 0.25 * vol, rel=1e-14)
    assert d["umax"] == pytest.approx(0.5, rel=1e-15)
    assert d["urms"] == pytest.approx(0.5, rel=1e-15)
    np.testing.assert_allclose(d["rms"], [np.log(2.0), 0.3, 0.4, 0.0, 0.25], rtol=1e-14)
    np.testing.assert_allclose(d["maxabs"], [np.log(2.0), 0.3, 0.4, 0.0, 0.25], rtol=1e-15)
    assert d["nonfinite"] == 0


def test_diagnostics_sine_mass_closed_form():
    """mass of rho = exp(a sin x) on a fine periodic grid -> 2 pi L^2 I0(a)."""
    from scipy.special import i0
    n = 64
    g = fd.Grid(n, 2, 2, 2 * np.pi, 1.0, 1.0)
    ph = fd.Physics(entropy_mode=0)
    st = np.zeros((4,) + g.shape)
    x = np.arange(n) * (2 * np.pi / n)
    st[0] = (0.7 * np.sin(x))[None, None, :]
    d = fd.diagnostics(st, g, ph)
    # trapezoid rule on a periodic analytic function is spectrally exact
    assert d["mass"] == pytest.approx(2 * np.pi * i0(0.7), rel=1e-14)


def test_diagnostics_flags_nonfinite():
    g = fd.Grid(4, 4, 4)
    ph = fd.Physics(entropy_mode=1)
    st = np.zeros((5,) + g.shape)
    st[3, 1, 2, 3] = np.nan
    assert fd.diagnostics(st, g, ph)["nonfinite"] == 1
    st[3, 1, 2, 3] = np.inf
    assert fd.diagnostics(st, g, ph)["nonfinite"] == 1


def test_cfl_dt_limits():
    g = fd.Grid(32, 32, 32)
    h = 2 * np.pi / 32
    st = np.zeros((5,) + g.shape)
    st[1] = 0.5
    ph = fd.Physics(cs=1.0, nu=5e-3)
    assert fd.cfl_dt(st, g, ph, cfl=0.4) == pytest.approx(0.4 * h / 1.5, rel=1e-15)
    ph = fd.Physics(cs=1.0, nu=1.0)  # viscous limit binds
    assert fd.cfl_dt(st, g, ph, cfl=0.4, cnu=0.25) == pytest.approx(0.25 * h * h, rel=1e-15)


def test_box_filter_preserves_constants_and_mean():
    fine = inputs.random_state((16, 16, 16), 9, scale=1.0)
    fine[2] = 3.5
    c = fd.box_filter(fine, 4)
    np.testing.assert_allclose(c[2], 3.5, rtol=1e-15)
    np.testing.assert_allclose(c.mean(axis=(1, 2, 3)), fine.mean(axis=(1, 2, 3)), atol=1e-15)


def test_box_filter_fourier_multiplier():
    """Per axis the filter weights (1/2,1,1,1,1/2)/4 multiply a mode of
    fine-grid phase step t by (cos 2t + 2 cos t + 1)/4, centred on the
    coarse vertex (no shift)."""
    n, r = 32, 4
    x = np.arange(n) * (2 * np.pi / n)
    fine = np.zeros((1, n, n, n))
    fine[0] = np.sin(3 * x)[None, None, :] * np.cos(2 * x)[None, :, None]
    c = fd.box_filter(fine, r)
    t3, t2 = 3 * 2 * np.pi / n, 2 * 2 * np.pi / n
    m3 = (np.cos(2 * t3) + 2 * np.cos(t3) + 1) / 4
    m2 = (np.cos(2 * t2) + 2 * np.cos(t2) + 1) / 4
    X = np.arange(n // r) * r * (2 * np.pi / n)
    want = m3 * m2 * np.sin(3 * X)[None, :] * np.cos(2 * X)[:, None]
    np.testing.assert_allclose(c[0, 0], want, atol=1e-14)
