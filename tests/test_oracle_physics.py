"""Pins of the oracle's right-hand side (Eqs. 1-3) and RK3 substep (Eq. 10,
Algorithms 2-3) against closed forms derived by hand from the paper's
equations and the stencils' Fourier eigenvalues, and against invariants.

Closed forms used (theta = k h, per axis):
  D1 sin(kx+p) = K1 cos(kx+p),  K1 h  = (45 sin t - 9 sin 2t + sin 3t)/30
  D2 sin(kx+p) = -K2 sin(kx+p), K2 h^2 = (490 - 540 cos t + 54 cos 2t - 4 cos 3t)/180
  Eq. 8 on sin(a x + b y + p) = MIX sin(...)
States that depend on one or two coordinates make every term of Eqs. 1-3
either exactly zero or a product of these eigenvalues, so each term's
coefficient and sign is checked separately.
"""
import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import inputs

from test_oracle_stencils import K1, K2, MIX

TWO_PI = 2 * np.pi


def _coord(g, axis):
    n = (g.nx, g.ny, g.nz)[axis]
    L = (g.lx, g.ly, g.lz)[axis]
    c = np.arange(n) * (L / n)
    shape = [1, 1, 1]
    shape[2 - axis] = n
    return c.reshape(shape)


def _bc(a, g):
    return np.broadcast_to(a, g.shape).copy()


G = fd.Grid(16, 12, 20, TWO_PI, 2.0, 3.0)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
@pytest.mark.parametrize("q", [0, 1, 2])
@pytest.mark.parametrize("emode", [0, 1])
def test_rhs_longitudinal_closed_form(form, q, emode):
    """lnrho = a sin(k x_q + phi), u_q = b sin(k x_q + psi), s = c sin(k x_q)."""
    g = G
    ph = fd.Physics(cs=1.3, nu=0.07, entropy_mode=emode)
    L = (g.lx, g.ly, g.lz)[q]
    h = g.spacing[q]
    k = TWO_PI * 2 / L
    k1, k2 = K1(k * h, h), K2(k * h, h)
    a, b, c, phi, psi = 0.3, 0.2, 0.5, 0.4, -0.9
    x = _coord(g, q)
    st = np.zeros((ph.nfields,) + g.shape)
    st[0] = _bc(a * np.sin(k * x + phi), g)
    st[1 + q] = _bc(b * np.sin(k * x + psi), g)
    if emode:
        st[4] = _bc(c * np.sin(k * x), g)
    r = fd.rhs(st, g, ph, form)

    Lx = a * k1 * np.cos(k * x + phi)
    uq = b * np.sin(k * x + psi)
    uqx = b * k1 * np.cos(k * x + psi)
    uqxx = -b * k2 * np.sin(k * x + psi)
    graddiv = uqxx if form == fd.FORM_55P else -b * k1 * k1 * np.sin(k * x + psi)
    want_l = -uq * Lx - uqx
    want_u = (-uq * uqx - ph.cs ** 2 * Lx
              + ph.nu * (uqxx + graddiv / 3.0 + (4.0 / 3.0) * uqx * Lx))
    tol = 1e-12
    np.testing.assert_allclose(r[0], _bc(want_l, g), atol=tol)
    np.testing.assert_allclose(r[1 + q], _bc(want_u, g), atol=tol)
    for j in range(3):
        if j != q:
            np.testing.assert_allclose(r[1 + j], 0.0, atol=tol)
    if emode:
        np.testing.assert_allclose(r[4], _bc(-uq * c * k1 * np.cos(k * x), g), atol=tol)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
@pytest.mark.parametrize("q,p", [(0, 1), (0, 2), (1, 2), (2, 0)])
def test_rhs_transverse_closed_form(form, q, p):
    """lnrho = a sin(k x_q + phi), u_p = b sin(k x_q + psi), p != q:
    tests the off-diagonal strain term 2 S_pq d_q lnrho and the pressure."""
    g = G
    ph = fd.Physics(cs=0.8, nu=0.05, entropy_mode=1)
    L = (g.lx, g.ly, g.lz)[q]
    h = g.spacing[q]
    k = TWO_PI * 3 / L
    k1, k2 = K1(k * h, h), K2(k * h, h)
    a, b, phi, psi = 0.25, 0.4, 1.1, 0.2
    x = _coord(g, q)
    st = np.zeros((5,) + g.shape)
    st[0] = _bc(a * np.sin(k * x + phi), g)
    st[1 + p] = _bc(b * np.sin(k * x + psi), g)
    r = fd.rhs(st, g, ph, form)
    Lq = a * k1 * np.cos(k * x + phi)
    upq = b * k1 * np.cos(k * x + psi)
    tol = 1e-12
    np.testing.assert_allclose(r[0], 0.0, atol=tol)
    np.testing.assert_allclose(r[1 + q], _bc(-ph.cs ** 2 * Lq, g), atol=tol)
    want_p = ph.nu * (-b * k2 * np.sin(k * x + psi) + upq * Lq)
    np.testing.assert_allclose(r[1 + p], _bc(want_p, g), atol=tol)
    other = 3 - q - p
    np.testing.assert_allclose(r[1 + other], 0.0, atol=tol)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
@pytest.mark.parametrize("q,p", [(0, 1), (1, 0), (0, 2), (2, 1)])
def test_rhs_mixed_derivative_closed_form(form, q, p):
    """u_q = b sin(kq x_q + kp x_p + psi), lnrho = 0: the grad(div u) term
    needs the bidiagonal Eq. 8 (55-point) or nested Eq. 6 (19-point)."""
    g = G
    ph = fd.Physics(cs=1.0, nu=0.09, entropy_mode=1)
    Ls = (g.lx, g.ly, g.lz)
    hq, hp = g.spacing[q], g.spacing[p]
    kq, kp = TWO_PI * 2 / Ls[q], TWO_PI * 1 / Ls[p]
    b, psi = 0.3, 0.5
    arg = kq * _coord(g, q) + kp * _coord(g, p) + psi
    st = np.zeros((5,) + g.shape)
    st[1 + q] = _bc(b * np.sin(arg), g)
    r = fd.rhs(st, g, ph, form)
    k1q, k1p = K1(kq * hq, hq), K1(kp * hp, hp)
    k2q, k2p = K2(kq * hq, hq), K2(kp * hp, hp)
    S, C = np.sin(arg), np.cos(arg)
    div = b * k1q * C
    if form == fd.FORM_55P:
        gd_q = -b * k2q * S
        gd_p = b * MIX(kq * hq, kp * hp, hq, hp) * S
    else:
        gd_q = -b * k1q * k1q * S
        gd_p = -b * k1q * k1p * S
    tol = 1e-12
    np.testing.assert_allclose(r[0], _bc(-div, g), atol=tol)
    want_q = -b * S * b * k1q * C + ph.nu * (-b * (k2q + k2p) * S + gd_q / 3.0)
    np.testing.assert_allclose(r[1 + q], _bc(want_q, g), atol=tol)
    np.testing.assert_allclose(r[1 + p], _bc(ph.nu * gd_p / 3.0, g), atol=tol)
    np.testing.assert_allclose(r[1 + (3 - q - p)], 0.0, atol=tol)


# ------------------------------------------------------------------ RK3

def G3(z):
    return 1 + z + z * z / 2 + z ** 3 / 6


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_shear_wave_discrete_decay_exact(form):
    """Sect. 6 test 1: u = u0 sin(kx) e_y.  All nonlinear and pressure terms
    vanish, so each RK3 step multiplies u_y by G(-nu K2 dt) exactly, with
    G(z) = 1 + z + z^2/2 + z^3/6 (any 3-stage third-order RK)."""
    g = fd.Grid(32, 8, 8)
    ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
    k, u0, dt, n = 5.0, 0.1, 0.05, 7
    st = inputs.shear_wave(g.shape, k, u0)
    out = fd.rk3_step(st, dt, g, ph, form, nsteps=n)
    h = g.spacing[0]
    x = np.arange(g.nx) * h
    want = u0 * np.sin(k * x) * G3(-ph.nu * K2(k * h, h) * dt) ** n
    np.testing.assert_allclose(out[2], _bc(want, g), rtol=0, atol=1e-15)
    for f in (0, 1, 3, 4):
        np.testing.assert_allclose(out[f], 0.0, atol=1e-15)


def test_rk3_coefficients_low_storage_third_order():
    """The 2N form with the coefficients in use reproduces the classical
    third-order conditions (b.1 = 1, b.c = 1/2, b.c^2 = 1/3, b.A c = 1/6)
    once rewritten as a Butcher tableau."""
    alpha, beta = fd.rk3_coefficients()
    assert alpha[0] == 0.0
    # Butcher tableau of the 2N scheme: w_s = alpha_s w_{s-1} + dt k_s,
    # u_s = u_{s-1} + beta_s w_s
    A = np.zeros((3, 3))
    bvec = np.zeros(3)
    wcoef = np.zeros(3)  # w in terms of k_1..k_s
    acc = np.zeros(3)    # u_s - u_0 in terms of k
    for s in range(3):
        A[s] = acc
        wcoef = alpha[s] * wcoef
        wcoef[s] += 1.0
        acc = acc + beta[s] * wcoef
    bvec = acc
    c = A.sum(axis=1)
    assert bvec.sum() == pytest.approx(1.0, abs=1e-15)
    assert bvec @ c == pytest.approx(0.5, abs=1e-15)
    assert bvec @ c ** 2 == pytest.approx(1.0 / 3.0, abs=1e-15)
    assert bvec @ A @ c == pytest.approx(1.0 / 6.0, abs=1e-15)


def test_rk3_third_order_on_nonlinear_problem():
    """Self-advecting compressible wave on a fixed grid: the time error of
    the whole PDE step shrinks by 8 per halving of dt."""
    g = fd.Grid(16, 1, 1)
    ph = fd.Physics(cs=1.0, nu=0.01, entropy_mode=1)
    x = np.arange(16) * (TWO_PI / 16)
    st = np.zeros((5,) + g.shape)
    st[0] = (0.2 * np.sin(x)).reshape(g.shape)
    st[1] = (0.3 * np.sin(x + 0.5)).reshape(g.shape)
    T = 0.8
    res = [fd.rk3_step(st, T / n, g, ph, nsteps=n) for n in (8, 16, 32, 64)]
    d = [np.max(np.abs(a - b)) for a, b in zip(res, res[1:])]
    for e0, e1 in zip(d, d[1:]):
        assert 7.0 < e0 / e1 < 9.0


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_linear_sound_wave(form):
    """lnrho = A sin(kx), u = 0 with A tiny: to O(A^2) the semi-discrete
    system for lnrho = a sin kx, u_x = b cos kx is d(a,b)/dt = M (a,b),
    M = [[0, K1], [-c_s^2 K1, -nu_eff]], nu_eff = (4/3) nu K2 (55-point) or
    nu (K2 + K1^2/3) (19-point); one RK3 step is exactly I + L + L^2/2 + L^3/6
    with L = dt M."""
    g = fd.Grid(24, 4, 4)
    ph = fd.Physics(cs=1.0, nu=0.03, entropy_mode=1)
    A, k, dt, n = 1e-9, 3.0, 0.04, 10
    h = g.spacing[0]
    x = np.arange(g.nx) * h
    st = np.zeros((5,) + g.shape)
    st[0] = _bc(A * np.sin(k * x), g)
    out = fd.rk3_step(st, dt, g, ph, form, nsteps=n)
    k1, k2 = K1(k * h, h), K2(k * h, h)
    nu_eff = (4.0 / 3.0) * ph.nu * k2 if form == fd.FORM_55P else ph.nu * (k2 + k1 * k1 / 3.0)
    M = np.array([[0.0, k1], [-ph.cs ** 2 * k1, -nu_eff]])
    Lm = dt * M
    P = np.eye(2) + Lm + Lm @ Lm / 2 + Lm @ Lm @ Lm / 6
    ab = np.linalg.matrix_power(P, n) @ np.array([A, 0.0])
    np.testing.assert_allclose(out[0], _bc(ab[0] * np.sin(k * x), g), atol=1e-6 * A)
    np.testing.assert_allclose(out[1], _bc(ab[1] * np.cos(k * x), g), atol=1e-6 * A)


def test_sound_speed_limit():
    """The discrete sound speed K1 c_s / k tends to c_s under refinement."""
    for n, tol in ((32, 1e-3), (64, 2e-5), (128, 3e-7)):
        h = TWO_PI / n
        assert abs(K1(1.0 * h, h) - 1.0) < tol


def test_viscous_decay_sixth_order_in_space():
    """Sect. 6 test 1 against the continuous solution u0 exp(-nu k^2 t)
    sin(kx) at k = 13, t = 1.5: the error falls by about 2^6 per halving of
    the grid spacing (the paper measured 2^5.7)."""
    k, u0, nu, T, nsteps = 13.0, 1.0, 1e-3, 1.5, 150
    errs = []
    for n in (64, 128, 256):
        g = fd.Grid(n, 1, 1)
        ph = fd.Physics(cs=1.0, nu=nu, entropy_mode=0)
        st = inputs.shear_wave(g.shape, k, u0, nfields=4)
        out = fd.rk3_step(st, T / nsteps, g, ph, nsteps=nsteps)
        x = np.arange(n) * (TWO_PI / n)
        exact = u0 * np.exp(-nu * k * k * T) * np.sin(k * x)
        errs.append(np.sqrt(np.mean((out[2].ravel() - exact) ** 2)))
    for e0, e1 in zip(errs, errs[1:]):
        assert 2 ** 5.5 < e0 / e1 < 2 ** 6.3


# ------------------------------------------------------------------ invariants

def _cfg1_like(n, seed=0):
    return inputs.sine_modes((n, n, n), seed)


def test_roll_equivariance_bitwise():
    g = fd.Grid(16, 16, 16)
    ph = fd.Physics(nu=5e-3)
    st = _cfg1_like(16)
    a = fd.rk3_step(st, 0.05, g, ph)
    b = fd.rk3_step(np.roll(st, (3, -5, 7), axis=(1, 2, 3)), 0.05, g, ph)
    assert np.array_equal(np.roll(a, (3, -5, 7), axis=(1, 2, 3)), b)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_axis_permutation_equivariance(form):
    """Swapping x and y (and u_x with u_y) commutes with the step."""
    g = fd.Grid(12, 12, 12)
    ph = fd.Physics(nu=0.02)
    st = inputs.random_state(g.shape, 3, scale=0.05)
    a = fd.rk3_step(st, 0.02, g, ph, form)
    sw = st[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2).copy()
    b = fd.rk3_step(sw, 0.02, g, ph, form)
    back = b[[0, 2, 1, 3, 4]].transpose(0, 1, 3, 2)
    np.testing.assert_allclose(back, a, rtol=0, atol=1e-14)


def test_two_pass_equals_single_update_of_19p_rhs():
    """Appendix A: the two passes of Algorithm 3 give the same substep as
    Eq. 10 applied with the full 19-point right-hand side."""
    g = fd.Grid(10, 12, 8)
    ph = fd.Physics(nu=0.03)
    st = inputs.random_state(g.shape, 5, scale=0.1)
    w0 = inputs.random_state(g.shape, 6, scale=0.01)
    alpha, beta = fd.rk3_coefficients()
    dt = 0.01
    for s in range(3):
        out, w = fd.substep(st, w0, s, dt, g, ph, fd.FORM_19P)
        r = fd.rhs(st, g, ph, fd.FORM_19P)
        w_ref = (alpha[s] * w0 if s else 0.0) + dt * r
        np.testing.assert_allclose(w, w_ref, rtol=0, atol=1e-15)
        np.testing.assert_allclose(out, st + beta[s] * w_ref, rtol=0, atol=1e-15)


def test_55p_and_19p_agree_to_truncation_and_converge():
    """Sect. 4.2: the two forms differ only in how grad(div u) is
    discretised; the difference is truncation-level and falls at 6th order."""
    diffs = []
    for n in (16, 32):
        g = fd.Grid(n, n, n)
        ph = fd.Physics(nu=0.05)
        st = inputs.sine_modes(g.shape, 11, kmax=2.0, u_amp=0.05)
        r55 = fd.rhs(st, g, ph, fd.FORM_55P)
        r19 = fd.rhs(st, g, ph, fd.FORM_19P)
        np.testing.assert_array_equal(r55[0], r19[0])
        diffs.append(np.max(np.abs(r55[1:4] - r19[1:4])))
    assert diffs[0] / diffs[1] > 40


def test_mass_drift_small_and_shrinks():
    """The log-density form does not conserve sum(rho) exactly (Sect. 6);
    the drift after 10 steps is small and falls under refinement."""
    drift = []
    for n in (16, 32):
        g = fd.Grid(n, n, n)
        ph = fd.Physics(nu=5e-3)
        st = inputs.sine_modes(g.shape, 0, kmax=2.0)
        m0 = fd.diagnostics(st, g, ph)["mass"]
        dt = fd.cfl_dt(st, g, ph, 0.4)
        out = fd.rk3_step(st, dt * 16 / n, g, ph, nsteps=10 * n // 16)
        m1 = fd.diagnostics(out, g, ph)["mass"]
        drift.append(abs(m1 / m0 - 1))
    assert drift[0] < 1e-6
    assert drift[1] < drift[0]


def test_entropy_mode0_matches_mode1_with_zero_entropy():
    g = fd.Grid(12, 10, 8)
    st5 = inputs.sine_modes(g.shape, 2, nfields=5)
    a = fd.rk3_step(st5, 0.03, g, fd.Physics(entropy_mode=1))
    b = fd.rk3_step(st5[:4], 0.03, g, fd.Physics(entropy_mode=0))
    np.testing.assert_array_equal(a[:4], b)
    assert np.all(a[4] == 0.0)
