"""Pins of the oracle's forcing (Sect. 6, Eqs. 20-21), independent of its
code: vector identities of f_k, the scaling laws of N, the closed form of
the right-hand side on a resting state, and the exact 2N-RK3 response to a
constant source."""
import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import inputs

TWO_PI = 2 * np.pi


def _rand_case(seed):
    rng = np.random.default_rng(seed)
    k = rng.integers(-4, 5, size=3)
    while not k.any():
        k = rng.integers(-4, 5, size=3)
    e = rng.standard_normal(3)
    e /= np.linalg.norm(e)
    return k, e


@pytest.mark.parametrize("seed", range(6))
def test_fk_is_a_unit_vector_normal_to_k_and_e(seed):
    k, e = _rand_case(seed)
    amp = fd.forcing_amplitude(k, e, f0=1.0, cs=1.0, dt=1.0)
    n = np.linalg.norm(amp)
    fk = amp / n
    assert np.dot(fk, k) == pytest.approx(0.0, abs=1e-12 * n)
    assert np.dot(fk, e) == pytest.approx(0.0, abs=1e-12)
    # right-handed: (k x e) . f_k > 0
    assert np.dot(np.cross(k, e), fk) > 0


def test_amplitude_scaling_laws():
    """N is linear in f0, goes as c_s^(3/2), |k|^(1/2) and dt^(-1/2)."""
    k, e = np.array([1, 2, -1]), np.array([0.6, 0.0, 0.8])
    ref = np.linalg.norm(fd.forcing_amplitude(k, e, 0.3, 1.0, 1e-3))
    assert np.linalg.norm(fd.forcing_amplitude(k, e, 0.6, 1.0, 1e-3)) == pytest.approx(2 * ref)
    assert np.linalg.norm(fd.forcing_amplitude(k, e, 0.3, 4.0, 1e-3)) == pytest.approx(8 * ref)
    assert np.linalg.norm(fd.forcing_amplitude(k, e, 0.3, 1.0, 4e-3)) == pytest.approx(ref / 2)
    assert np.linalg.norm(fd.forcing_amplitude(4 * k, e, 0.3, 1.0, 1e-3)) == pytest.approx(2 * ref)
    # physical k = 2 pi k / L: halving every L doubles |k|
    half = np.linalg.norm(fd.forcing_amplitude(k, e, 0.3, 1.0, 1e-3, lengths=(np.pi,) * 3))
    assert half == pytest.approx(np.sqrt(2) * ref)
    with pytest.raises(ValueError):
        fd.forcing_amplitude([0, 0, 0], e, 0.3, 1.0, 1e-3)
    with pytest.raises(ValueError):
        fd.forcing_amplitude([0, 0, 2], [0.0, 0.0, 1.0], 0.3, 1.0, 1e-3)


@pytest.mark.parametrize("form", [fd.FORM_55P, fd.FORM_19P])
def test_resting_state_rhs_is_the_forcing(form):
    """u = 0, lnrho = 0, s = 0: every other term of Eqs. 1-3 vanishes, so the
    momentum right-hand side is N f_k cos(k.x + phi) and the rest is 0."""
    nx, ny, nz = 12, 8, 10
    lx, ly, lz = TWO_PI, 2.0, 3.0
    g = fd.Grid(nx, ny, nz, lx, ly, lz)
    ph = fd.Physics(cs=1.3, nu=0.02, entropy_mode=1)
    st = np.zeros((5, nz, ny, nx))
    k, e, phi, dt, f0 = np.array([2, -1, 3]), np.array([1.0, 0.0, 0.0]), 0.7, 2e-3, 0.05
    r = fd.rhs_forced(st, g, ph, dt, f0, k, phi, e, form=form)
    amp = fd.forcing_amplitude(k, e, f0, ph.cs, dt, lengths=(lx, ly, lz))
    z, y, x = np.meshgrid(np.arange(nz) * lz / nz, np.arange(ny) * ly / ny,
                          np.arange(nx) * lx / nx, indexing="ij")
    c = np.cos(TWO_PI * (k[0] * x / lx + k[1] * y / ly + k[2] * z / lz) + phi)
    for i in range(3):
        np.testing.assert_allclose(r[1 + i], amp[i] * c, rtol=0, atol=1e-13 * np.abs(amp).max())
    assert np.all(r[0] == 0) and np.all(r[4] == 0)


def test_constant_source_rk3_step_is_exact():
    """From rest with nu = 0 the first substep's source is the forcing alone
    and 2N-RK3 integrates a constant source exactly (weights sum to 1); what
    the nonlinear terms add is second order in the forcing."""
    nx = ny = nz = 12
    g = fd.Grid(nx, ny, nz)
    ph = fd.Physics(cs=1.0, nu=0.0, entropy_mode=1)
    st = np.zeros((5, nz, ny, nx))
    k, e, phi, dt = np.array([1, 1, 0]), np.array([0.0, 0.0, 1.0]), 0.3, 1e-3
    res = []
    for f0 in (1e-6, 2e-6):
        out = fd.rk3_step_forced(st, dt, g, ph, f0, [k], [phi], [e])
        f = fd.rhs_forced(st, g, ph, dt, f0, k, phi, e)
        res.append(np.abs(out[1:4] - dt * f[1:4]).max() / np.abs(dt * f[1:4]).max())
    # the deviation is quadratic in the forcing: doubling f0 doubles the relative deviation
    assert res[0] < 1e-6
    assert res[1] == pytest.approx(2 * res[0], rel=0.05)


def test_zero_forcing_is_the_unforced_step():
    g = fd.Grid(16, 12, 8)
    ph = fd.Physics(cs=1.0, nu=5e-3, entropy_mode=1)
    st = inputs.spectrum((8, 12, 16), 3, mach=0.2, lnrho_rms=1e-2)
    ks, phis, es = inputs.forcing_sequence(5, 2)
    a = fd.rk3_step_forced(st, 0.01, g, ph, 0.0, ks, phis, es)
    b = fd.rk3_step(st, 0.01, g, ph, nsteps=2)
    assert np.array_equal(a, b)


def test_forcing_sequence_draws():
    ks, phis, es = inputs.forcing_sequence(11, 200, kmin=1.0, kmax=2.0)
    kn = np.linalg.norm(ks, axis=1)
    assert np.all((kn >= 1.0) & (kn <= 2.0))
    assert np.allclose(np.linalg.norm(es, axis=1), 1.0)
    assert np.allclose(np.einsum("ij,ij->i", ks, es), 0.0, atol=1e-12)
    assert np.all((phis >= 0) & (phis < TWO_PI))
    # the set {1 <= |k| <= 2} has mean |k| 1.53 (the paper's smallest k_f)
    pool = inputs.forcing_set(1.0, 2.0)
    assert np.linalg.norm(pool, axis=1).mean() == pytest.approx(1.53, abs=0.01)
