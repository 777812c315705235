"""Seeded synthetic initial conditions (host side, NumPy).

This module is the only code that both the CUDA path's tests and the CPU
oracle's tests use: it draws initial states and holds none of the solver's
arithmetic (no derivative, no right-hand side, no time step).

States are float64 arrays shaped ``(nfields, nz, ny, nx)`` with fields
(lnrho, u_x, u_y, u_z[, s]); grid point i sits at x_i = i L / N.

Recipes (the paper's performance runs use no dataset; its physics tests fix
only the shear wave and the explosion shell):

* ``sine_modes``: a sum of 8 distinct integer wave vectors drawn uniformly
  from 1 <= |k| <= kmax, each with a uniform random phase, amplitude `amp`
  per mode.  Used for the 32^3 FP64 parity case (lnrho and each velocity
  component get their own 8 modes).
* ``spectrum``: complex Gaussian Fourier amplitudes on the shell
  k1 <= |k| <= k2 with |a_k| ~ |k|^((p-2)/2), so the shell-summed energy
  goes as k^p; inverse real FFT; velocity scaled so rms |u| = Mach c_s,
  density perturbation at p = -2 scaled to the given rms, zero mean.
* ``shear_wave``: u = u0 sin(k x) e_y, lnrho = 0 (the paper's viscous decay
  test, Sect. 6).
* ``explosion``: radial Gaussian velocity shell, u = u_ampl exp(-(r - r_s)^2
  / (2 d^2)) e_r about the box centre (Sect. 6; the printed exponent lacks
  its minus sign).
* ``forcing_sequence``: the random draws of the non-helical forcing (Sect.
  6): per time step an integer wave vector picked uniformly from the
  isotropic set of all integer vectors with kmin <= |k| <= kmax, a phase
  uniform in [0, 2 pi), and a unit vector e perpendicular to k (uniform
  direction in that plane).  Only the draws live here; the forcing itself
  (N, f_k, the field) is computed by the solver and the oracle.
"""
import os

import numpy as np
import scipy.fft

TWO_PI = 2.0 * np.pi
_WORKERS = os.cpu_count() or 1


def coords(n, length):
    return np.arange(n, dtype=np.float64) * (length / n)


def _empty_state(shape, nfields):
    return np.zeros((nfields,) + tuple(shape), dtype=np.float64)


def _integer_vectors(kmax):
    r = int(np.floor(kmax))
    ks = []
    for kz in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kx in range(-r, r + 1):
                m2 = kx * kx + ky * ky + kz * kz
                if 1 <= m2 <= kmax * kmax:
                    ks.append((kx, ky, kz))
    return np.array(ks, dtype=np.int64)


def sine_field(rng, shape, lengths, nmodes=8, kmax=4.0, amp=0.01):
    """amp * sum_m sin(k_m . x + phi_m) over nmodes distinct integer k_m."""
    nz, ny, nx = shape
    lx, ly, lz = lengths
    pool = _integer_vectors(kmax)
    pick = rng.choice(len(pool), size=nmodes, replace=False)
    phases = rng.uniform(0.0, TWO_PI, size=nmodes)
    z = coords(nz, lz)[:, None, None]
    y = coords(ny, ly)[None, :, None]
    x = coords(nx, lx)[None, None, :]
    out = np.zeros(shape)
    for (kx, ky, kz), ph in zip(pool[pick], phases):
        arg = (TWO_PI / lx) * kx * x + (TWO_PI / ly) * ky * y + (TWO_PI / lz) * kz * z + ph
        out += np.sin(arg)
    return amp * out


def sine_modes(shape, seed, lengths=(TWO_PI,) * 3, lnrho_amp=0.01, u_amp=0.01, nmodes=8,
               kmax=4.0, nfields=5):
    """lnrho = lnrho_amp * (8 modes), each u_i = u_amp per mode (8 modes), s = 0."""
    rng = np.random.default_rng(seed)
    st = _empty_state(shape, nfields)
    st[0] = sine_field(rng, shape, lengths, nmodes, kmax, lnrho_amp)
    for i in range(3):
        st[1 + i] = sine_field(rng, shape, lengths, nmodes, kmax, u_amp)
    return st


def _shell_field(rng, shape, p, k1, k2):
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz, 1.0 / nz)[:, None, None]
    ky = np.fft.fftfreq(ny, 1.0 / ny)[None, :, None]
    kx = np.fft.rfftfreq(nx, 1.0 / nx)[None, None, :]
    kk = np.sqrt(kx * kx + ky * ky + kz * kz)
    rshape = (nz, ny, nx // 2 + 1)
    re = rng.standard_normal(rshape)
    im = rng.standard_normal(rshape)
    shell = (kk >= k1) & (kk <= k2)
    amp = np.zeros(rshape)
    amp[shell] = kk[shell] ** ((p - 2.0) / 2.0)
    return scipy.fft.irfftn((re + 1j * im) * amp, s=shape, axes=(0, 1, 2), workers=_WORKERS)


def spectrum(shape, seed, p=-2.0, k1=1.0, k2=8.0, mach=0.1, cs=1.0, lnrho_rms=1e-3,
             nfields=5):
    """Velocity with shell energy ~ k^p over k1..k2 and rms|u| = mach*cs;
    lnrho perturbation at p = -2 over the same shell, rms lnrho_rms, mean 0."""
    rng = np.random.default_rng(seed)
    st = _empty_state(shape, nfields)
    for i in range(3):
        st[1 + i] = _shell_field(rng, shape, p, k1, k2)
    urms = np.sqrt(np.mean(st[1] ** 2 + st[2] ** 2 + st[3] ** 2))
    st[1:4] *= (mach * cs) / urms
    ln = _shell_field(rng, shape, -2.0, k1, k2)
    ln -= ln.mean()
    st[0] = ln * (lnrho_rms / np.sqrt(np.mean(ln * ln)))
    return st


def shear_wave(shape, k, u0, lengths=(TWO_PI,) * 3, nfields=5):
    """u = u0 sin(k x) e_y, lnrho = 0, s = 0."""
    nz, ny, nx = shape
    st = _empty_state(shape, nfields)
    x = coords(nx, lengths[0])
    st[2] = u0 * np.sin(k * x)[None, None, :]
    return st


def explosion(shape, u_ampl=1.0, d_shell=0.2, r_shell=0.8, lengths=(TWO_PI,) * 3, nfields=5):
    """Radial Gaussian velocity shell about the box centre, lnrho = 0."""
    nz, ny, nx = shape
    lx, ly, lz = lengths
    z = coords(nz, lz)[:, None, None] - lz / 2
    y = coords(ny, ly)[None, :, None] - ly / 2
    x = coords(nx, lx)[None, None, :] - lx / 2
    r = np.sqrt(x * x + y * y + z * z)
    prof = u_ampl * np.exp(-((r - r_shell) ** 2) / (2.0 * d_shell ** 2))
    rs = np.where(r > 0, r, 1.0)
    st = _empty_state(shape, nfields)
    st[1] = prof * x / rs
    st[2] = prof * y / rs
    st[3] = prof * z / rs
    return st


def random_state(shape, seed, scale=0.05, nfields=5):
    """Plain seeded normal noise on every field (edge-case parity inputs)."""
    rng = np.random.default_rng(seed)
    return scale * rng.standard_normal((nfields,) + tuple(shape))


def forcing_set(kmin, kmax):
    """All integer wave vectors with kmin <= |k| <= kmax (isotropic set)."""
    r = int(np.floor(kmax))
    ks = []
    for kz in range(-r, r + 1):
        for ky in range(-r, r + 1):
            for kx in range(-r, r + 1):
                m2 = kx * kx + ky * ky + kz * kz
                if kmin * kmin <= m2 <= kmax * kmax and m2 > 0:
                    ks.append((kx, ky, kz))
    return np.array(ks, dtype=np.int64)


def forcing_sequence(seed, nsteps, kmin=1.0, kmax=2.0):
    """(k[nsteps, 3] int, phi[nsteps], e[nsteps, 3]) for `nsteps` forced steps."""
    rng = np.random.default_rng(seed)
    pool = forcing_set(kmin, kmax)
    ks = pool[rng.integers(0, len(pool), size=nsteps)]
    phis = rng.uniform(0.0, TWO_PI, size=nsteps)
    es = np.zeros((nsteps, 3))
    for i in range(nsteps):
        kh = ks[i] / np.linalg.norm(ks[i])
        while True:
            v = rng.standard_normal(3)
            v -= np.dot(v, kh) * kh
            nv = np.linalg.norm(v)
            if nv > 1e-3:
                es[i] = v / nv
                break
    return ks, phis, es
