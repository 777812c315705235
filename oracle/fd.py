"""ctypes wrapper around the C oracle ``fd_oracle.c`` (test infrastructure).

Arrays are NumPy float64, C-contiguous.  A state is shaped
``(nfields, nz, ny, nx)`` with fields (lnrho, u_x, u_y, u_z[, s]); nfields is
4 (the paper's isothermal model, entropy_mode 0) or 5 (passive entropy s,
entropy_mode 1).  Every routine follows one definition of the paper; see the
header of ``fd_oracle.c`` for the list.
"""
import ctypes
from dataclasses import dataclass

import numpy as np

from . import build_oracle

_lib = None
_D = ctypes.c_double
_L = ctypes.c_long
_I = ctypes.c_int
_P = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = build_oracle.build()
        L = ctypes.CDLL(path)
        L.or_d1_point.restype = _D
        L.or_d1_point.argtypes = [_P, _D]
        L.or_d2_point.restype = _D
        L.or_d2_point.argtypes = [_P, _D]
        L.or_dmix_point.restype = _D
        L.or_dmix_point.argtypes = [_P, _D, _D]
        for name in ("or_grid_d1", "or_grid_d2"):
            getattr(L, name).argtypes = [_P, _P, _L, _L, _L, _D, _D, _D, _I]
        L.or_grid_dmix.argtypes = [_P, _P, _L, _L, _L, _D, _D, _D, _I, _I]
        L.or_rhs.argtypes = [_P, _P, _L, _L, _L, _D, _D, _D, _D, _D, _I, _I]
        L.or_rk3_coefficients.argtypes = [_P, _P]
        L.or_substep55.argtypes = [_P, _P, _P, _I, _D, _L, _L, _L, _D, _D, _D, _D, _D, _I]
        L.or_substep19.argtypes = [_P, _P, _P, _P, _I, _D, _L, _L, _L, _D, _D, _D, _D, _D, _I]
        L.or_substep55_wall.argtypes = L.or_substep55.argtypes
        L.or_substep19_wall.argtypes = L.or_substep19.argtypes
        L.or_substep55_slab.argtypes = L.or_substep55.argtypes
        L.or_fill_ghosts_z.argtypes = [_P, _L, _L, _L, _I, _P]
        L.or_diagnostics.argtypes = [_P, _L, _L, _L, _D, _D, _D, _I, _P]
        L.or_cfl_dt.restype = _D
        L.or_cfl_dt.argtypes = [_P, _L, _L, _L, _D, _D, _D, _D, _D, _D, _D]
        L.or_box_filter.argtypes = [_P, _P, _L, _L, _L, _I, _I]
        L.or_set_threads.restype = _I
        L.or_set_threads.argtypes = [_I]
        _LP = ctypes.POINTER(ctypes.c_long)
        L.or_forcing_amplitude.restype = _I
        L.or_forcing_amplitude.argtypes = [_LP, _P, _D, _D, _D, _D, _D, _D, _P]
        L.or_rhs_forced.restype = _I
        L.or_rhs_forced.argtypes = [_P, _P, _L, _L, _L, _D, _D, _D, _D, _D, _I, _I, _D, _D, _LP,
                                    _D, _P]
        L.or_substep_forced.restype = _I
        L.or_substep_forced.argtypes = [_P, _P, _P, _P, _I, _D, _I, _L, _L, _L, _D, _D, _D, _D,
                                        _D, _I, _D, _LP, _D, _P]
        _lib = L
    return _lib


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_P)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n):
    """Set the OpenMP thread count of the substep loops; returns the count."""
    return lib().or_set_threads(int(n))


# ---------------------------------------------------------------- stencils

def d1_point(samples, h):
    """Eq. 6 applied to 7 samples at offsets -3..3."""
    s = _f64(samples)
    assert s.shape == (7,)
    return lib().or_d1_point(_p(s), h)


def d2_point(samples, h):
    """Eq. 7 (with 1/(180 h^2)) applied to 7 samples at offsets -3..3."""
    s = _f64(samples)
    assert s.shape == (7,)
    return lib().or_d2_point(_p(s), h)


def dmix_point(patch, ha, hb):
    """Eq. 8 applied to a 7x7 patch, patch[ia+3, ib+3] = f(a+ia ha, b+ib hb)."""
    s = _f64(patch)
    assert s.shape == (7, 7)
    return lib().or_dmix_point(_p(s), ha, hb)


@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    lx: float = 2 * np.pi
    ly: float = 2 * np.pi
    lz: float = 2 * np.pi

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def spacing(self):
        return (self.lx / self.nx, self.ly / self.ny, self.lz / self.nz)

    def dims(self):
        return (self.nx, self.ny, self.nz, self.lx, self.ly, self.lz)


def grid_d1(f, grid, axis):
    f = _f64(f)
    out = np.empty_like(f)
    lib().or_grid_d1(_p(f), _p(out), *grid.dims(), axis)
    return out


def grid_d2(f, grid, axis):
    f = _f64(f)
    out = np.empty_like(f)
    lib().or_grid_d2(_p(f), _p(out), *grid.dims(), axis)
    return out


def grid_dmix(f, grid, a, b):
    f = _f64(f)
    out = np.empty_like(f)
    lib().or_grid_dmix(_p(f), _p(out), *grid.dims(), a, b)
    return out


# ---------------------------------------------------------------- physics

@dataclass
class Physics:
    cs: float = 1.0
    nu: float = 5e-3
    entropy_mode: int = 1

    @property
    def nfields(self):
        return 5 if self.entropy_mode else 4


FORM_55P = 0
FORM_19P = 1


def rhs(state, grid, phys, form=FORM_55P):
    """d(state)/dt from Eqs. 1-3 (f = 0) in the given stencil form."""
    st = _f64(state)
    assert st.shape == (phys.nfields,) + grid.shape
    out = np.zeros_like(st)
    lib().or_rhs(_p(st), _p(out), *grid.dims(), phys.cs, phys.nu, phys.entropy_mode, form)
    return out


def rk3_coefficients():
    a = np.zeros(3)
    b = np.zeros(3)
    lib().or_rk3_coefficients(_p(a), _p(b))
    return a, b


def substep(state_in, w, s, dt, grid, phys, form=FORM_55P):
    """One RK3 substep (s = 0, 1, 2).  Returns (state_out, w_new)."""
    st = _f64(state_in).copy()
    wn = _f64(w).copy()
    out = np.zeros_like(st)
    if form == FORM_55P:
        lib().or_substep55(_p(st), _p(wn), _p(out), s, dt, *grid.dims(), phys.cs, phys.nu,
                           phys.entropy_mode)
    else:
        divf = np.zeros(grid.shape)
        lib().or_substep19(_p(st), _p(wn), _p(out), _p(divf), s, dt, *grid.dims(), phys.cs,
                           phys.nu, phys.entropy_mode)
    return out, wn


def rk3_step(state, dt, grid, phys, form=FORM_55P, nsteps=1):
    """Advance `nsteps` full RK3 steps of length dt; returns the new state."""
    st = _f64(state).copy()
    w = np.zeros_like(st)
    for _ in range(nsteps):
        for s in range(3):
            st, w = substep(st, w, s, dt, grid, phys, form)
    return st


# ---------------------------------------------------------------- walls in z

# Parity of each field under the mirror about a wall point (lnrho, u_x,
# u_y, u_z, s): an impermeable, free-slip wall keeps u_z odd, the rest even.
WALL_PARITY = (1.0, 1.0, 1.0, -1.0, 1.0)
GZ_WALL = 3


def fill_ghosts_z(ext, parity=WALL_PARITY):
    """Fill the ghost planes of a ghost-extended state (nf, nz + 6, ny, nx) in
    place: mirror images about the walls at interior planes 0 and nz - 1."""
    assert ext.dtype == np.float64 and ext.flags.c_contiguous
    nf, nzt, ny, nx = ext.shape
    par = _f64(np.asarray(parity[:nf], dtype=np.float64))
    lib().or_fill_ghosts_z(_p(ext), nx, ny, nzt - 2 * GZ_WALL, nf, _p(par))
    return ext


def extend_wall(state):
    """Interior state (nf, nz, ny, nx) -> ghost-extended copy with ghosts filled."""
    st = _f64(state)
    nf, nz, ny, nx = st.shape
    ext = np.zeros((nf, nz + 2 * GZ_WALL, ny, nx))
    ext[:, GZ_WALL:GZ_WALL + nz] = st
    return fill_ghosts_z(ext)


def interior_wall(ext):
    return np.ascontiguousarray(ext[:, GZ_WALL:ext.shape[1] - GZ_WALL])


def wall_spacing(grid):
    """Grid spacing with walls through z = 0 and z = lz: lz / (nz - 1) in z."""
    return (grid.lx / grid.nx, grid.ly / grid.ny, grid.lz / (grid.nz - 1))


def substep_wall(ext_in, w, s, dt, grid, phys, form=FORM_55P):
    """One RK3 substep with walls in z on ghost-extended arrays (ghosts of
    ext_in filled).  Returns (ext_out with its ghosts filled, w_new)."""
    st = _f64(ext_in)
    wn = _f64(w).copy()
    out = np.zeros_like(st)
    if form == FORM_55P:
        lib().or_substep55_wall(_p(st), _p(wn), _p(out), s, dt, *grid.dims(), phys.cs, phys.nu,
                                phys.entropy_mode)
    else:
        divf = np.zeros((1,) + st.shape[1:])
        lib().or_substep19_wall(_p(st), _p(wn), _p(out), _p(divf), s, dt, *grid.dims(),
                                phys.cs, phys.nu, phys.entropy_mode)
    return fill_ghosts_z(out), wn


def rk3_step_wall(state, dt, grid, phys, form=FORM_55P, nsteps=1):
    """`nsteps` RK3 steps with walls in z (Algorithm 1: boundary step, then
    each substep); interior state in and out."""
    ext = extend_wall(state)
    w = np.zeros_like(ext)
    for _ in range(nsteps):
        for s in range(3):
            ext, w = substep_wall(ext, w, s, dt, grid, phys, form)
    return interior_wall(ext)


def substep_slab(ext_in, w, s, dt, grid, phys):
    """One 55-point substep on a z-slab (ghost-extended arrays, nz + 6
    planes, ghosts filled by the caller from the neighbouring slabs); `grid`
    is the slab's (nz interior planes, lz = nz x the z spacing).  Returns
    (ext_out with its interior written and its ghost planes zero, w_new)."""
    st = _f64(ext_in)
    wn = _f64(w).copy()
    out = np.zeros_like(st)
    lib().or_substep55_slab(_p(st), _p(wn), _p(out), s, dt, *grid.dims(), phys.cs, phys.nu,
                            phys.entropy_mode)
    return out, wn


def cfl_dt_wall(state, grid, phys, cfl=0.4, cnu=0.25):
    """The dt rule on the wall grid (z spacing lz / (nz - 1))."""
    st = _f64(state)
    lz_eff = grid.lz * grid.nz / (grid.nz - 1)  # so that the routine's lz / nz is the spacing
    return lib().or_cfl_dt(_p(st), grid.nx, grid.ny, grid.nz, grid.lx, grid.ly, lz_eff,
                           phys.cs, phys.nu, cfl, cnu)


def diagnostics(state, grid, phys):
    """FP64 reductions of a state (see ``or_diagnostics``)."""
    st = _f64(state)
    out = np.zeros(15)
    lib().or_diagnostics(_p(st), *grid.dims(), phys.entropy_mode, out.ctypes.data_as(_P))
    return {
        "mass": out[0], "ekin": out[1], "umax": out[2], "urms": out[3],
        "rms": out[4:9].copy(), "maxabs": out[9:14].copy(), "nonfinite": int(out[14]),
    }


def cfl_dt(state, grid, phys, cfl=0.4, cnu=0.25):
    st = _f64(state)
    return lib().or_cfl_dt(_p(st), *grid.dims(), phys.cs, phys.nu, cfl, cnu)


def box_filter(fine, r=4):
    """Centred box filter to a grid r times coarser per axis (fields first)."""
    f = _f64(fine)
    nf, nz, ny, nx = f.shape
    out = np.zeros((nf, nz // r, ny // r, nx // r))
    lib().or_box_filter(_p(f), _p(out), nx, ny, nz, r, nf)
    return out


# ---------------------------------------------------------------- forcing

def _kvec(k):
    a = np.ascontiguousarray(np.asarray(k, dtype=np.int64).reshape(3), dtype=ctypes.c_long)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def forcing_amplitude(k, e, f0, cs, dt, lengths=(2 * np.pi,) * 3):
    """N f_k of Eq. 21 for integer wave vector k (physical k_i = 2 pi k_i / L_i)
    and unit vector e (Sect. 6)."""
    ka, kp = _kvec(k)
    ev = _f64(np.asarray(e, dtype=np.float64).reshape(3))
    out = np.zeros(3)
    if lib().or_forcing_amplitude(kp, _p(ev), f0, cs, dt, *lengths, _p(out)):
        raise ValueError("f_k undefined: k is zero or parallel to e")
    return out


def rhs_forced(state, grid, phys, dt, f0, k, phi, e, form=FORM_55P):
    """d(state)/dt of Eqs. 1-3 with the forcing of Eqs. 20-21 for one step."""
    st = _f64(state)
    out = np.zeros_like(st)
    ka, kp = _kvec(k)
    ev = _f64(np.asarray(e, dtype=np.float64).reshape(3))
    if lib().or_rhs_forced(_p(st), _p(out), *grid.dims()[:6], phys.cs, phys.nu,
                           phys.entropy_mode, form, dt, f0, kp, phi, _p(ev)):
        raise ValueError("f_k undefined")
    return out


def rk3_step_forced(state, dt, grid, phys, f0, ks, phis, es, form=FORM_55P):
    """len(phis) RK3 steps; step i is forced with ks[i], phis[i], es[i]."""
    st = _f64(state).copy()
    w = np.zeros_like(st)
    divf = np.zeros(grid.shape)
    for i in range(len(phis)):
        ka, kp = _kvec(ks[i])
        ev = _f64(np.asarray(es[i], dtype=np.float64).reshape(3))
        for s in range(3):
            out = np.zeros_like(st)
            if lib().or_substep_forced(_p(st), _p(w), _p(out), _p(divf), s, dt, form,
                                       *grid.dims()[:6], phys.cs, phys.nu, phys.entropy_mode,
                                       f0, kp, float(phis[i]), _p(ev)):
                raise ValueError("f_k undefined")
            st = out
    return st
