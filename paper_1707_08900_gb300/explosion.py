"""Radial kinetic explosion and its spherical-symmetry measure (Sect. 6,
Eq. 19; the paper's second physics test).

The initial velocity is a Gaussian shell directed radially outward from the
box centre (``inputs.explosion``).  The symmetry measure compares seven
axes through the centre: x, y, z and the four body diagonals.  Along each
axis the excess density (rho - 1, rho = exp(lnrho)) and the speed |u| are
integrated over a common radius |s| <= r_max (the sample spacing is the grid
spacing along x, y, z and sqrt(3) times it along a diagonal), so the
background and the different axis lengths drop out; Delta is the standard
deviation of the seven integrals divided by their mean.

Readings (the paper gives neither a formula nor c_s or the run length):
"integrated the sum of values of each axis" is the integral above; Re =
u_ampl d_shell / nu; c_s = 1 and t = 0.5.  With u_ampl = c_s = 1 the shell
is sonic; its inward half collapses on the centre and, on these grids and
viscosities, the central scheme (no shock capturing) loses the solution
near t = 0.8-1.0, so the measure is taken before that.

    python -m paper_1707_08900_gb300.explosion --n 128 --form 55p --nu 1e-3 --t 0.5
"""
import argparse
import json

import numpy as np

from . import inputs

AXES = ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 1), (1, 1, -1), (1, -1, 1), (-1, 1, 1))


def axis_integrals(state, lengths=(2 * np.pi,) * 3, r_max=None):
    """(7,) integrals of rho - 1 and of |u| along the seven axes through the
    centre of a cubic grid (state (nf, n, n, n), fields lnrho, u_x, u_y, u_z)."""
    nf, nz, ny, nx = state.shape
    assert nx == ny == nz and nx % 2 == 0, "cubic grid with a centre point"
    n = nx
    h = lengths[0] / n
    assert np.allclose(lengths, lengths[0])
    c = n // 2
    r_max = r_max if r_max is not None else 0.45 * lengths[0]
    with np.errstate(over="ignore", invalid="ignore"):
        rho1 = np.expm1(state[0])
    speed = np.sqrt(state[1] ** 2 + state[2] ** 2 + state[3] ** 2)
    out_rho, out_u = np.zeros(7), np.zeros(7)
    for a, (dx, dy, dz) in enumerate(AXES):
        step = h * np.sqrt(dx * dx + dy * dy + dz * dz)
        m = int(np.floor(r_max / step))
        idx = np.arange(-m, m + 1)
        xs, ys, zs = (c + dx * idx) % n, (c + dy * idx) % n, (c + dz * idx) % n
        out_rho[a] = rho1[zs, ys, xs].sum() * step
        out_u[a] = speed[zs, ys, xs].sum() * step
    return out_rho, out_u


def asymmetry(state, lengths=(2 * np.pi,) * 3, r_max=None):
    """(Delta(sum rho), Delta(sum |u|)): std / |mean| of the seven integrals."""
    ir, iu = axis_integrals(state, lengths, r_max)
    rel = lambda v: float(np.std(v) / max(abs(np.mean(v)), 1e-300))
    return rel(ir), rel(iu)


def reynolds(nu, u_ampl=1.0, d_shell=0.2):
    return u_ampl * d_shell / nu


def run(n=128, nu=1e-3, t_end=0.5, precision="fp32", form="55p", cfl=0.4, samples=5):
    """GPU run of the explosion to t_end; Delta at `samples` times."""
    import torch  # noqa: F401
    from . import gbfd
    st = inputs.explosion((n, n, n))
    s = gbfd.Solver((n, n, n), precision=precision, form=form, nu=nu)
    s.set_state(st if precision == "fp64" else st.astype(np.float32))
    dt = s.cfl_dt(cfl)
    nsteps = int(np.ceil(t_end / dt))
    dt = t_end / nsteps
    marks = sorted(set(int(round(nsteps * (i + 1) / samples)) for i in range(samples)))
    done, hist = 0, []
    for mk in marks:
        s.rk3_step(dt, mk - done)
        done = mk
        dr, du = asymmetry(s.get_state())
        hist.append({"t": done * dt, "delta_rho": dr, "delta_u": du})
    s.close()
    return {"n": n, "nu": nu, "Re": reynolds(nu), "precision": precision, "form": form,
            "dt": dt, "steps": nsteps, "history": hist}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--nu", type=float, nargs="+", default=[4e-3, 2e-3, 1e-3, 5e-4])
    ap.add_argument("--t", type=float, default=0.5)
    ap.add_argument("--precision", default="fp32")
    ap.add_argument("--form", default="55p")
    a = ap.parse_args()
    from . import build
    build.build()
    for nu in a.nu:
        print(json.dumps(run(a.n, nu, a.t, a.precision, a.form)))


if __name__ == "__main__":
    main()
