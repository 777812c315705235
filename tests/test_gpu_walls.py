"""GPU parity of the wall variant (z bounded by free-slip, impermeable walls
through the first and last planes; ghost planes filled as parity mirrors
after every substep, Sect. 4 / Algorithm 1's boundary step) against the
oracle's wall variant, through the C ABI.  Bars as in the periodic tests
(tests/bars.py)."""
import numpy as np
import pytest

from bars import FP32_TOL, FP64_TOL, TERM_NU, inc_bar, inc_err, max_abs, rel_l2
from oracle import fd
from paper_1707_08900_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1707_08900_gb300 import build
    build.build()


def wall_state(shape, seed, nf=5, amp=0.05):
    """Smooth random state with u_z = 0 on both walls: even fields from
    cosines in z, u_z from sines (z / Lz in [0, 1] over the nz planes)."""
    nz, ny, nx = shape
    rng = np.random.default_rng(seed)
    z = np.arange(nz) * np.pi / (nz - 1)
    y = np.arange(ny) * 2 * np.pi / ny
    x = np.arange(nx) * 2 * np.pi / nx
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    st = np.zeros((nf,) + shape)
    for f in range(nf):
        for _ in range(8):
            m, ky, kx = rng.integers(0, 6), rng.integers(0, 4), rng.integers(0, 4)
            a = (0.4 if f == 0 else 1.0) * amp * rng.standard_normal()
            zf = np.sin(m * Z) if f == 3 else np.cos(m * Z)
            st[f] += a * zf * np.cos(ky * Y + kx * X + rng.uniform(0, 2 * np.pi))
    return st


def _solver(shape, **kw):
    from paper_1707_08900_gb300 import gbfd
    return gbfd.Solver(shape, bc_z="wall", **kw)


@pytest.mark.parametrize("form", ["55p", "19p"])
@pytest.mark.parametrize("path", [0, 1])
def test_fp64_wall_steps_match_oracle(form, path):
    """36 x 44 x 72 with unequal lengths, walls in z: partial x/y tiles, several
    z-chunks (chunk seams away from the walls), the tiled (0) and the simple
    (1) kernels, three RK3 steps."""
    from paper_1707_08900_gb300 import gbfd
    shape = (72, 44, 36)
    lengths = (3.0, 4.5, 2.5)
    nz, ny, nx = shape
    g = fd.Grid(nx, ny, nz, *lengths)
    ph = fd.Physics(cs=1.0, nu=0.02, entropy_mode=1)
    st = wall_state(shape, 4)
    ofm = fd.FORM_55P if form == "55p" else fd.FORM_19P
    s = _solver(shape, precision="fp64", form=form, nu=0.02, lengths=lengths)
    s.set_option(gbfd.GBFD_OPT_KERNEL_PATH, path)
    s.set_state(st)
    ref = st
    for _ in range(3):
        dt = fd.cfl_dt_wall(ref, g, ph, 0.4)
        ref = fd.rk3_step_wall(ref, dt, g, ph, ofm)
        s.rk3_step(dt, 1)
    got = s.get_state()
    s.close()
    err = rel_l2(got, ref)
    assert np.all(err <= FP64_TOL), err
    assert np.abs(got - st).max() > 1e-3  # the state moved


@pytest.mark.parametrize("precision", ["fp32", "fp32_acc64", "fp32_acc64_w64"])
@pytest.mark.parametrize("form", ["55p", "19p"])
def test_fp32_wall_step_elementwise(precision, form):
    """One step from the FP32-rounded state: relative L2 and the element-wise
    increment bar, on the default kernels of each precision form."""
    shape = (40, 32, 64)
    nz, ny, nx = shape
    g = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, 3.0)
    ph = fd.Physics(cs=1.0, nu=TERM_NU, entropy_mode=1)
    st = wall_state(shape, 7, amp=0.2).astype(np.float32).astype(np.float64)
    dt = fd.cfl_dt_wall(st, g, ph, 0.4)
    ref = fd.rk3_step_wall(st, dt, g, ph, fd.FORM_55P if form == "55p" else fd.FORM_19P)
    s = _solver(shape, precision=precision, form=form, nu=TERM_NU,
                lengths=(2 * np.pi, 2 * np.pi, 3.0))
    s.set_state(st.astype(np.float32))
    s.rk3_step(dt, 1)
    got = s.get_state()
    s.close()
    err, inc, bar = rel_l2(got, ref), inc_err(got, ref, st), inc_bar(ref, st)
    print(f"{precision} {form}: relL2 {err} inc {inc} bar {bar} maxabs {max_abs(got, ref)}")
    assert np.all(err <= FP32_TOL), err
    assert np.all(inc <= bar), (inc, bar)


def test_every_fp32_tile_entry_with_walls():
    """Every FP32 tile-table entry (kernels and z-chunk lengths) with walls
    against the oracle, on a grid whose z-chunks end on and away from the
    wall planes."""
    from paper_1707_08900_gb300 import gbfd
    shape = (37, 24, 32)
    nz, ny, nx = shape
    g = fd.Grid(nx, ny, nz)
    ph = fd.Physics(cs=1.0, nu=0.01, entropy_mode=1)
    st = wall_state(shape, 9, amp=0.1).astype(np.float32).astype(np.float64)
    dt = fd.cfl_dt_wall(st, g, ph, 0.4)
    ref = fd.rk3_step_wall(st, dt, g, ph)
    bar = inc_bar(ref, st)
    n = 0
    for cfg in range(256):
        s = _solver(shape, precision="fp32", nu=0.01)
        try:
            s.set_option(gbfd.GBFD_OPT_TILE_CONFIG, cfg)
        except gbfd.GbfdError:
            s.close()
            break
        s.set_state(st.astype(np.float32))
        s.rk3_step(dt, 1)
        got = s.get_state()
        s.close()
        err, inc = rel_l2(got, ref), inc_err(got, ref, st)
        assert np.all(err <= FP32_TOL), (cfg, err)
        assert np.all(inc <= bar), (cfg, inc, bar)
        n += 1
    assert n >= 20


def test_wall_run_is_the_periodic_run_of_the_mirror_extension_on_the_gpu():
    """GPU against GPU: the FP64 wall run on nz planes reproduces the
    periodic GPU run on the 2 (nz - 1) planes of the mirror-extended state."""
    shape = (24, 16, 32)
    nz, ny, nx = shape
    st = wall_state(shape, 11)
    par = np.array([1.0, 1.0, 1.0, -1.0, 1.0])
    ext = np.concatenate([st, st[:, nz - 2:0:-1] * par[:, None, None, None]], axis=1)
    from paper_1707_08900_gb300 import gbfd
    a = _solver(shape, precision="fp64", nu=0.02, lengths=(2 * np.pi, 2 * np.pi, 2.0))
    b = gbfd.Solver((2 * (nz - 1), ny, nx), precision="fp64", nu=0.02,
                    lengths=(2 * np.pi, 2 * np.pi, 4.0))
    a.set_state(st)
    b.set_state(np.ascontiguousarray(ext))
    for _ in range(3):
        a.rk3_step(0.02, 1)
        b.rk3_step(0.02, 1)
    ga, gb_ = a.get_state(), b.get_state()[:, :nz]
    a.close()
    b.close()
    err = np.abs(ga - gb_).max(axis=(1, 2, 3)) / np.abs(gb_).max(axis=(1, 2, 3))
    assert np.all(err < 1e-14), err


def test_wall_diagnostics_and_unsupported_calls():
    """Diagnostics use the wall spacing lz / (nz - 1); forcing and the network
    need a periodic box."""
    from paper_1707_08900_gb300 import gbfd
    shape = (17, 16, 16)
    nz, ny, nx = shape
    st = wall_state(shape, 2)
    s = _solver(shape, precision="fp64", lengths=(2 * np.pi, 2 * np.pi, 2.0))
    s.set_state(st)
    d = s.diagnostics()
    g_eff = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, 2.0 * nz / (nz - 1))
    o = fd.diagnostics(st, g_eff, fd.Physics())
    assert d["mass"] == pytest.approx(o["mass"], rel=1e-12)
    assert d["ekin"] == pytest.approx(o["ekin"], rel=1e-12)
    g = fd.Grid(nx, ny, nz, 2 * np.pi, 2 * np.pi, 2.0)
    assert s.cfl_dt(0.4) == pytest.approx(fd.cfl_dt_wall(st, g, fd.Physics(), 0.4), rel=1e-14)
    ks, phis, es = inputs.forcing_sequence(3, 1)
    with pytest.raises(gbfd.GbfdError) as e:
        s.rk3_step_forced(0.01, 0.1, ks, phis, es)
    assert e.value.status == 5  # GBFD_ERR_UNSUPPORTED
    s.close()
