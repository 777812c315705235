"""GPU tests of the paper's physics test cases (Sect. 6) through the C ABI:
the forced steps (Eqs. 20-21) and the radial explosion (Eq. 19) against the
FP64 oracle.  Bars as in the unforced parity tests: FP64 relative L2 <= 1e-12
per field; FP32 forms <= 1e-5 per step from the FP32-rounded state."""
import numpy as np
import pytest

from oracle import fd
from paper_1707_08900_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FP64_TOL = 1e-12
FP32_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1707_08900_gb300 import build
    build.build()


def _rel(got, ref):
    out = []
    for g, o in zip(got, ref):
        no = np.linalg.norm(o.ravel())
        d = np.linalg.norm((g - o).ravel())
        out.append(d / no if no > 0 else d)
    return np.array(out)


CASES = [("fp64", "55p", 0), ("fp64", "19p", 0), ("fp64", "55p", 1), ("fp32", "55p", 0),
         ("fp32", "19p", 0), ("fp32", "55p", 1), ("fp32_acc64", "55p", 0),
         ("fp32_acc64_w64", "19p", 0)]


@pytest.mark.parametrize("precision,form,path", CASES)
def test_forced_steps_match_oracle(precision, form, path):
    """Three forced steps, each with its own k, phi and e, on a ragged
    non-cubic box (tiled path 0, simple path 1)."""
    from paper_1707_08900_gb300 import gbfd
    shape = (20, 44, 36)
    lengths = (2 * np.pi, 5.0, 4.0)  # (lx, ly, lz)
    g = fd.Grid(shape[2], shape[1], shape[0], *lengths)
    ph = fd.Physics(cs=1.0, nu=0.01, entropy_mode=1)
    st = inputs.spectrum(shape, 31, mach=0.1, lnrho_rms=1e-2)
    if precision != "fp64":
        st = st.astype(np.float32).astype(np.float64)
    ks, phis, es = inputs.forcing_sequence(7, 3, kmin=1.0, kmax=3.0)
    dt, f0 = 0.01, 0.05
    ref = fd.rk3_step_forced(st, dt, g, ph, f0, ks, phis, es,
                             form=fd.FORM_55P if form == "55p" else fd.FORM_19P)
    s = gbfd.Solver(shape, lengths=lengths, nu=0.01, precision=precision, form=form)
    if path:
        s.set_option(gbfd.GBFD_OPT_KERNEL_PATH, 1)
    s.set_state(st)
    s.rk3_step_forced(dt, f0, ks, phis, es)
    got = s.get_state()
    s.close()
    # the forcing must have acted: the forced and unforced oracle steps differ
    base = fd.rk3_step(st, dt, g, ph, form=fd.FORM_55P if form == "55p" else fd.FORM_19P,
                       nsteps=3)
    assert np.linalg.norm((ref[1:4] - base[1:4]).ravel()) > 1e-3 * np.linalg.norm(base[1:4].ravel())
    tol = FP64_TOL if precision == "fp64" else 3 * FP32_TOL
    err = _rel(got, ref)
    assert np.all(err[:4] <= tol), err


@pytest.mark.parametrize("form", ["55p", "19p"])
def test_forced_fp32_steps_on_whole_tiles_match_oracle(form):
    """Forced FP32 steps where the kernels run their per-substep
    instantiations with the forcing compiled in (whole 32 x 8 tiles, equal
    spacing on every axis: the default 55-point kernel, the 19-point form's
    first pass): one forced step on the term-exposing state within the FP32
    bars (relative L2 and the element-wise increment bar), then three steps
    with new k, phi and e each within 3 x the per-step bar."""
    fm = fd.FORM_55P if form == "55p" else fd.FORM_19P
    from bars import inc_bar, inc_err, max_abs, term_exposing_state
    from paper_1707_08900_gb300 import gbfd
    shape = (24, 16, 64)  # (nz, ny, nx)
    h = 2 * np.pi / 64
    lengths = (64 * h, 16 * h, 24 * h)  # (lx, ly, lz)
    g = fd.Grid(shape[2], shape[1], shape[0], *lengths)
    nu = 0.02
    ph = fd.Physics(cs=1.0, nu=nu, entropy_mode=1)
    st = term_exposing_state(shape, 17, inputs)
    ks, phis, es = inputs.forcing_sequence(11, 3, kmin=1.0, kmax=3.0)
    dt, f0 = fd.cfl_dt(st, g, ph, 0.4), 0.2
    s = gbfd.Solver(shape, lengths=lengths, nu=nu, precision="fp32", form=form)
    s.set_state(st)
    s.rk3_step_forced(dt, f0, ks[:1], phis[:1], es[:1])
    got = s.get_state()
    ref = fd.rk3_step_forced(st, dt, g, ph, f0, ks[:1], phis[:1], es[:1], form=fm)
    base = fd.rk3_step(st, dt, g, ph, form=fm)
    # the forcing must have acted on this step
    assert np.linalg.norm((ref[1:4] - base[1:4]).ravel()) > 1e-2 * np.linalg.norm(
        (base[1:4] - st[1:4]).ravel())
    err, inc, bar = _rel(got, ref), inc_err(got, ref, st), inc_bar(ref, st)
    print(f"{form} one forced step: relL2 {err} inc {inc} bar {bar} maxabs {max_abs(got, ref)}")
    assert np.all(err <= FP32_TOL), err
    assert np.all(inc <= bar), (inc, bar)
    s.set_state(st)
    s.rk3_step_forced(dt, f0, ks, phis, es)
    got3 = s.get_state()
    s.close()
    ref3 = fd.rk3_step_forced(st, dt, g, ph, f0, ks, phis, es, form=fm)
    err3 = _rel(got3, ref3)
    assert np.all(err3 <= 3 * FP32_TOL), err3


def test_every_fp32_tile_entry_runs_forced_on_the_default_kernel():
    from paper_1707_08900_gb300 import gbfd
    shape = (16, 24, 32)
    st = inputs.spectrum(shape, 8, mach=0.2, lnrho_rms=1e-2).astype(np.float32)
    ks, phis, es = inputs.forcing_sequence(9, 2)
    outs = []
    for cfg in (-1, 0, 5, 10, 15):
        s = gbfd.Solver(shape, precision="fp32", nu=5e-3)
        s.set_option(gbfd.GBFD_OPT_TILE_CONFIG, cfg)
        s.set_state(st)
        s.rk3_step_forced(0.01, 0.1, ks, phis, es)
        outs.append(s.get_state(fp64=False))
        s.close()
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


def test_zero_amplitude_is_the_unforced_step_and_bad_args():
    from paper_1707_08900_gb300 import gbfd
    shape = (16, 16, 16)
    st = inputs.spectrum(shape, 2, mach=0.2, lnrho_rms=1e-2)
    ks, phis, es = inputs.forcing_sequence(3, 2)
    a = gbfd.Solver(shape, precision="fp64")
    b = gbfd.Solver(shape, precision="fp64")
    a.set_state(st)
    b.set_state(st)
    a.rk3_step_forced(0.01, 0.0, ks, phis, es)
    b.rk3_step(0.01, 2)
    assert np.array_equal(a.get_state(), b.get_state())
    with pytest.raises(gbfd.GbfdError):
        a.rk3_step_forced(0.01, 0.1, [[0, 0, 0]], [0.0], [[1.0, 0.0, 0.0]])
    with pytest.raises(gbfd.GbfdError):
        a.rk3_step_forced(0.01, 0.1, [[0, 0, 2]], [0.0], [[0.0, 0.0, 1.0]])
    with pytest.raises(gbfd.GbfdError):
        a.rk3_step_forced(-0.01, 0.1, ks, phis, es)
    a.close()
    b.close()


@pytest.mark.parametrize("precision,form", [("fp64", "55p"), ("fp64", "19p"), ("fp32", "55p")])
def test_explosion_on_the_gpu(precision, form):
    """The explosion test (Sect. 6, Eq. 19): the GPU run matches the oracle
    and keeps the x/y/z and the diagonal integrals equal among themselves."""
    from paper_1707_08900_gb300 import explosion, gbfd
    n = 32
    g = fd.Grid(n, n, n)
    ph = fd.Physics(cs=1.0, nu=5e-3, entropy_mode=1)
    st = inputs.explosion((n, n, n))
    if precision != "fp64":
        st = st.astype(np.float32).astype(np.float64)
    dt = fd.cfl_dt(st, g, ph, 0.4)
    frm = fd.FORM_55P if form == "55p" else fd.FORM_19P
    ref = fd.rk3_step(st, dt, g, ph, form=frm, nsteps=12)
    s = gbfd.Solver((n, n, n), precision=precision, form=form, nu=5e-3)
    s.set_state(st)
    s.rk3_step(dt, 12)
    got = s.get_state()
    s.close()
    tol = FP64_TOL if precision == "fp64" else 12 * FP32_TOL
    assert np.all(_rel(got, ref)[:4] <= tol)
    sym = 1e-12 if precision == "fp64" else 1e-5
    for v in explosion.axis_integrals(got):
        scale = np.abs(v).max()
        assert np.ptp(v[:3]) <= sym * scale and np.ptp(v[3:]) <= sym * scale, v
    np.testing.assert_allclose(explosion.asymmetry(got), explosion.asymmetry(ref),
                               rtol=1e-3 if precision == "fp32" else 1e-9)
