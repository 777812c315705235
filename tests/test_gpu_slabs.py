"""Domain decomposition along z with halo exchange (Sect. 7), ranks emulated
on one GPU: a periodic box split into z-slabs, each a context with
exchanged ghost planes, must reproduce the undivided box.  Every point runs
the same arithmetic on the same values whatever slab, tile or chunk it falls
in, so the agreement is bit for bit; the FP64 run also matches the oracle."""
import numpy as np
import pytest

from bars import FP64_TOL, rel_l2
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


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("path", [0, 1])
def test_slabs_reproduce_the_undivided_box(precision, nslabs, path):
    from paper_1707_08900_gb300 import gbfd, slabs
    shape = (50, 24, 32)
    lengths = (2 * np.pi, 3.0, 4.0)
    st = inputs.spectrum(shape, 3, mach=0.3, lnrho_rms=0.05)
    if precision == "fp32":
        st = st.astype(np.float32).astype(np.float64)
    one = gbfd.Solver(shape, lengths=lengths, precision=precision, nu=0.02)
    one.set_option(gbfd.GBFD_OPT_KERNEL_PATH, path)
    one.set_state(st)
    dt = one.cfl_dt(0.4)
    one.rk3_step(dt, 2)
    want = one.get_state()
    one.close()
    dec = slabs.Slabs(shape, nslabs, lengths=lengths, precision=precision, nu=0.02)
    for sl in dec.slabs:
        sl.solver.set_option(gbfd.GBFD_OPT_KERNEL_PATH, path)
    dec.set_state(st)
    dec.rk3_step(dt, 2)
    got = dec.get_state()
    dec.close()
    assert np.array_equal(got, want)
    if precision == "fp64":
        g = fd.Grid(shape[2], shape[1], shape[0], *lengths)
        ref = fd.rk3_step(st, dt, g, fd.Physics(cs=1.0, nu=0.02), nsteps=2)
        assert np.all(rel_l2(got, ref) <= FP64_TOL)


def test_halo_calls_need_an_exchange_context():
    from paper_1707_08900_gb300 import gbfd
    s = gbfd.Solver((16, 16, 16), precision="fp32")
    buf = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    assert gbfd.load().gbfd_halo_bytes(s.ctx) == 0
    with pytest.raises(gbfd.GbfdError) as e:
        gbfd._check(gbfd.load().gbfd_halo_pack(s.ctx, 0, gbfd._VP(buf.data_ptr())), s.ctx)
    assert e.value.status == 5  # GBFD_ERR_UNSUPPORTED
    s.close()
