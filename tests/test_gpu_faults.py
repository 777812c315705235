"""Failure detection on the GPU without a GPU fault: a test-only option makes
the first CTA of the tiled kernel skip one TMA copy, so its mbarrier wait
runs out (bounded, about 2 s).  The kernel must record the failure and
leave; gbfd_sync must report GBFD_ERR_TIMEOUT; the context must stay usable
and give correct results once the option is cleared."""
import numpy as np
import pytest

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


@pytest.mark.parametrize("precision,cfg,report", [("fp32", -1, "sync"), ("fp32", -1, "get_state"),
                                                  ("fp32", 10, "sync"), ("fp32", 20, "get_state"),
                                                  ("fp64", -1, "sync")])
def test_bounded_wait_times_out_and_context_recovers(precision, cfg, report):
    """The FP32 default kernel and the lagged-output kernels (registers,
    tensor memory), and the FP64 default (lagged output, 5-slot ring: the
    skipped copy is one of the first ring fill, waited for in the prologue);
    the timeout is reported by gbfd_sync or by gbfd_get_state to host memory,
    which waits for the stream too."""
    from paper_1707_08900_gb300 import gbfd
    shape = (16, 16, 32)
    st = inputs.spectrum(shape, 12, mach=0.1, lnrho_rms=1e-3)
    if precision == "fp32":
        st = st.astype(np.float32)
    s = gbfd.Solver(shape, precision=precision, nu=5e-3)
    s.set_option(gbfd.GBFD_OPT_TILE_CONFIG, cfg)
    s.set_state(st)
    s.set_option(gbfd.GBFD_OPT_FAULT_SKIP_COPY, 4)  # a plane every column has
    s.substep(0, 0.01)
    with pytest.raises(gbfd.GbfdError) as err:
        if report == "sync":
            s.sync()
        else:
            s.get_state()
    assert err.value.status == 4  # GBFD_ERR_TIMEOUT
    s.set_option(gbfd.GBFD_OPT_FAULT_SKIP_COPY, -1)
    s.sync()  # the error word was cleared
    s.set_state(st)
    s.rk3_step(0.01, 1)
    s.sync()
    got = s.get_state()
    g = fd.Grid(32, 16, 16)
    ref = fd.rk3_step(st.astype(np.float64), 0.01, g, fd.Physics(cs=1.0, nu=5e-3))
    err = [np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-30)
           for a, b in zip(got[:4], ref[:4])]
    assert max(err) < (1e-5 if precision == "fp32" else 1e-12)
    s.close()
