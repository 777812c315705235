"""gbfd_diagnostics_noalloc: the diagnostics for callers that may not
allocate device memory (no context, no workspace; its partial sums live in a
fixed device array inside the library).

Checked against the regular context-based gbfd_diagnostics on two calls in
a row: a larger grid first, then a smaller one, so the second call runs over
scratch rows the first call left behind.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_1707_08900_gb300 import build as gb
from paper_1707_08900_gb300 import gbfd, inputs

FP64_TOL = 1e-12


def test_noalloc_rejects_bad_arguments_without_touching_the_gpu():
    gb.build()
    lib = gbfd.load()
    out = ctypes.c_void_p(0x1000)
    st = ctypes.c_void_p(0x2000)
    assert lib.gbfd_diagnostics_noalloc(None, 1, 8, 8, 8, 5, 1.0, 1.0, 1.0, None, out) == 1
    assert lib.gbfd_diagnostics_noalloc(st, 1, 8, 8, 8, 3, 1.0, 1.0, 1.0, None, out) == 1
    assert "nfields" in gbfd.gbfd_last_error(None)
    assert lib.gbfd_diagnostics_noalloc(st, 1, 0, 8, 8, 5, 1.0, 1.0, 1.0, None, out) == 1
    assert lib.gbfd_diagnostics_noalloc(st, 1, 1 << 12, 1 << 12, 1 << 12, 5, 1.0, 1.0, 1.0,
                                        None, out) == 1
    assert "2^33" in gbfd.gbfd_last_error(None)
    assert lib.gbfd_diagnostics_noalloc(st, 1, 8, 8, 8, 5, -1.0, 1.0, 1.0, None, out) == 1


@pytest.mark.gpu
@pytest.mark.parametrize("fp64", [True, False])
def test_noalloc_matches_context_diagnostics_on_two_calls(fp64):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    gb.build()
    lib = gbfd.load()
    stream = torch.cuda.current_stream()
    lengths = (2 * np.pi, 3.0, 4.0)
    cases = [((24, 40, 32), 11), ((16, 12, 8), 12)]  # big first, then small
    for shape, seed in cases:
        st = inputs.spectrum(shape, seed, mach=0.2, lnrho_rms=0.05)
        st[4] = 0.3 * st[2]
        if not fp64:
            st = st.astype(np.float32)
        dev = torch.from_numpy(np.ascontiguousarray(st)).cuda()
        out = torch.full((16,), float("nan"), dtype=torch.float64, device="cuda")
        nz, ny, nx = shape
        status = lib.gbfd_diagnostics_noalloc(ctypes.c_void_p(dev.data_ptr()), int(fp64), nx, ny,
                                              nz, 5, *lengths,
                                              ctypes.c_void_p(stream.cuda_stream),
                                              ctypes.c_void_p(out.data_ptr()))
        assert status == 0, gbfd.gbfd_last_error(None)
        torch.cuda.synchronize()
        got = out.cpu().numpy()

        s = gbfd.Solver(shape, lengths=lengths, precision="fp64", entropy_mode=1)
        s.set_state(st.astype(np.float64))
        ref = s.diagnostics()
        s.close()
        for i, k in enumerate(("mass", "ekin", "umax", "urms")):
            assert got[i] == pytest.approx(ref[k], rel=FP64_TOL), k
        np.testing.assert_allclose(got[4:9], ref["rms"], rtol=FP64_TOL)
        np.testing.assert_allclose(got[9:14], ref["maxabs"], rtol=FP64_TOL)
        assert got[14] == ref["nonfinite"] == 0
