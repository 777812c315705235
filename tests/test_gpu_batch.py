"""Batched form (many uneven periodic boxes, one persistent launch per
substep, CUDA-graph replay) and the autotuners, on the GPU.

Each box of a batch must reproduce (a) the FP64 oracle within the FP32
per-step bar and (b) the single-box solver (same arithmetic, same tile)."""
import numpy as np
import pytest

from bars import FP32_TOL, TERM_NU, inc_bar, inc_err, max_abs, term_exposing_state
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


def rel_l2(got, ref):
    out = []
    for g, o in zip(got, ref):
        no = np.linalg.norm(o.ravel())
        d = np.linalg.norm((g - o).ravel())
        out.append(d / no if no > 0 else d)
    return np.array(out)


def _states(ns, seed0, lengths):
    sts = []
    for i, n in enumerate(ns):
        st = inputs.spectrum((n, n, n), seed0 + i, p=-2.0, k1=1, k2=min(8, n // 4),
                             mach=0.05 + 0.05 * (i % 5), lnrho_rms=1e-2)
        sts.append(st.astype(np.float32))
    return sts


@pytest.mark.parametrize("graph", [1, 0])
def test_batch_matches_oracle_and_single_box(graph):
    from paper_1707_08900_gb300 import gbfd
    ns = [16, 32, 24, 40, 8]
    lengths = [2 * np.pi, 2 * np.pi, 3.0, 5.0, 1.0]
    nus = [2e-3, 5e-3, 1e-2, 4e-3, 8e-3]
    sts = _states(ns, 100, lengths)
    dts = [0.3 * (L / n) for L, n in zip(lengths, ns)]
    b = gbfd.Batch(ns, lengths, nus)
    b.set_option(gbfd.GBFD_BATCH_OPT_GRAPH, graph)
    for i, st in enumerate(sts):
        b.set_state(i, st)
    b.step(dts, 2)
    b.sync()
    for i, (n, L, nu, st, dt) in enumerate(zip(ns, lengths, nus, sts, dts)):
        got = b.get_state(i)
        g = fd.Grid(n, n, n, L, L, L)
        ref = fd.rk3_step(st.astype(np.float64), dt, g, fd.Physics(cs=1.0, nu=nu), nsteps=2)
        assert np.all(rel_l2(got, ref) <= 2 * FP32_TOL), (i, rel_l2(got, ref))
        s = gbfd.Solver((n, n, n), lengths=(L, L, L), precision="fp32", nu=nu)
        s.set_state(st)
        s.rk3_step(dt, 2)
        single = s.get_state()
        s.close()
        np.testing.assert_allclose(got, single, rtol=0, atol=1e-6 * np.abs(single).max())
    b.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_batch_one_step_elementwise_against_oracle(kind):
    """One batched RK3 step of uneven boxes on the term-exposing state (nu
    0.02): every box within the FP32 bars, relative L2 and the element-wise
    increment bar, for the two-plane routine (kind 0) and the lagged routine
    (kind 1; its 32^3 and 64^3 boxes are whole tiles and take the
    per-substep instantiations, the others the general one)."""
    from paper_1707_08900_gb300 import gbfd
    ns = [16, 32, 24, 40, 64]
    lengths = [2 * np.pi, 3.0, 2 * np.pi, 5.0, 2 * np.pi]
    sts = [term_exposing_state((n, n, n), 50 + i, inputs) for i, n in enumerate(ns)]
    b = gbfd.Batch(ns, lengths, [TERM_NU] * len(ns))
    b.set_option(gbfd.GBFD_BATCH_OPT_KERNEL, kind)
    dts = []
    for i, (n, L, st) in enumerate(zip(ns, lengths, sts)):
        b.set_state(i, st.astype(np.float32))
        g = fd.Grid(n, n, n, L, L, L)
        dts.append(fd.cfl_dt(st, g, fd.Physics(cs=1.0, nu=TERM_NU), 0.4))
    b.step(dts, 1)
    b.sync()
    for i, (n, L, st, dt) in enumerate(zip(ns, lengths, sts, dts)):
        got = b.get_state(i)
        g = fd.Grid(n, n, n, L, L, L)
        ref = fd.rk3_step(st, dt, g, fd.Physics(cs=1.0, nu=TERM_NU))
        err, inc, bar = rel_l2(got, ref), inc_err(got, ref, st), inc_bar(ref, st)
        print(f"box {i} ({n}^3): relL2 {err} inc {inc} bar {bar} maxabs {max_abs(got, ref)}")
        assert np.all(err <= FP32_TOL), (i, err)
        assert np.all(inc <= bar), (i, inc, bar)
    b.close()


def test_batch_graph_replay_equals_direct_launches_bitwise():
    from paper_1707_08900_gb300 import gbfd
    ns = [32, 16, 48]
    sts = _states(ns, 7, [2 * np.pi] * 3)
    outs = []
    for graph in (1, 0):
        b = gbfd.Batch(ns, [2 * np.pi] * 3, [5e-3, 3e-3, 8e-3])
        b.set_option(gbfd.GBFD_BATCH_OPT_GRAPH, graph)
        for i, st in enumerate(sts):
            b.set_state(i, st)
        for _ in range(3):  # odd step counts exercise both buffer parities
            b.step([0.01, 0.02, 0.005], 1)
        b.step([0.01, 0.02, 0.005], 2)
        outs.append([b.get_state(i, fp64=False) for i in range(len(ns))])
        b.close()
    for a, c in zip(*outs):
        assert np.array_equal(a, c)


def test_batch_autotune_keeps_state_and_chunks_agree():
    """The autotuner times every column routine x z-chunk x launch mode on
    dt = 0 steps, which leave the state unchanged; chunk lengths, launch
    modes and the two-plane tile widths give the same bits (same arithmetic
    per point), the lagged routine agrees to rounding."""
    from paper_1707_08900_gb300 import gbfd
    ns = [32, 64, 16]
    sts = _states(ns, 31, [2 * np.pi] * 3)
    b = gbfd.Batch(ns, [2 * np.pi] * 3, [5e-3] * 3)
    for i, st in enumerate(sts):
        b.set_state(i, st)
    zc, ms = b.autotune(steps=1)
    assert zc in (8, 16, 32, 64) and ms > 0
    assert b.get_option(gbfd.GBFD_BATCH_OPT_KERNEL) in (0, 1, 2)
    assert b.get_option(gbfd.GBFD_BATCH_OPT_DATAFLOW) in (0, 1)
    for i, st in enumerate(sts):
        assert np.array_equal(b.get_state(i, fp64=False), st)
    outs = {}
    for kind in (0, 2, 1):
        b.set_option(gbfd.GBFD_BATCH_OPT_KERNEL, kind)
        for flow in (1, 0):
            b.set_option(gbfd.GBFD_BATCH_OPT_DATAFLOW, flow)
            for z in (8, 32, 64):
                b.set_option(gbfd.GBFD_BATCH_OPT_ZCHUNK, z)
                for i, st in enumerate(sts):
                    b.set_state(i, st)
                b.step([0.01] * 3, 2)
                outs[(kind, flow, z)] = [b.get_state(i, fp64=False) for i in range(3)]
    base = outs[(0, 1, 8)]
    for key, out in outs.items():
        for a, c in zip(base, out):
            if key[0] == 1:
                np.testing.assert_allclose(a, c, rtol=0, atol=2e-6 * np.abs(c).max())
            else:
                assert np.array_equal(a, c), key
    # the lagged routine's chunk lengths and launch modes agree bitwise among themselves
    for key, out in outs.items():
        if key[0] == 1:
            for a, c in zip(outs[(1, 1, 8)], out):
                assert np.array_equal(a, c), key
    b.close()


@pytest.mark.parametrize("kind", [0, 1])
def test_dataflow_wait_times_out_and_batch_recovers(kind):
    """A dataflow work item that is never counted as done (fault injection on
    the host side: GBFD_BATCH_OPT_FAULT_STALL) makes its box's next substep
    wait until the bounded wait gives up: gbfd_batch_sync reports
    GBFD_ERR_TIMEOUT, and the batch steps correctly afterwards."""
    from paper_1707_08900_gb300 import gbfd
    ns = [16, 24]
    sts = _states(ns, 5, [2 * np.pi] * 2)
    b = gbfd.Batch(ns, [2 * np.pi] * 2, [5e-3] * 2)
    b.set_option(gbfd.GBFD_BATCH_OPT_KERNEL, kind)
    b.set_option(gbfd.GBFD_BATCH_OPT_DATAFLOW, 1)
    for i, st in enumerate(sts):
        b.set_state(i, st)
    b.set_option(gbfd.GBFD_BATCH_OPT_FAULT_STALL, 0)  # box 0, first column, first substep
    b.step([0.01, 0.01], 1)
    with pytest.raises(gbfd.GbfdError) as err:
        b.sync()
    assert err.value.status == 4  # GBFD_ERR_TIMEOUT
    b.set_option(gbfd.GBFD_BATCH_OPT_FAULT_STALL, -1)
    b.sync()  # the error word was cleared
    for i, st in enumerate(sts):
        b.set_state(i, st)
    b.step([0.01, 0.01], 1)
    b.sync()
    for i, (n, st) in enumerate(zip(ns, sts)):
        g = fd.Grid(n, n, n)
        ref = fd.rk3_step(st.astype(np.float64), 0.01, g, fd.Physics(cs=1.0, nu=5e-3))
        assert np.all(rel_l2(b.get_state(i), ref) <= FP32_TOL)
    b.close()


def test_single_box_autotune_cache(tmp_path):
    from paper_1707_08900_gb300 import gbfd
    shape = (32, 32, 64)
    st = inputs.spectrum(shape, 3, mach=0.1, lnrho_rms=1e-3).astype(np.float32)
    s = gbfd.Solver(shape, precision="fp32")
    s.set_state(st)
    path = str(tmp_path / "tune.json")
    cfg, ms = s.autotune(reps=1, cache_path=path)
    assert ms > 0 and 0 <= cfg < 64
    assert np.array_equal(s.get_state(fp64=False), st)  # state untouched
    s2 = gbfd.Solver(shape, precision="fp32")
    cfg2, ms2 = s2.autotune(reps=1, cache_path=path)
    assert cfg2 == cfg and ms2 == 0.0  # cache hit
    text = open(path).read()
    assert "fields5" in text and '"cfg"' in text
    s.close()
    s2.close()


def test_config4_batch_96_boxes_sampled():
    """The 96-box batch (32 each of 32^3, 64^3, 128^3; rms Mach drawn from
    0.05-0.3 and nu from 2e-3-1e-2, seeds 100..195): two steps, boxes of
    every size checked against the single-box solver, a 32^3 one against
    the oracle."""
    from paper_1707_08900_gb300 import gbfd
    rng = np.random.default_rng(4)
    ns = [32] * 32 + [64] * 32 + [128] * 32
    mach = rng.uniform(0.05, 0.3, 96)
    nus = rng.uniform(2e-3, 1e-2, 96)
    b = gbfd.Batch(ns, [2 * np.pi] * 96, nus)
    sts = {}
    for i, n in enumerate(ns):
        st = inputs.spectrum((n, n, n), 100 + i, p=-2.0, k1=1, k2=8, mach=mach[i],
                             lnrho_rms=1e-3).astype(np.float32)
        b.set_state(i, st)
        if i in (0, 40, 95):
            sts[i] = st
    dts = [0.4 * (2 * np.pi / n) / (1.0 + 1.5 * m) for n, m in zip(ns, mach)]
    b.step(dts, 2)
    b.sync()
    for i, st in sts.items():
        n = ns[i]
        s = gbfd.Solver((n, n, n), precision="fp32", nu=nus[i])
        s.set_state(st)
        s.rk3_step(dts[i], 2)
        single = s.get_state()
        s.close()
        got = b.get_state(i)
        np.testing.assert_allclose(got, single, rtol=0, atol=1e-6 * np.abs(single).max())
    g = fd.Grid(32, 32, 32)
    ref = fd.rk3_step(sts[0].astype(np.float64), dts[0], g, fd.Physics(cs=1.0, nu=nus[0]),
                      nsteps=2)
    assert np.all(rel_l2(b.get_state(0), ref) <= 2 * FP32_TOL)
    b.close()
