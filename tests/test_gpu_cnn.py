"""GPU tests of the learned coarse-grid correction: the tensor-core network
against the FP64 oracle (forward and parameter gradients, within BF16
bounds), the box filter, and a short end-to-end training that must make the
corrected coarse solver track the filtered fine solution better than the
plain coarse solver."""
import numpy as np
import pytest

from oracle import cnn as ocnn
from oracle import fd
from paper_1707_08900_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BF16_FWD_TOL = 2e-2
BF16_GRAD_TOL = 2e-2


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_1707_08900_gb300 import build
    build.build()


def _params(seed):
    p = ocnn.init_params(seed)
    rng = np.random.default_rng(seed + 1)
    p["W3"] *= 10.0
    for k in ("b1", "b2", "b3"):
        p[k] = 0.05 * rng.standard_normal(p[k].shape)
    return p


def _rel(a, b):
    return np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel())


def _net(n, batch, p):
    from paper_1707_08900_gb300 import gbfd
    net = gbfd.CNN(n, batch=batch)
    net.set_params(p)
    net.set_norm(np.zeros(5), np.ones(5), np.ones(5))
    return net


@pytest.mark.parametrize("n,batch,grid", [(8, 2, 0), (12, 1, 0), (8, 2, 1), (12, 1, 2),
                                          (32, 2, 0), (32, 2, 7)])
def test_forward_matches_oracle(n, batch, grid):
    """`grid` caps the CTAs of each convolution launch (0: the default, one
    per SM), so that every CTA walks several tiles (tiles of 8 x 16 x 4
    points: 8^3 x 2 has 4, 32^3 x 2 has 128; 7 CTAs give 18-19 tiles each),
    reusing its halo stages, barrier phases and both TMEM accumulator
    buffers."""
    from paper_1707_08900_gb300 import gbfd
    p = _params(3)
    rng = np.random.default_rng(4)
    xs = rng.standard_normal((batch, 5, n, n, n))
    net = _net(n, batch, p)
    net.set_option(gbfd.GBFD_CNN_OPT_CONV_GRID, grid)
    ys = net.forward(torch.from_numpy(xs.astype(np.float32)).cuda()).cpu().numpy()
    for b in range(batch):
        y_ref, _ = ocnn.forward(xs[b], p)
        assert _rel(ys[b], y_ref) < BF16_FWD_TOL
    # parameters round-trip exactly
    back = net.unflatten(net.get_params())
    for k in p:
        np.testing.assert_allclose(back[k], p[k].astype(np.float32), rtol=0, atol=0)
    net.close()


@pytest.mark.parametrize("n,batch,grid,parts", [(8, 2, 0, 0), (8, 2, 1, 3), (32, 2, 0, 0),
                                                (32, 2, 5, 17)])
def test_gradients_match_oracle(n, batch, grid, parts):
    """Loss and parameter gradients against the FP64 oracle; `grid` caps the
    convolution CTAs as in the forward test, `parts` the CTAs of the weight
    gradient sums (0: defaults), so CTAs loop over many tiles and points."""
    from paper_1707_08900_gb300 import gbfd
    p = _params(5)
    rng = np.random.default_rng(6)
    xs = rng.standard_normal((batch, 5, n, n, n))
    tgt = rng.standard_normal((batch, 5, n, n, n))  # normalised residual targets
    net = _net(n, batch, p)
    net.set_option(gbfd.GBFD_CNN_OPT_CONV_GRID, grid)
    net.set_option(gbfd.GBFD_CNN_OPT_WGRAD_PARTS, parts)
    xs_d = torch.from_numpy(xs.astype(np.float32)).cuda()
    ts_d = torch.from_numpy((xs + tgt).astype(np.float32)).cuda()
    g, loss = net.gradients(xs_d, ts_d)
    ref_loss, ref_g = ocnn.loss_and_grads(list(xs), list(tgt), p)
    assert loss == pytest.approx(ref_loss, rel=BF16_FWD_TOL)
    gg = net.unflatten(g)
    errs = {k: _rel(gg[k], ref_g[k]) for k in ref_g}
    print({k: f"{v:.2e}" for k, v in errs.items()})
    for k in ref_g:
        assert errs[k] < BF16_GRAD_TOL, (k, errs)
    net.close()


def test_train_step_lowers_the_loss():
    p = _params(7)
    n, batch = 8, 4
    rng = np.random.default_rng(8)
    xs = torch.from_numpy(rng.standard_normal((batch, 5, n, n, n)).astype(np.float32)).cuda()
    ts = xs + 0.3 * torch.roll(xs, 1, dims=4)
    net = _net(n, batch, p)
    losses = [net.train_step(xs, ts, 1e-3) for _ in range(30)]
    assert losses[-1] < 0.7 * losses[0]
    net.close()


def test_box_filter_matches_oracle():
    from paper_1707_08900_gb300 import gbfd
    n = 32
    st = inputs.spectrum((n, n, n), 9, mach=0.2, lnrho_rms=1e-2).astype(np.float32)
    s = gbfd.Solver((n, n, n), precision="fp32")
    s.set_state(st)
    got = gbfd.box_filter(s, 4).cpu().numpy()
    ref = fd.box_filter(st.astype(np.float64), 4)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-6 * np.abs(ref).max())
    s.close()


def test_zero_network_leaves_the_coarse_step_unchanged():
    from paper_1707_08900_gb300 import gbfd
    n = 16
    p = _params(1)
    p["W3"][:] = 0.0
    p["b3"][:] = 0.0
    st = inputs.spectrum((n, n, n), 2, mach=0.2, lnrho_rms=1e-2).astype(np.float32)
    a = gbfd.Solver((n, n, n), precision="fp32")
    b = gbfd.Solver((n, n, n), precision="fp32")
    a.set_state(st)
    b.set_state(st)
    net = _net(n, 1, p)
    a.rk3_step(0.02, 3)
    net.step_corrected(b, 0.02, 3)
    assert np.array_equal(a.get_state(fp64=False), b.get_state(fp64=False))
    s64 = gbfd.Solver((n, n, n), precision="fp64")
    with pytest.raises(gbfd.GbfdError):
        net.apply(s64)
    net.close()


@pytest.mark.parametrize("n,grid", [(16, 0), (24, 3)])
def test_apply_matches_oracle_correct(n, grid):
    """gbfd_cnn_apply on a solver's state (normalise, three convolutions,
    de-normalise, add to the state with its ghost copies) against the
    oracle's state + std_out * net((state - mean_in) / std_in): the
    increment within the BF16 bound; `grid` caps the convolution CTAs so
    that each walks several tiles.  A step afterwards must read the
    updated ghosts: it is compared with a fresh context holding the same
    state."""
    from paper_1707_08900_gb300 import gbfd
    p = _params(11)
    st = inputs.spectrum((n, n, n), 12, mach=0.3, lnrho_rms=5e-2).astype(np.float32)
    st[4] = 0.02 * np.random.default_rng(13).standard_normal((n, n, n)).astype(np.float32)
    mean_in = np.array([0.01, 0.02, -0.01, 0.0, 0.005])
    std_in = np.array([0.05, 0.3, 0.25, 0.3, 0.02])
    std_out = np.array([1e-3, 2e-3, 3e-3, 2.5e-3, 1e-3])
    s = gbfd.Solver((n, n, n), precision="fp32", nu=5e-3)
    s.set_state(st)
    net = gbfd.CNN(n, batch=1)
    net.set_params(p)
    net.set_norm(mean_in, std_in, std_out)
    net.set_option(gbfd.GBFD_CNN_OPT_CONV_GRID, grid)
    net.apply(s)
    got = s.get_state()
    st64 = st.astype(np.float64)
    ref = ocnn.correct(st64, p, mean_in, std_in, std_out)
    assert _rel(got - st64, ref - st64) < BF16_FWD_TOL
    # the ghost copies were updated with the interior: one step from the
    # corrected context equals one step from a fresh copy of its state
    fresh = gbfd.Solver((n, n, n), precision="fp32", nu=5e-3)
    fresh.set_state(s.get_state(fp64=False))
    s.rk3_step(0.01, 1)
    fresh.rk3_step(0.01, 1)
    assert np.array_equal(s.get_state(fp64=False), fresh.get_state(fp64=False))
    for x in (s, fresh, net):
        x.close()


def test_training_beats_the_plain_coarse_solver():
    """64^3 fine runs filtered to 16^3: after a short GPU training the
    corrected coarse solver is closer to the filtered fine solution than the
    plain coarse solver on held-out seeds."""
    from paper_1707_08900_gb300 import learned
    res = learned.run(fine=64, ratio=4, train_seeds=16, eval_seeds=3, nsnap=8, gap=4, steps=16,
                      train_steps=400, batch=8, lr=1e-3, k2=6, check_every=16, noise=0.0)
    assert res["train_loss_final_mean"] < 0.5 * res["train_loss_initial_mean"]
    assert res["rel_l2_u_corrected"] < 0.9 * res["rel_l2_u_plain"], res
