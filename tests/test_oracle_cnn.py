"""Pins of the FP64 network oracle (oracle/cnn.py) against facts that do not
come from its own code: brute-force direct summation of the periodic
cross-correlation on a tiny grid, convolution with a delta kernel (a pure
periodic shift), the adjoint identity <conv(x), y> = <x, conv^T(y)>, central
finite differences of the loss, GELU against its closed-form derivative and
Phi, and Adam's first step (lr * sign(g))."""
import itertools
import math

import numpy as np
import pytest

from oracle import cnn


def test_conv_matches_brute_force_sum():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 3, 4, 5))
    W = rng.standard_normal((3, 2, 3, 3, 3))
    b = rng.standard_normal(3)
    y = cnn.conv3d(x, W, b)
    nz, ny, nx = x.shape[1:]
    for o, z, yy, xx in itertools.product(range(3), range(nz), range(ny), range(nx)):
        acc = b[o]
        for c, i, j, k in itertools.product(range(2), range(3), range(3), range(3)):
            acc += W[o, c, i, j, k] * x[c, (z + i - 1) % nz, (yy + j - 1) % ny, (xx + k - 1) % nx]
        assert y[o, z, yy, xx] == pytest.approx(acc, abs=1e-12)


def test_delta_kernel_is_a_periodic_shift():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((1, 4, 5, 6))
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 2, 0, 1] = 1.0  # tap (dz, dy, dx) = (1, -1, 0)
    y = cnn.conv3d(x, W, np.zeros(1))
    assert np.array_equal(y[0], np.roll(x[0], shift=(-1, 1, 0), axis=(0, 1, 2)))


def test_conv_backward_is_the_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((3, 4, 4, 5))
    W = rng.standard_normal((2, 3, 3, 3, 3))
    dy = rng.standard_normal((2, 4, 4, 5))
    dx, dW, db = cnn.conv3d_backward(x, W, dy)
    y = cnn.conv3d(x, W, np.zeros(2))
    assert np.sum(y * dy) == pytest.approx(np.sum(x * dx), rel=1e-12)
    assert np.sum(y * dy) == pytest.approx(np.sum(W * dW), rel=1e-12)
    assert np.allclose(db, dy.sum(axis=(1, 2, 3)))


def test_gelu_closed_forms():
    h = np.linspace(-4, 4, 41)
    phi = 0.5 * (1 + np.array([math.erf(v / math.sqrt(2)) for v in h]))
    np.testing.assert_allclose(cnn.gelu(h), h * phi, rtol=1e-14, atol=1e-15)
    eps = 1e-6
    fd = (cnn.gelu(h + eps) - cnn.gelu(h - eps)) / (2 * eps)
    np.testing.assert_allclose(cnn.gelu_grad(h), fd, rtol=1e-7, atol=1e-9)


def test_network_gradients_match_finite_differences():
    rng = np.random.default_rng(3)
    p = cnn.init_params(5, hidden=4)
    p["W3"] *= 10.0
    for k in ("b1", "b2", "b3"):
        p[k] = 0.1 * rng.standard_normal(p[k].shape)
    xs = [rng.standard_normal((5, 4, 4, 4)) for _ in range(2)]
    ts = [rng.standard_normal((5, 4, 4, 4)) for _ in range(2)]
    loss, g = cnn.loss_and_grads(xs, ts, p)
    h = 1e-6
    for k, idxs in (("W1", [(0, 1, 0, 2, 1), (3, 4, 2, 2, 2)]), ("W2", [(1, 2, 1, 0, 1)]),
                    ("W3", [(4, 3, 0, 0, 0), (2, 0, 1, 2, 1)]), ("b1", [(2,)]), ("b3", [(0,)])):
        for idx in idxs:
            pp = {kk: v.copy() for kk, v in p.items()}
            pm = {kk: v.copy() for kk, v in p.items()}
            pp[k][idx] += h
            pm[k][idx] -= h
            lp, _ = cnn.loss_and_grads(xs, ts, pp)
            lm, _ = cnn.loss_and_grads(xs, ts, pm)
            fdg = (lp - lm) / (2 * h)
            assert g[k][idx] == pytest.approx(fdg, rel=1e-7, abs=1e-10), (k, idx)


def test_adam_first_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -0.1, 0.0])}
    cnn.adam(p, g, {}, lr=0.01)
    np.testing.assert_allclose(p["w"], [0.99, -1.99, 3.0], atol=1e-7)


def test_zero_last_layer_means_no_correction():
    rng = np.random.default_rng(6)
    p = cnn.init_params(0, hidden=4)
    p["W3"][:] = 0.0
    st = rng.standard_normal((5, 4, 4, 4))
    out = cnn.correct(st, p, np.zeros(5), np.ones(5), np.ones(5))
    assert np.array_equal(out, st)
