"""FP64 NumPy reference of the coarse-grid correction network (TEST
INFRASTRUCTURE ONLY; only tests and the benchmark's baseline legs use it).

The paper has no learned component; the network is the spec addition
that corrects a coarse-grid RK3 step towards the box-filtered fine-grid
solution.  Readings used (none is fixed by the paper):
  * three 3x3x3 convolutions with circular (periodic) padding, channels
    5 -> 32 -> 32 -> 5, exact GELU, h*Phi(h) = h/2 (1 + erf(h/sqrt 2)), after
    the first two;
  * the convolution is a cross-correlation:
        y[o, p] = b[o] + sum_{c, t} W[o, c, t] x[c, p + t],  t in {-1,0,1}^3,
    with W indexed [o, c, dz+1, dy+1, dx+1] (the torch conv3d convention);
  * input normalisation (state - mean_in) / std_in per channel; the output is
    the normalised residual, de-normalised by std_out per channel and added
    to the state;
  * loss: mean squared error over batch, channel and point of the normalised
    residual.
Everything is plain FP64: np.roll for the periodic taps, einsum for the
channel contractions; no blocking or fusion.
"""
import numpy as np
from scipy.special import erf

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, t):
    """x[..., p + t] on the periodic grid (last three axes z, y, x)."""
    dz, dy, dx = t
    return np.roll(x, shift=(-dz, -dy, -dx), axis=(-3, -2, -1))


def unshift(x, t):
    dz, dy, dx = t
    return np.roll(x, shift=(dz, dy, dx), axis=(-3, -2, -1))


def conv3d(x, W, b):
    """x: (C, nz, ny, nx); W: (O, C, 3, 3, 3); b: (O,)."""
    y = np.zeros((W.shape[0],) + x.shape[1:])
    for t in TAPS:
        Wt = W[:, :, t[0] + 1, t[1] + 1, t[2] + 1]
        y += np.einsum("oc,czyx->ozyx", Wt, shift(x, t))
    return y + b[:, None, None, None]


def conv3d_backward(x, W, dy):
    """Gradients of sum(dy * conv3d(x, W, b)) w.r.t. x, W and b."""
    dW = np.zeros_like(W)
    dx = np.zeros_like(x)
    for t in TAPS:
        xs = shift(x, t)
        dW[:, :, t[0] + 1, t[1] + 1, t[2] + 1] = np.einsum("ozyx,czyx->oc", dy, xs)
        dx += unshift(np.einsum("oc,ozyx->czyx", W[:, :, t[0] + 1, t[1] + 1, t[2] + 1], dy), t)
    db = dy.sum(axis=(1, 2, 3))
    return dx, dW, db


def gelu(h):
    return 0.5 * h * (1.0 + erf(h / np.sqrt(2.0)))


def gelu_grad(h):
    return 0.5 * (1.0 + erf(h / np.sqrt(2.0))) + h * np.exp(-0.5 * h * h) / np.sqrt(2.0 * np.pi)


def init_params(seed, cin=5, hidden=32, cout=5):
    """Seeded He-style initialisation (the starting point of training)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, c) in (("1", (hidden, cin)), ("2", (hidden, hidden)), ("3", (cout, hidden))):
        p["W" + name] = rng.standard_normal((o, c, 3, 3, 3)) * np.sqrt(2.0 / (27 * c))
        p["b" + name] = np.zeros(o)
    p["W3"] *= 0.1  # start close to "no correction"
    return p


def forward(x0, p):
    """x0: normalised input (5, n, n, n).  Returns (y, cache)."""
    h1 = conv3d(x0, p["W1"], p["b1"])
    a1 = gelu(h1)
    h2 = conv3d(a1, p["W2"], p["b2"])
    a2 = gelu(h2)
    y = conv3d(a2, p["W3"], p["b3"])
    return y, (x0, h1, a1, h2, a2)


def backward(dy, p, cache):
    x0, h1, a1, h2, a2 = cache
    g = {}
    da2, g["W3"], g["b3"] = conv3d_backward(a2, p["W3"], dy)
    dh2 = da2 * gelu_grad(h2)
    da1, g["W2"], g["b2"] = conv3d_backward(a1, p["W2"], dh2)
    dh1 = da1 * gelu_grad(h1)
    _, g["W1"], g["b1"] = conv3d_backward(x0, p["W1"], dh1)
    return g


def mse_loss(ys, ts):
    """Mean over batch, channel and point; returns (loss, dloss/dy list)."""
    n = sum(y.size for y in ys)
    loss = sum(float(np.sum((y - t) ** 2)) for y, t in zip(ys, ts)) / n
    return loss, [2.0 * (y - t) / n for y, t in zip(ys, ts)]


def loss_and_grads(xs, ts, p):
    """Batch loss and parameter gradients (summed over the batch)."""
    ys, caches = zip(*(forward(x, p) for x in xs))
    loss, dys = mse_loss(ys, ts)
    total = None
    for dy, cache in zip(dys, caches):
        g = backward(dy, p, cache)
        total = g if total is None else {k: total[k] + g[k] for k in g}
    return loss, total


def adam(p, g, state, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015) on the dict p, in place."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m" + k, np.zeros_like(p[k]))
        v = state.setdefault("v" + k, np.zeros_like(p[k]))
        m[:] = b1 * m + (1 - b1) * g[k]
        v[:] = b2 * v + (1 - b2) * g[k] ** 2
        mh = m / (1 - b1 ** t)
        vh = v / (1 - b2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
    return p


def correct(state, p, mean_in, std_in, std_out):
    """state + std_out * net((state - mean_in) / std_in), per channel."""
    x0 = (state - mean_in[:, None, None, None]) / std_in[:, None, None, None]
    y, _ = forward(x0, p)
    return state + std_out[:, None, None, None] * y
