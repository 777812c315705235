"""Learned coarse-grid correction: training data from the solver's own
fine-grid runs, training on the GPU with the library's kernels, evaluation
against the box-filtered fine solution.

    python -m paper_1707_08900_gb300.learned --fine 256 --ratio 4 \\
        --train-seeds 200 --eval-seeds 20 --steps 200 --out learned.json

Recipe (the paper has no learned component; these are the readings used):
* fine runs: n_fine^3 FP32 55-point solver, k^-2 velocity spectrum over
  1 <= k <= 8 at rms Mach drawn uniformly from [0.1, 0.3], lnrho 1e-3,
  entropy 0, nu = 5e-3, seeds 1000 + i (training) and 1200 + i (held out);
  dt_fine from CFL 0.4 on the initial state, dt_coarse = ratio * dt_fine;
* a training pair: the filtered fine state c_t advanced one coarse step by
  the coarse solver (x), and the filtered fine state one coarse step later
  (t); the network learns (t - x) / std_out from (x - mean_in) / std_in;
* Adam with a cosine learning-rate decay from lr to lr/10, mini-batches
  drawn without replacement each epoch; each input is perturbed by Gaussian
  noise of `noise` x std_out per channel, and the target residual is taken
  from the perturbed input, so the network also learns to remove error that
  earlier corrected steps left behind (this keeps long rollouts stable);
* evaluation: from the filtered initial state, the plain coarse solver and
  the corrected one (RK3 step + network after every step) against the
  filtered fine run, relative L2 of velocity and lnrho, and wall times of
  the three runs.
"""
import argparse
import json
import time

import numpy as np

from . import gbfd, inputs


def _spectrum_state(n, seed, k2, mach_range):
    rng = np.random.default_rng(seed)
    mach = rng.uniform(*mach_range)
    st = inputs.spectrum((n, n, n), seed, p=-2.0, k1=1, k2=k2, mach=mach, lnrho_rms=1e-3)
    return st.astype(np.float32), mach


def generate_pairs(seeds, n_fine, ratio, nsnap, gap, nu=5e-3, k2=8, mach_range=(0.1, 0.3)):
    """Training pairs (x, t) as torch CUDA tensors [S, 5, nc, nc, nc]."""
    import torch
    nc = n_fine // ratio
    xs, ts = [], []
    for seed in seeds:
        st, _ = _spectrum_state(n_fine, seed, k2, mach_range)
        fine = gbfd.Solver((n_fine,) * 3, precision="fp32", nu=nu)
        coarse = gbfd.Solver((nc,) * 3, precision="fp32", nu=nu)
        fine.set_state(st)
        dt_f = fine.cfl_dt(0.4)
        for _ in range(nsnap):
            c = gbfd.box_filter(fine, ratio)
            coarse.set_state(c)
            coarse.rk3_step(ratio * dt_f, 1)
            x = torch.empty_like(c)
            coarse.get_state(out=x)
            fine.rk3_step(dt_f, ratio)
            xs.append(x)
            ts.append(gbfd.box_filter(fine, ratio))
            if gap:
                fine.rk3_step(dt_f, gap)
        fine.close()
        coarse.close()
    torch.cuda.synchronize()
    return torch.stack(xs), torch.stack(ts)


def norm_stats(xs, ts):
    dims = (0, 2, 3, 4)
    mean_in = xs.mean(dim=dims).double().cpu().numpy()
    std_in = xs.std(dim=dims).double().cpu().numpy()
    std_out = (ts - xs).std(dim=dims).double().cpu().numpy()
    std_in[std_in < 1e-12] = 1.0
    std_out[std_out < 1e-12] = 1.0
    return mean_in, std_in, std_out


def init_params(seed, hidden=32):
    """Seeded He-style start, last layer scaled down (near 'no correction')."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, (o, c) in (("1", (hidden, 5)), ("2", (hidden, hidden)), ("3", (5, hidden))):
        p["W" + name] = rng.standard_normal((o, c, 3, 3, 3)) * np.sqrt(2.0 / (27 * c))
        p["b" + name] = np.zeros(o)
    p["W3"] *= 0.1
    return p


def train(net, xs, ts, steps, batch, lr=3e-4, seed=0, log_every=50, noise=0.0, std_out=None):
    import torch
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=xs.device)
    gen.manual_seed(seed)
    scale = None
    if noise > 0:
        scale = torch.as_tensor(noise * np.asarray(std_out), dtype=torch.float32,
                                device=xs.device).view(1, -1, 1, 1, 1)
    S = xs.shape[0]
    order = rng.permutation(S)
    pos = 0
    hist = []
    for it in range(steps):
        if pos + batch > S:
            order = rng.permutation(S)
            pos = 0
        idx = torch.as_tensor(order[pos:pos + batch], device=xs.device)
        pos += batch
        want = (it % log_every == 0) or (it == steps - 1)
        lr_t = lr * (0.1 + 0.9 * 0.5 * (1.0 + np.cos(np.pi * it / max(steps - 1, 1))))
        xb = xs.index_select(0, idx)
        if scale is not None:
            xb = xb + scale * torch.randn(xb.shape, generator=gen, device=xb.device)
        loss = net.train_step(xb, ts.index_select(0, idx), lr_t, want_loss=want)
        if want:
            hist.append((it, loss))
    return hist


def _rel(a, b, fields):
    import torch
    d = torch.linalg.vector_norm((a[fields] - b[fields]).double())
    return float(d / torch.linalg.vector_norm(b[fields].double()))


def evaluate(net, seeds, n_fine, ratio, nsteps, nu=5e-3, k2=8, mach_range=(0.1, 0.3),
             check_every=None):
    """Plain and corrected coarse runs against the filtered fine run."""
    import torch
    nc = n_fine // ratio
    res = {"plain_u": [], "corrected_u": [], "plain_lnrho": [], "corrected_lnrho": [],
           "ms_fine": 0.0, "ms_plain": 0.0, "ms_corrected": 0.0, "curve": []}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn):
        ev[0].record()
        fn()
        ev[1].record()
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1])

    check_every = check_every or nsteps
    for seed in seeds:
        st, _ = _spectrum_state(n_fine, seed, k2, mach_range)
        fine = gbfd.Solver((n_fine,) * 3, precision="fp32", nu=nu)
        fine.set_state(st)
        dt_f = fine.cfl_dt(0.4)
        c0 = gbfd.box_filter(fine, ratio)
        plain = gbfd.Solver((nc,) * 3, precision="fp32", nu=nu)
        corr = gbfd.Solver((nc,) * 3, precision="fp32", nu=nu)
        plain.set_state(c0)
        corr.set_state(c0)
        done, curve = 0, []
        while done < nsteps:
            k = min(check_every, nsteps - done)
            res["ms_fine"] += timed(lambda: fine.rk3_step(dt_f, ratio * k))
            res["ms_plain"] += timed(lambda: plain.rk3_step(ratio * dt_f, k))
            if net is not None:
                res["ms_corrected"] += timed(lambda: net.step_corrected(corr, ratio * dt_f, k))
            done += k
            f = gbfd.box_filter(fine, ratio)
            xp = torch.empty_like(f)
            plain.get_state(out=xp)
            xc = torch.empty_like(f)
            corr.get_state(out=xc)
            curve.append((done, _rel(xp, f, slice(1, 4)),
                          _rel(xc, f, slice(1, 4)) if net is not None else None))
        res["plain_u"].append(_rel(xp, f, slice(1, 4)))
        res["plain_lnrho"].append(_rel(xp, f, slice(0, 1)))
        if net is not None:
            res["corrected_u"].append(_rel(xc, f, slice(1, 4)))
            res["corrected_lnrho"].append(_rel(xc, f, slice(0, 1)))
        res["curve"].append(curve)
        for s in (fine, plain, corr):
            s.close()
    return res


def device_cost(net, n_fine, ratio, nsteps, nu=5e-3, k2=8):
    """GPU time per step of the fine, plain coarse and corrected coarse runs,
    each `nsteps` (fine: ratio x nsteps) steps back to back on one stream
    after a warm-up: the device cost, without the host time between the
    evaluation's timed segments."""
    import torch
    nc = n_fine // ratio
    st, _ = _spectrum_state(n_fine, 1200, k2, (0.1, 0.3))
    fine = gbfd.Solver((n_fine,) * 3, precision="fp32", nu=nu)
    fine.set_state(st)
    dt_f = fine.cfl_dt(0.4)
    c0 = gbfd.box_filter(fine, ratio)
    plain = gbfd.Solver((nc,) * 3, precision="fp32", nu=nu)
    corr = gbfd.Solver((nc,) * 3, precision="fp32", nu=nu)
    plain.set_state(c0)
    corr.set_state(c0)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def timed(fn, n):
        fn(3)
        torch.cuda.synchronize()
        ev[0].record()
        fn(n)
        ev[1].record()
        ev[1].synchronize()
        return ev[0].elapsed_time(ev[1]) / n

    out = {"fine": timed(lambda n: fine.rk3_step(dt_f, n), ratio * nsteps),
           "plain": timed(lambda n: plain.rk3_step(ratio * dt_f, n), nsteps),
           "corrected": timed(lambda n: net.step_corrected(corr, ratio * dt_f, n), nsteps)}
    for s in (fine, plain, corr):
        s.close()
    return out


def run(fine=256, ratio=4, train_seeds=200, eval_seeds=20, nsnap=10, gap=None, steps=200,
        train_steps=4000, batch=8, lr=3e-4, nu=5e-3, k2=8, seed=0, check_every=25, noise=1.0):
    """The full pipeline; returns a JSON-able summary."""
    import torch
    nc = fine // ratio
    gap = gap if gap is not None else max(0, (ratio * steps) // nsnap - ratio)
    t0 = time.perf_counter()
    xs, ts = generate_pairs(range(1000, 1000 + train_seeds), fine, ratio, nsnap, gap, nu, k2)
    t_data = time.perf_counter() - t0
    mean_in, std_in, std_out = norm_stats(xs, ts)
    net = gbfd.CNN(nc, batch=batch)
    net.set_params(init_params(seed))
    net.set_norm(mean_in, std_in, std_out)

    def set_loss():  # one-step objective over the whole training set, noise-free
        return float(np.mean([net.gradients(xs[i:i + batch], ts[i:i + batch])[1]
                              for i in range(0, xs.shape[0] - batch + 1, batch)]))

    loss0 = set_loss()
    t0 = time.perf_counter()
    hist = train(net, xs, ts, train_steps, batch, lr, seed, noise=noise, std_out=std_out)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    loss1 = set_loss()
    ev = evaluate(net, range(1200, 1200 + eval_seeds), fine, ratio, steps, nu, k2,
                  check_every=check_every)
    dev = device_cost(net, fine, ratio, steps, nu, k2)
    mean = lambda v: float(np.mean(v)) if v else None
    return {
        "fine": fine, "coarse": nc, "ratio": ratio, "train_pairs": int(xs.shape[0]),
        "train_seeds": train_seeds, "eval_seeds": eval_seeds, "coarse_steps": steps,
        "train_steps": train_steps, "batch": batch, "lr": lr, "input_noise": noise,
        "loss_first": hist[0][1], "loss_last": hist[-1][1], "loss_history": hist,
        "train_loss_initial_mean": loss0, "train_loss_final_mean": loss1,
        "seconds_data": t_data, "seconds_train": t_train,
        "rel_l2_u_plain": mean(ev["plain_u"]), "rel_l2_u_corrected": mean(ev["corrected_u"]),
        "rel_l2_lnrho_plain": mean(ev["plain_lnrho"]),
        "rel_l2_lnrho_corrected": mean(ev["corrected_lnrho"]),
        "ms_fine_total": ev["ms_fine"], "ms_plain_total": ev["ms_plain"],
        "ms_corrected_total": ev["ms_corrected"], "error_curves": ev["curve"],
        "device_ms_per_step": dev,
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--fine", type=int, default=256)
    ap.add_argument("--ratio", type=int, default=4)
    ap.add_argument("--train-seeds", type=int, default=200)
    ap.add_argument("--eval-seeds", type=int, default=20)
    ap.add_argument("--nsnap", type=int, default=10)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--train-steps", type=int, default=4000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=3e-4)
    ap.add_argument("--k2", type=int, default=8)
    ap.add_argument("--noise", type=float, default=1.0)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    res = run(a.fine, a.ratio, a.train_seeds, a.eval_seeds, a.nsnap, None, a.steps,
              a.train_steps, a.batch, a.lr, k2=a.k2, noise=a.noise)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text + "\n")
    print(json.dumps({k: v for k, v in res.items() if k not in ("loss_history", "error_curves")}))


if __name__ == "__main__":
    main()
