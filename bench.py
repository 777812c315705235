"""Benchmark: RK3 grid-point updates per second on a 256^3 periodic box.

One benchmark step = one full RK3 step (three fused 55-point substeps,
Algorithm 2) of a 256^3 box, FP32 (the headline), on synthetic input of the
paper's kind: velocity with a k^-2 spectrum over 1 <= k <= 8 at rms Mach 0.1,
lnrho perturbation 1e-3, entropy 0 (seed 1 + rank).  The same line carries
the FP64 and 19-point forms, the precision form, an end-to-end number
through the public API with host buffers, the roofline of the dominant
kernel and the CPU oracle timed on the host's cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) every rank steps its own independent box (weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
import argparse
import glob
import hashlib
import re
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 256
SHAPE = (N, N, N)
NF = 5
METRIC = "RK3 grid-point updates/s (FP32 vs FP64) and fraction of HBM roofline"
UNIT = "updates/s"
WORKLOAD = ("256^3 periodic box, c_s=1, nu=5e-3, k^-2 velocity spectrum 1<=k<=8 at rms Mach 0.1 "
            "(seed 1+rank), lnrho 1e-3, entropy 0; one step = one RK3 step (3 substeps), dt from CFL 0.4")
# Algorithmic HBM bytes per point per RK3 step, 55-point form, F fields of w
# bytes: substep 1 reads u and writes u_out, w (alpha_1 = 0: w not read);
# substep 2 reads u, w, writes u_out, w; substep 3 reads u, w, writes u_out
# (w is dead afterwards): 10 F w.
ALG_BYTES_55 = {4: 10 * NF * 4, 8: 10 * NF * 8}
# 19-point form (Algorithm 3): per substep pass 1 reads u (F) [+ w], writes
# u_out (F), w, div (1); pass 2 reads div, u_out (3) [+ w (3)], writes u_out
# (3) [+ w (3)]; w neither read in substep 1 nor written in substep 3:
# (16 + 13) + (21 + 13) + (16 + 7) = 86 values.
ALG_VALUES_19 = 86
# Algorithmic flops per point per substep of the 55-point right-hand side and
# update as written in stencil.cuh / common.cuh (FMA = 2): 15 first
# derivatives x 8, 9 second derivatives x 10, 6 bidiagonal mixed x 14,
# Laplacian and grad-div sums 12, physics of Eqs. 1-3 with passive entropy 87,
# Eq. 10 update 5 fields x 5 = 418.
FLOPS_55_SUBSTEP = 418
FP64_NOMINAL_TFLOPS = 1.25  # GB300 FP64 (non-tensor), nominal (context; the peak is measured)


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ------------------------------------------------------------------ helpers

def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured", d
    return 6800.0, "fallback", {}


def kernel_source_sha():
    """Fingerprint of the code the headline kernel is compiled from (comments
    and whitespace removed): the FP32 tiled translation unit with every
    header it includes (followed recursively), and the tile table."""
    d = os.path.join(ROOT, "paper_1707_08900_gb300", "csrc")
    files = []

    def walk(f):
        if f in files:
            return
        files.append(f)
        for line in open(f):
            m = re.match(r'\s*#include\s+"([^"]+)"', line)
            if m:
                p = os.path.normpath(os.path.join(os.path.dirname(f), m.group(1)))
                if os.path.exists(p):
                    walk(p)

    walk(os.path.join(d, "tiled_f32.cu"))
    walk(os.path.join(d, "tiled_common.cu"))
    h = hashlib.sha256()
    for f in sorted(files):
        # the code only: comments and whitespace do not change a kernel
        text = open(f).read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
        text = re.sub(r"//[^\n]*", " ", text)
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]


def profile_summary(kernel_key):
    """Key-value lines of the committed ncu summary for kernel_key, or None
    when it is missing or was taken on different kernel sources."""
    sha = kernel_source_sha()
    for f in glob.glob(os.path.join(ROOT, "profiles", "*.txt")):
        kv = {}
        for line in open(f):
            if ":" in line:
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        if kv.get("bench_key") == kernel_key and kv.get("source_sha", "").split(" ")[0] == sha:
            return kv
    return None


def profile_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu summary (None as above)."""
    kv = profile_summary(kernel_key)
    try:
        return float(kv["dram_bytes_per_launch_scaled"]) if kv else None
    except (KeyError, ValueError):
        return None


def profile_dram_gbs(kernel_key):
    """ncu's own achieved DRAM rate: the summary's bytes per launch over its
    mean launch duration (both from the same capture), or None."""
    kv = profile_summary(kernel_key)
    try:
        return (float(kv["dram_bytes_per_launch_scaled"]) /
                (float(kv["ncu_duration_us_mean"].split()[0]) * 1e-6) / 1e9) if kv else None
    except (KeyError, ValueError, ZeroDivisionError):
        return None


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()
        time.sleep(0.5)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self):
        return time.time()

    def stop(self, t0, t1):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"],
                    "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = [l for (t, l) in self.lines if t0 - 0.15 <= t <= t1 + 0.15]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            parts = [p.strip() for p in r.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid_for(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev)


def flush_l2(buf):
    buf.zero_()


# ------------------------------------------------------------------ ranks

def max_over_ranks(v, world, dist=None, device=None):
    """Max of a per-rank scalar over all ranks (the slowest rank's time)."""
    if world == 1:
        return v
    import torch
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(points_per_rank, steps, ms_max, world):
    """Updates/s of the whole job: every rank advances its own box (weak
    scaling), the job takes as long as its slowest rank."""
    return world * points_per_rank * steps / (ms_max * 1e-3)


# ------------------------------------------------------------------ our arm

def timed_steps(s, dt, steps, stream, torch):
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    l0 = s.launches()
    ev0.record(stream)
    s.rk3_step(dt, steps)
    ev1.record(stream)
    ev1.synchronize()
    return ev0.elapsed_time(ev1), s.launches() - l0


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_1707_08900_gb300 import build as gb
    from paper_1707_08900_gb300 import gbfd, inputs

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    if rank == 0:
        gb.build()
    if world > 1:
        dist.barrier()
    gbfd.load()

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks_(v):
        return max_over_ranks(v, world, dist, dev)

    stream = torch.cuda.current_stream(dev)
    peak_gbs, peak_kind, peaks = measured_peaks()
    st0 = inputs.spectrum(SHAPE, 1 + rank, p=-2.0, k1=1, k2=8, mach=0.1, lnrho_rms=1e-3)
    st0_32 = st0.astype(np.float32)
    npts = N ** 3

    def make(precision, form):
        s = gbfd.Solver(SHAPE, precision=precision, form=form, entropy_mode=1, nu=5e-3, cs=1.0,
                        device=dev, stream=stream)
        s.set_state(st0_32 if precision != "fp64" else st0)
        return s

    # ---- headline: FP32, 55-point, fused single pass
    s = make("fp32", "55p")
    dt = s.cfl_dt(0.4)
    s.rk3_step(dt, args.warmup)
    torch.cuda.synchronize()
    sampler = ClockSampler(gpu_uuid_for(local))
    if rank == 0:
        sampler.start()
    barrier()
    torch.cuda.synchronize()
    t0 = time.time()
    ms, launches = timed_steps(s, dt, args.steps, stream, torch)
    t1 = time.time()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop(t0, t1) if rank == 0 else None
    ms_max = max_over_ranks_(ms)
    value = whole_job_rate(npts, args.steps, ms_max, world)
    avg_launch_s = ms * 1e-3 / launches
    alg_per_launch = npts * ALG_BYTES_55[4] / 3.0
    achieved = alg_per_launch / avg_launch_s / 1e9
    traffic = profile_traffic("substep55_fp32_lag_tmem_256")
    ncu_gbs = profile_dram_gbs("substep55_fp32_lag_tmem_256")
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak_gbs, "unit": "GB/s",
                "frac": round(achieved / peak_gbs, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": "k_substep_lag<float,5,55p,32x8,packed,U=2,TMEM,substep s,whole tiles> (3 launches per step, one instantiation per RK3 substep)",
                "alg_bytes_per_launch": alg_per_launch,
                "frac_of_8TBs_nominal": round(achieved / 8000.0, 4),
                # each field read and written once per substep (12 F w per
                # step, the literal count) instead of the 10 F w the kernel needs
                "frac_literal_12Fw": round(achieved * 1.2 / peak_gbs, 4),
                # ncu's DRAM bytes over ncu's launch time, same capture
                "ncu_dram_gbs": round(ncu_gbs, 1) if ncu_gbs else None,
                "ncu_dram_frac_of_8TBs": round(ncu_gbs / 8000.0, 4) if ncu_gbs else None}
    s.close()

    extra = {}
    # ---- the same kernel at 512^3 on the 512^3 workload's state (k^-5/3
    # over 1 <= k <= 16, rms Mach 0.3, seed 2, lnrho 1e-2): the HBM fraction
    # at the second size
    n5 = 512
    st5 = inputs.spectrum((n5,) * 3, 2 + rank, p=-5.0 / 3.0, k1=1, k2=16, mach=0.3,
                          lnrho_rms=1e-2).astype(np.float32)
    s5 = gbfd.Solver((n5,) * 3, precision="fp32", form="55p", entropy_mode=1, nu=5e-3, cs=1.0,
                     device=dev, stream=stream)
    s5.set_state(st5)
    del st5
    dt5 = s5.cfl_dt(0.4)
    s5.rk3_step(dt5, 3)
    torch.cuda.synchronize()
    k5 = max(5, min(args.steps // 50, 40))
    ms5, _ = timed_steps(s5, dt5, k5, stream, torch)
    ms5 = max_over_ranks_(ms5)
    extra["fp32_55p_512"] = {
        "value": world * n5 ** 3 * k5 / (ms5 * 1e-3), "steps": k5, "ms_per_step": ms5 / k5,
        "hbm_frac": round(n5 ** 3 * ALG_BYTES_55[4] / (ms5 / k5 * 1e-3) / 1e9 / peak_gbs, 4),
        "frac_of_8TBs_nominal": round(n5 ** 3 * ALG_BYTES_55[4] / (ms5 / k5 * 1e-3) / 1e9 / 8000.0, 4),
        "state": "k^-5/3 over 1<=k<=16, rms Mach 0.3, seed 2, lnrho 1e-2"}
    s5.close()
    # ---- FP64, 55-point (FP64-ALU bound on GB300)
    k64 = max(3, args.steps // 20)
    s = make("fp64", "55p")
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    ms64, l64 = timed_steps(s, dt, k64, stream, torch)
    v64 = npts * k64 / (max_over_ranks_(ms64) * 1e-3)  # per GPU
    tflops64 = v64 * 3 * FLOPS_55_SUBSTEP / 1e12
    # the FP64 pipe's own rate on this GPU: independent FMA chains on every SM
    fp64_peak = gbfd.gbfd_fp64_fma_rate(stream.cuda_stream)
    extra["fp64_55p"] = {
        "value": world * v64, "steps": k64, "ms_per_step": ms64 / k64,
        "roofline": {"bound": "alu", "achieved": round(tflops64, 3), "peak": round(fp64_peak, 3),
                     "unit": "TFLOP/s", "frac": round(tflops64 / fp64_peak, 4),
                     "peak_kind": "measured (gbfd_fp64_fma_rate: independent FP64 FMA chains "
                                  "on every SM, FMA = 2 flop)",
                     "frac_of_nominal_1p25": round(tflops64 / FP64_NOMINAL_TFLOPS, 4),
                     "flops_per_update": 3 * FLOPS_55_SUBSTEP},
        "hbm_frac": round(npts * ALG_BYTES_55[8] / (ms64 / k64 * 1e-3) / 1e9 / peak_gbs, 4),
    }
    # error of the FP32 forms against this FP64 run: same initial state, same steps
    ref64 = s.get_state()
    s.close()
    nerr = 2 + k64
    errs = {}
    for prec in ("fp32", "fp32_acc64", "fp32_accff"):
        s2 = make(prec, "55p")
        s2.rk3_step(dt, nerr)
        x = s2.get_state()
        s2.close()
        errs[prec] = [float(np.linalg.norm((x[f] - ref64[f]).ravel())
                            / np.linalg.norm(ref64[f].ravel())) for f in range(4)]
    del ref64
    # the 19-point form the same way: FP32 against FP64, both 19-point
    s19 = make("fp64", "19p")
    s19.rk3_step(dt, nerr)
    ref19 = s19.get_state()
    s19.close()
    s2 = make("fp32", "19p")
    s2.rk3_step(dt, nerr)
    x = s2.get_state()
    s2.close()
    errs19 = [float(np.linalg.norm((x[f] - ref19[f]).ravel()) / np.linalg.norm(ref19[f].ravel()))
              for f in range(4)]
    del ref19, x
    extra["error_vs_fp64"] = {"steps": nerr, "grid": "256^3",
                              "rel_l2_lnrho_ux_uy_uz": errs,
                              "rel_l2_lnrho_ux_uy_uz_19p": {"fp32": errs19}}
    extra["fp32_vs_fp64_speedup"] = round(value / world / v64, 2)

    # ---- FP32, 19-point two-pass form
    k19 = max(3, args.steps // 4)
    s = make("fp32", "19p")
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    ms19, l19 = timed_steps(s, dt, k19, stream, torch)
    v19 = npts * k19 / (max_over_ranks_(ms19) * 1e-3)
    extra["fp32_19p"] = {
        "value": world * v19, "steps": k19, "ms_per_step": ms19 / k19,
        "hbm_frac_own_ideal": round(npts * ALG_VALUES_19 * 4 / (ms19 / k19 * 1e-3) / 1e9
                                    / peak_gbs, 4),
        "hbm_frac_55p_ideal": round(npts * ALG_BYTES_55[4] / (ms19 / k19 * 1e-3) / 1e9
                                    / peak_gbs, 4),
    }
    s.close()

    # ---- forced (Sect. 6, Eqs. 20-21): a new k, phi, e every step from the
    # isotropic set 1 <= |k| <= 2 (k_f = 1.53); the paper's forcing runs use
    # the 19-point form at 256^3 with nu = 1.4e-4
    kfo = max(3, args.steps // 8)
    fks, fphis, fes = inputs.forcing_sequence(17 + rank, kfo + 2, kmin=1.0, kmax=2.0)
    for form_f in ("19p", "55p"):
        s = gbfd.Solver(SHAPE, precision="fp32", form=form_f, entropy_mode=1, nu=1.4e-4, cs=1.0,
                        device=dev, stream=stream)
        s.set_state(st0_32)
        s.rk3_step_forced(dt, 0.02, fks[:2], fphis[:2], fes[:2])
        torch.cuda.synchronize()
        evf0 = torch.cuda.Event(enable_timing=True)
        evf1 = torch.cuda.Event(enable_timing=True)
        evf0.record(stream)
        s.rk3_step_forced(dt, 0.02, fks[2:], fphis[2:], fes[2:])
        evf1.record(stream)
        evf1.synchronize()
        msf = max_over_ranks_(evf0.elapsed_time(evf1))
        extra[f"fp32_{form_f}_forced"] = {
            "value": world * npts * kfo / (msf * 1e-3), "steps": kfo, "ms_per_step": msf / kfo,
            "forcing": "k from 1 <= |k| <= 2 (k_f 1.53), f0 0.02, nu 1.4e-4, new k/phi/e per step"}
        s.close()

    # ---- radial explosion (Sect. 6, Eq. 19): seven-axis asymmetry at t = 0.5,
    # nu = 1e-3 (Re = u_ampl d_shell / nu = 200), both stencil forms
    from paper_1707_08900_gb300 import explosion
    for form_e in ("55p", "19p"):
        ex = explosion.run(n=SHAPE[0], nu=1e-3, t_end=0.5, precision="fp32", form=form_e,
                           samples=1)
        extra[f"explosion_{form_e}"] = {"Re": ex["Re"], "t": ex["history"][-1]["t"],
                                        "steps": ex["steps"],
                                        "delta_sum_rho": ex["history"][-1]["delta_rho"],
                                        "delta_sum_u": ex["history"][-1]["delta_u"]}

    # ---- walls in z (the ghost-zone boundary variant, Sect. 4): the same
    # box bounded by free-slip walls through its first and last planes; the
    # ghost planes are refilled after every substep
    kw = max(3, args.steps // 8)
    stw = st0_32.copy()
    stw[3, 0] = 0.0
    stw[3, -1] = 0.0  # no flow through the walls
    s = gbfd.Solver(SHAPE, precision="fp32", form="55p", entropy_mode=1, nu=5e-3, cs=1.0,
                    device=dev, stream=stream, bc_z="wall")
    s.set_state(stw)
    del stw
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    msw, lw = timed_steps(s, dt, kw, stream, torch)
    extra["fp32_55p_wall"] = {"value": world * npts * kw / (max_over_ranks_(msw) * 1e-3),
                              "steps": kw, "ms_per_step": msw / kw,
                              "launches_per_step": lw / kw,
                              "what": "z bounded by free-slip walls, ghost planes refilled "
                                      "after every substep"}
    s.close()

    # ---- the headline kernel with its x neighbours exchanged by warp shuffles
    # (tile table entry 30: the same kernel, z-chunk and grid as the default
    # entry, paired shared loads replaced by shuffles and halo quads)
    ksh = max(3, args.steps // 8)
    s = make("fp32", "55p")
    s.set_option(gbfd.GBFD_OPT_TILE_CONFIG, 30)
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    mssh, _ = timed_steps(s, dt, ksh, stream, torch)
    extra["fp32_55p_shfl"] = {"value": world * npts * ksh / (max_over_ranks_(mssh) * 1e-3),
                              "steps": ksh, "ms_per_step": mssh / ksh,
                              "what": "default kernel with warp-shuffle x neighbours "
                                      "(tile table entry 30)"}
    s.close()

    # ---- precision form: FP32 stencil, FP64 RK3 registers
    kacc = max(3, args.steps // 4)
    s = make("fp32_acc64", "55p")
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    msa, _ = timed_steps(s, dt, kacc, stream, torch)
    extra["fp32_acc64_55p"] = {"value": world * npts * kacc / (max_over_ranks_(msa) * 1e-3),
                               "steps": kacc, "ms_per_step": msa / kacc}
    s.close()
    # ---- the same update in float-float FP32 pairs (Dekker / Knuth
    # error-free products and sums) on the FP32 default kernel
    s = make("fp32_accff", "55p")
    s.rk3_step(dt, 2)
    torch.cuda.synchronize()
    msf, _ = timed_steps(s, dt, kacc, stream, torch)
    extra["fp32_accff_55p"] = {"value": world * npts * kacc / (max_over_ranks_(msf) * 1e-3),
                               "steps": kacc, "ms_per_step": msf / kacc}
    s.close()

    # ---- batched form: 96 boxes (32 each of 32^3, 64^3, 128^3), rms Mach
    # U(0.05, 0.3), nu U(2e-3, 1e-2), seeds 100..195, 20 RK3 steps replayed
    # from a CUDA graph, work-item chunk picked by the batch autotuner
    rng = np.random.default_rng(4 + rank)
    bns = [32] * 32 + [64] * 32 + [128] * 32
    bmach = rng.uniform(0.05, 0.3, 96)
    bnu = rng.uniform(2e-3, 1e-2, 96)
    bat = gbfd.Batch(bns, [2 * np.pi] * 96, bnu, device=dev, stream=stream)
    for i, n in enumerate(bns):
        bst = inputs.spectrum((n, n, n), 100 + i, p=-2.0, k1=1, k2=8, mach=bmach[i],
                              lnrho_rms=1e-3)
        bat.set_state(i, bst.astype(np.float32))
    bdt = [0.4 * (2 * np.pi / n) / (1.0 + bat.diagnostics(i)["umax"]) for i, n in enumerate(bns)]
    bzc, _ = bat.autotune(steps=1)
    bsteps = 20
    bat.step(bdt, bsteps)  # warm-up: captures the graph
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    bl0 = bat.launches()
    e0.record(stream)
    bat.step(bdt, bsteps)
    e1.record(stream)
    e1.synchronize()
    bms = max_over_ranks_(e0.elapsed_time(e1))
    bpts = sum(n ** 3 for n in bns)
    extra["fp32_batched_96"] = {
        "value": world * bpts * bsteps / (bms * 1e-3), "steps": bsteps, "ms_per_step": bms / bsteps,
        "boxes": "32 x 32^3 + 32 x 64^3 + 32 x 128^3", "zchunk": bzc,
        "launches_per_step": (bat.launches() - bl0) / bsteps, "graph": True,
        "hbm_frac": round(bpts * ALG_BYTES_55[4] / (bms / bsteps * 1e-3) / 1e9 / peak_gbs, 4),
    }
    bat.close()

    # ---- learned coarse-grid form: 64^3 FP32 coarse step plain vs with the
    # correction network (3 tcgen05 implicit-GEMM convolutions after every
    # RK3 step); timing only (accuracy comes from the training runs)
    from paper_1707_08900_gb300 import learned
    nc = 64
    cst = inputs.spectrum((nc,) * 3, 1200 + rank, p=-2.0, k1=1, k2=8, mach=0.1,
                          lnrho_rms=1e-3).astype(np.float32)
    cs_ = gbfd.Solver((nc,) * 3, precision="fp32", nu=5e-3, device=dev, stream=stream)
    cs_.set_state(cst)
    cdt = cs_.cfl_dt(0.4)
    net = gbfd.CNN(nc, batch=1, device=dev, stream=stream)
    net.set_params(learned.init_params(0))
    csteps = max(10, args.steps // 10)
    cs_.rk3_step(cdt, 3)
    net.step_corrected(cs_, cdt, 3)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    ev[0].record(stream)
    cs_.rk3_step(cdt, csteps)
    ev[1].record(stream)
    net.step_corrected(cs_, cdt, csteps)
    ev[2].record(stream)
    ev[2].synchronize()
    ms_plain = max_over_ranks_(ev[0].elapsed_time(ev[1])) / csteps
    ms_corr = max_over_ranks_(ev[1].elapsed_time(ev[2])) / csteps
    # tensor-core work of one network application: 2 M K N flop per conv
    # (K = 27 x padded input channels, N = padded output channels)
    cnn_flop = 2 * nc ** 3 * (27 * 16 * 32 + 27 * 32 * 32 + 27 * 32 * 16)
    extra["fp32_learned_64"] = {
        "plain_ms_per_step": ms_plain, "corrected_ms_per_step": ms_corr,
        "network_ms_per_application": ms_corr - ms_plain,
        "network_tensor_tflops": cnn_flop / ((ms_corr - ms_plain) * 1e-3) / 1e12,
        "value_corrected": world * nc ** 3 / (ms_corr * 1e-3), "steps": csteps,
        # SM cycles per tcgen05 MMA (M = 128, K = 16) against N: the
        # convolutions stack their three z taps along N (96 / 48 columns)
        "tc_mma_cycles": {str(nn): round(gbfd.gbfd_tc_mma_cycles(nn, stream.cuda_stream), 1)
                          for nn in (32, 48, 96, 128, 256)},
    }
    net.close()
    cs_.close()

    # ---- end to end through the public API with pinned host buffers:
    # every step copies the state in (H2D), advances one RK3 step and reads
    # the new state back (D2H).  Sequential: one context, each call after the
    # previous one has finished.
    s = make("fp32", "55p")
    host_in = torch.from_numpy(st0_32).pin_memory()
    # one trajectory: the state makes the round trip through host memory
    # every step (step n's result is step n + 1's input)
    host_io = host_in.clone().pin_memory()
    ke = max(3, min(args.steps, 50))
    for _ in range(2):
        s.set_state(host_io)
        s.rk3_step(dt, 1)
        s.get_state(out=host_io)
    host_io.copy_(host_in)
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    for _ in range(ke):
        gbfd.gbfd_set_state(s.ctx, host_io.data_ptr(), 0, 0)
        gbfd.gbfd_rk3_step(s.ctx, dt, 1)
        gbfd.gbfd_get_state(s.ctx, host_io.data_ptr(), 0, 0)  # synchronises
    te = time.perf_counter() - te0
    te = max_over_ranks_(te)
    state_bytes = host_in.numel() * host_in.element_size()
    e2e = {"value": world * npts * ke / te, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes, "steps": ke, "ms_per_step": te / ke * 1e3,
           "what": "one trajectory through the public API: per step gbfd_set_state from a "
                   "pinned host FP32 buffer, gbfd_rk3_step(dt,1), gbfd_get_state back into the "
                   "same buffer (the next step's input), one context, each call waiting for the "
                   "last; overlapped independent steps in forms.e2e_overlapped"}
    s.close()
    # Pipelined: the steps are independent (each uploads the same input), so
    # NCTX contexts on NCTX streams take them in turn; the copies go through
    # the copy engines (GBFD_OPT_HOST_PATH = 1) and gbfd_get_state only
    # enqueues its copy (GBFD_OPT_HOST_ASYNC = 1), so one step's download, the
    # next one's upload and a third one's RK3 step overlap.  All streams are
    # waited for inside the timed region.
    NCTX = 3
    pstreams = [torch.cuda.Stream(dev) for _ in range(NCTX)]
    pctx = []
    for k in range(NCTX):
        sk = gbfd.Solver(SHAPE, precision="fp32", form="55p", entropy_mode=1, nu=5e-3, cs=1.0,
                         device=dev, stream=pstreams[k])
        sk.set_option(gbfd.GBFD_OPT_HOST_PATH, 1)
        sk.set_option(gbfd.GBFD_OPT_HOST_ASYNC, 1)
        pctx.append(sk)
    pouts = [torch.empty_like(host_in).pin_memory() for _ in range(NCTX)]

    def pipelined(n):
        for i in range(n):
            sk = pctx[i % NCTX]
            gbfd.gbfd_set_state(sk.ctx, host_in.data_ptr(), 0, 0)
            gbfd.gbfd_rk3_step(sk.ctx, dt, 1)
            gbfd.gbfd_get_state(sk.ctx, pouts[i % NCTX].data_ptr(), 0, 0)
        for sk in pctx:
            sk.sync()

    pipelined(2 * NCTX)
    barrier()
    torch.cuda.synchronize()
    te0 = time.perf_counter()
    pipelined(ke)
    tp = max_over_ranks_(time.perf_counter() - te0)
    extra["e2e_overlapped"] = {
        "value": world * npts * ke / tp, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
        "d2h_bytes_per_step": state_bytes, "steps": ke, "ms_per_step": tp / ke * 1e3,
        "what": f"independent steps (each uploads the same input, not one trajectory): per step "
                f"gbfd_set_state from pinned host FP32, gbfd_rk3_step(dt,1), gbfd_get_state to "
                f"pinned host FP32; {NCTX} contexts on {NCTX} streams take the steps in turn "
                f"(copies by the copy engines, get_state asynchronous), so neighbouring steps' "
                f"copies and compute overlap"}
    for sk in pctx:
        sk.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(target_s=args.cpu_seconds)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "256^3", "form": "55-point fused",
                   "precision": "fp32", "fields": NF, "tile": "default (32x8, two points per thread, packed FP32x2, output lagged 3 planes with pending RHS in TMEM, isotropic weights, z-chunks of 40 planes)",
                   "l2": "inputs larger than L2: 3 x 335 MB padded FP32 state buffers",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "forms": extra,
        "impl": "ours",
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ------------------------------------------------------------------ CPU oracle

def _oracle_sample(nyz, threads):
    from oracle import fd
    from paper_1707_08900_gb300 import inputs
    ny, nz = nyz
    fd.set_threads(threads)
    shape = (nz, ny, N)
    st = inputs.spectrum(shape, 1, p=-2.0, k1=1, k2=8, mach=0.1, lnrho_rms=1e-3)
    h = 2 * np.pi / N
    g = fd.Grid(N, ny, nz, 2 * np.pi, h * ny, h * nz)
    ph = fd.Physics(cs=1.0, nu=5e-3, entropy_mode=1)
    return fd, st, g, ph


def cpu_baseline(target_s=15.0):
    """The FP64 C oracle as it stands, OpenMP over z on all host cores: RK3
    steps on a 256 x ny x nz slab of the workload (periodic), sized to run
    for about target_s seconds."""
    threads = os.cpu_count() or 1
    fd, st, g, ph = _oracle_sample((64, 16), threads)
    t = time.perf_counter()
    fd.rk3_step(st, 1e-3, g, ph)
    per_pt = (time.perf_counter() - t) / (N * 64 * 16)
    nz = int(np.clip(target_s / (per_pt * N * N), 8, 256))
    fd, st, g, ph = _oracle_sample((N, nz), threads)
    t = time.perf_counter()
    fd.rk3_step(st, 1e-3, g, ph)
    el = time.perf_counter() - t
    return {"value": N * N * nz / el, "unit": UNIT, "cores": fd.set_threads(0), "kind": "oracle",
            "sample": f"one FP64 RK3 step (55-point) of a 256x256x{nz} slab of the workload, "
                      f"{el:.1f} s"}


def run_reference(args):
    """Reference arm: the CPU oracle on the host cores, one bounded sample
    of the workload per step."""
    if int(os.environ.get("RANK", 0)) != 0:
        return
    from oracle import build_oracle
    build_oracle.build()
    threads = os.cpu_count() or 1
    fd, st, g, ph = _oracle_sample((64, 8), threads)
    t = time.perf_counter()
    fd.rk3_step(st, 1e-3, g, ph)
    per_pt = (time.perf_counter() - t) / (N * 64 * 8)
    budget = 150.0 / (args.steps + args.warmup)  # whole run within a few minutes
    ny = int(np.clip(budget / (per_pt * N * 8), 8, 256))
    fd, st, g, ph = _oracle_sample((ny, 8), threads)
    for _ in range(args.warmup):
        fd.rk3_step(st, 1e-3, g, ph)
    t = time.perf_counter()
    for _ in range(args.steps):
        fd.rk3_step(st, 1e-3, g, ph)
    el = time.perf_counter() - t
    pts = N * ny * 8
    value = pts * args.steps / el
    sample = f"each step: one FP64 RK3 step (55-point) of a 256x{ny}x8 periodic slab of the workload"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": int(os.environ.get("WORLD_SIZE", 1)),
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": "256^3 (sampled)", "form": "55-point",
                   "precision": "fp64 oracle"},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": fd.set_threads(0), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
