"""Benchmark: projection steps of the channel-flow solver on GB300.

A step is one pass of the whole hot path: eddy viscosity (Smagorinsky with
van Driest damping), explicit terms + AB3, Crank-Nicolson sweeps, the
divergence / Poisson right-hand side, the pressure solve to 1e-8 relative
residual from the previous pressure (SRJ with z-line relaxation, FP32
sweeps inside an FP64 refinement loop), the velocity correction with the
constant-flux fix-up.  Workload: the turbulent LES channel, 256 x 128 x 192
cells with tanh-stretched walls (gamma 2), Lx = 4 pi, Ly = 2 pi, Lz = 2,
nu = 1/2800, Cs 0.1, U_b = 1, dt 1e-3, laminar start + 10 % noise (seed 1).
Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W]
  python bench.py --impl reference ...   (the CPU oracle on the host cores)

N > 1 runs under torch.distributed.run: independent replicas, one per GPU,
no data exchange ("replicas only"); the timed region is bracketed by a
barrier and the maximum over ranks is reported.
"""
import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "les_channel"
WORKLOAD_DESC = ("les_channel 256x128x192, Lx 4pi Ly 2pi Lz 2, tanh walls gamma 2, nu 1/2800 (bulk Re 5600), "
                 "Smagorinsky Cs 0.1 + van Driest A 25, constant flux U_b 1, dt 1e-3, laminar + 10% noise (seed 1); "
                 "FP32 stencils and sweeps, FP64 reductions and refinement, z-line SRJ, Poisson to 1e-8")
METRIC = "Mcell*steps/s (projection step, Poisson to 1e-8 rel. residual)"
LINE_NAMES = {1: "k_line_sweep_chunk<32,6> (z-line SRJ sweep: residual, column recurrences in registers by level "
                 "chunks, update)",
              0: "k_line_sweep_vec<float,RB> (z-line SRJ sweep: residual, twisted column solve in shared memory, "
                 "update)"}
TILE_NAMES = {0: "k_sweep_f32_z<1,8>", 1: "k_sweep_f32_z<2,8>", 2: "k_sweep_f32_z<4,8>", 3: "k_sweep_f32_z<2,4>",
              4: "k_sweep_f32_z<4,4>", 5: "k_sweep_f32_z<8,4>", 6: "k_sweep_f32_flat<2>", 7: "k_sweep_f32_flat<4>",
              8: "k_sweep_f32_flat<8>", 9: "k_sweep_f32_pair<8,4>", 10: "k_sweep_f32_pair<4,4>",
              11: "k_sweep_f32_pair<4,8>"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, choices=["les_channel", "os_instability"],
                    help="headline workload (profiling runs may pick the instability case)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"], help="profiling runs only")
    ap.add_argument("--solver", default="zline", choices=["zline", "point"], help="profiling runs only")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--grid", default=None, help="override the cell counts, NXxNYxNZ (profiling runs)")
    ap.add_argument("--only-headline", action="store_true", help="skip every side measurement (profiling runs)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-guess comparison")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched uneven-channel measurement")
    ap.add_argument("--no-les", action="store_true", help="skip the paper's LES workload")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the point-SRJ, instability-workload and above-L2 sweep measurements")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def reduce_max(value, device=None):
    """Maximum of a per-rank scalar over all ranks (identity on one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def source_digest(files):
    """sha256 over the given source files under the package's csrc/: the
    traffic figures of a kernel apply while the sources defining it are
    unchanged."""
    csrc = os.path.join(ROOT, "paper_1511_07800_gb300", "csrc")
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def traffic_for(key):
    """Per-launch DRAM bytes (read + write) of a kernel from the committed
    ncu summary profiles/kernel_traffic.json, scaled to the launch's cells
    when the capture was on a smaller grid; None when the kernel's sources
    changed since the capture or no record exists."""
    path = os.path.join(ROOT, "profiles", "kernel_traffic.json")
    try:
        rec = json.load(open(path))["kernels"][key]
        if rec["source_sha256"] != source_digest(rec["sources"]):
            return None
        return rec
    except Exception:
        return None


def cpu_baseline_sample(cfg, fields, sweeps_per_step, omega):
    """The CPU oracle on the host cores: one step of the same workload from
    the same initial fields, its pressure solve held to the GPU's mean sweep
    count per step in whole cycles (the same work per step)."""
    import oracle
    ncores = len(os.sched_getaffinity(0))
    oracle.set_threads(ncores)
    M = len(omega)
    cycles = max(1, int(round(sweeps_per_step / M)))
    o = oracle.Oracle(dict(cfg, omega=omega, ptol=0.0, pmaxit=cycles * M, cn_sweeps=cfg["cn_sweeps"]))
    o.set_fields(*fields)
    t0 = time.perf_counter()
    o.step(1)
    dt = time.perf_counter() - t0
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    return {"value": cells / dt / 1e6, "unit": "Mcell*steps/s", "cores": oracle.get_threads(), "kind": "oracle",
            "sample": "1 FP64 oracle step of the full %dx%dx%d workload from the initial fields, %s SRJ held to "
                      "%d sweeps (%d cycles of %d, the GPU's mean per timed step); %.2f s wall"
                      % (cfg["nx"], cfg["ny"], cfg["nz"], "z-line" if cfg.get("zline") else "point", cycles * M,
                         cycles, M, dt)}


def _oracle_threads():
    import oracle
    oracle.set_threads(len(os.sched_getaffinity(0)))
    return oracle.get_threads()


def oracle_us_per_sweep(cfg, zline, seed=5):
    """The oracle's time per SRJ sweep (point or z-line) on the grid of cfg,
    on the host cores.  The oracle tests its sweep cap once per cycle, so
    this times one and three whole cycles of a fixed 32-weight schedule
    from the same seeded start, after a warm-up cycle, each the fastest of
    three runs (other work on the host cores only adds time): the
    difference is 64 sweeps and two residual evaluations (the set-up
    cancels)."""
    import numpy as np

    import oracle
    o = oracle.Oracle(dict(cfg, omega=[0.8, 1.0] * 16, zline=zline))
    rng = np.random.default_rng(seed)
    shape = (cfg["nz"], cfg["ny"], cfg["nx"])
    b = rng.standard_normal(shape)
    p0 = rng.standard_normal(shape) * 0.1
    o.poisson(b, p0, tol=0.0, maxit=1)
    t = {}
    for n in (32, 96):
        best = float("inf")
        for _ in range(3):
            t0 = time.perf_counter()
            _, it, _, _ = o.poisson(b, p0, tol=0.0, maxit=n)
            best = min(best, time.perf_counter() - t0)
            assert it == n
        t[n] = best
    return 1e6 * (t[96] - t[32]) / 64


def learned_comparison(cfg, steps, oracle_sample=True):
    """Poisson time to 1e-8, learned against plain, on the workload grid:
    train the U-Net on (residual, correction) pairs harvested from channels
    of the same workload (seeds 0-9, 60 steps each), then step two unseen
    channels (seeds 7 and 50, each with its own random mode amplitude and
    noise level) plainly, with the network as the initial guess of every
    solve and with it as a preconditioner at every refinement pass (FP32)
    or SRJ cycle (FP64), and compare the solves.  A mode's speed-up is the
    geometric mean over the two channels."""
    import numpy as np
    import torch
    from paper_1511_07800_gb300 import learn, stp
    shape = (cfg["nz"], cfg["ny"], cfg["nx"])
    t0 = time.perf_counter()
    R, DP = learn.harvest(cfg, seeds=range(10), steps_per_seed=60)
    K = learn.output_scale(R, DP, 4, shape)
    net = stp.UNet(4, *shape)
    theta = learn.he_init(0)
    net.set_params(theta)
    net.set_output_scale(K)
    losses = learn.train(net, R, DP, 1500, 4, 1e-3) + learn.train(net, R, DP, 500, 4, 3e-4)
    t_train = time.perf_counter() - t0
    npairs = int(R.shape[0])
    del R, DP
    torch.cuda.empty_cache()
    one = stp.UNet(1, *shape)
    one.set_params(net.get_params())
    one.set_output_scale(K)
    net.close()
    net = one
    eval_seeds = (7, 50)
    res = {sd: learn.compare_modes(cfg, net, seed=sd, nsteps=max(3, min(steps, 8)), precision="fp32")
           for sd in eval_seeds}
    res64 = {sd: learn.compare_modes(cfg, net, seed=sd, nsteps=8, precision="fp64") for sd in eval_seeds}

    def gmean(runs, mode):
        return float(np.exp(np.mean([np.log(r[mode]["speedup"]) for r in runs.values()])))
    # one forward of the trained network on the workload grid (CUDA events)
    fwd_ms = None
    try:
        xg = torch.randn((1,) + shape, device="cuda")
        yg = torch.zeros_like(xg)
        for _ in range(2):
            net.forward(xg, yg)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            net.forward(xg, yg)
        e1.record()
        e1.synchronize()
        fwd_ms = e0.elapsed_time(e1) / 5
    except Exception as ex:  # report, never fake
        fwd_ms = {"error": str(ex)[:200]}
    net.close()
    out_cpu = None
    if oracle_sample:
        try:
            # the oracle network (FP64 numpy) on one eighth of the voxels, scaled
            from oracle import unet as unet_oracle
            half = tuple(n // 2 for n in shape)
            xs = np.random.default_rng(11).standard_normal((1,) + half + (1,))
            t1 = time.perf_counter()
            unet_oracle.forward(theta.astype(np.float64), xs)
            t_s = time.perf_counter() - t1
            out_cpu = {"kind": "oracle", "unit": "ms per forward", "value": 8e3 * t_s,
                       "sample": "one FP64 oracle forward at %dx%dx%d (an eighth of the voxels, %.2f s), scaled "
                                 "by voxels to %dx%dx%d" % (half[2], half[1], half[0], t_s, shape[2], shape[1],
                                                            shape[0])}
        except Exception as ex:  # report, never fake
            out_cpu = {"value": None, "error": str(ex)[:200]}
    by_mode = {"fp64_guess": gmean(res64, "guess"), "fp64_preconditioner": gmean(res64, "precond"),
               "fp32_guess": gmean(res, "guess"), "fp32_preconditioner": gmean(res, "precond")}
    return {"speedup_by_mode": by_mode, "speedup": max(by_mode.values()),
            "forward_ms": fwd_ms, "fp32": {"seed_%d" % sd: r for sd, r in res.items()},
            "fp64": {"seed_%d" % sd: r for sd, r in res64.items()},
            "train": {"pairs": npairs, "adam_steps": len(losses), "batch": 4,
                      "final_loss": float(np.mean(losses[-10:])), "output_scale": K, "seconds": t_train},
            "cpu_baseline": out_cpu,
            "note": "time per pressure solve to 1e-8 (GPU events) on two unseen channels of the instability "
                    "workload (128x64x128), previous-step pressure as the plain guess; guess: the network once per "
                    "solve; precond: at every refinement pass (FP32) or SRJ cycle (FP64); a mode's speed-up is the "
                    "geometric mean over the channels, speedup the best mode. The 20k-pair experiment is "
                    "learn.config4"}


def batched_channels(steps, warmup, peak, oracle_sample=True):
    """Uneven-channel batch: 64 instances with sizes drawn from
    {32, 48, 64, 96, 128}^3 (seed 2), Re uniform in [5000, 10000],
    Orr-Sommerfeld amplitude log-uniform in [1e-5, 1e-3], FP32 with FP64
    refinement, all advanced by one graph launch per call.  Measured grouped
    (lock-step solves, the default), with every channel on its own solve,
    and with the channels stepped one after another; GPU time by CUDA events
    around the launch."""
    import torch
    from paper_1511_07800_gb300 import inputs, stp
    inst = inputs.batched_instances(count=64, seed=2)
    cells = sum(c["nx"] * c["ny"] * c["nz"] for c, _ in inst)
    chans = []
    for cfg, f in inst:
        ch = stp.Channel(cfg, precision="fp32")
        ch.set_fields(*f)
        chans.append(ch)
    out = {"instances": len(chans), "cells": cells, "precision": "fp32", "steps": steps,
           "warmup": max(3, warmup), "l2": "working set of the 64 channels (about 3 GB) far above L2",
           "data": "synthetic (seeded)"}
    saved = os.environ.get("STP_BATCH_GROUPS")
    try:
        for mode, env in (("ungrouped", "0"), ("grouped", "1")):
            os.environ["STP_BATCH_GROUPS"] = env
            b = stp.Batch(chans)
            b.step(max(3, warmup))
            st = b.step(steps)
            r = {"value": cells * steps / (st["gpu_ms"] / 1e3) / 1e6, "unit": "Mcell*steps/s",
                 "ms_per_step": st["gpu_ms"] / steps, "gpu_launches": st["kernels"],
                 "sweeps_per_step": st["sweeps"] / steps, "converged": st["converged"]}
            if mode == "grouped":
                last_sweeps = [c["sweeps"] for c in st["channels"]]
                groups = b.groups()
                r["groups"] = groups
                g = max(groups, key=lambda x: x["cells"]) if groups else None
                if g and g["sweep_us"] > 0:
                    ach = 12.0 * g["cells"] / (g["sweep_us"] * 1e-6) / 1e9
                    r["roofline"] = {"bound": "hbm", "kernel": "kg_sweep (grouped FP32 SRJ sweep, largest group)",
                                     "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                     "traffic": None, "bytes_per_launch": 12 * g["cells"],
                                     "mean_launch_us": g["sweep_us"],
                                     "note": "autotuner's timing: 20 back-to-back grouped sweeps, all channels active"}
            out[mode] = r
            b.close()
    finally:
        if saved is None:
            os.environ.pop("STP_BATCH_GROUPS", None)
        else:
            os.environ["STP_BATCH_GROUPS"] = saved
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for ch in chans:
        ch.step(steps)
    ts = time.perf_counter() - t0
    out["sequential"] = {"value": cells * steps / ts / 1e6, "unit": "Mcell*steps/s",
                         "note": "each channel stepped on its own, one after another (wall clock)"}
    for ch in chans:
        ch.close()
    if oracle_sample:
        import oracle
        from oracle import srj
        cores = _oracle_threads()
        cells_o, t_o, held = 0, 0.0, []
        for (cfg, f), s_gpu in list(zip(inst, last_sweeps))[:4]:
            om, _, _ = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"],
                                        cfg.get("stretch", 0.0))
            n = max(1, int(round(s_gpu / len(om)))) * len(om)
            o = oracle.Oracle(dict(cfg, omega=om, ptol=0.0, pmaxit=n))
            o.set_fields(*f)
            t0 = time.perf_counter()
            o.step(1)
            t_o += time.perf_counter() - t0
            cells_o += cfg["nx"] * cfg["ny"] * cfg["nz"]
            held.append("%dx%dx%d:%d" % (cfg["nx"], cfg["ny"], cfg["nz"], n))
        out["cpu_baseline"] = {
            "kind": "oracle", "cores": cores, "value": cells_o / t_o / 1e6, "unit": "Mcell*steps/s",
            "sample": "one FP64 oracle step of each of the first 4 instances from their start fields, each solve "
                      "held to its channel's GPU sweep count of the last grouped step in whole cycles "
                      "(grid:sweeps %s); %.2f s" % (", ".join(held), t_o)}
    return out


def les_paper_steps(steps, warmup, oracle_sample=True):
    """The paper's LES workload (Sec. 6) at its own grid, 240 x 140 x 120,
    Lx = 8, Ly = 4, Lz = 1, Re_* = 360, dt = 1e-4, Smagorinsky + van Driest,
    FP32 with FP64 refinement, from its random Fourier-curl start; the
    plane statistics are accumulated after every step, as a run gathering
    the paper's averages would.  GPU time by CUDA events around the steps.
    The headline is the paper's point SRJ; the same run with z-line
    relaxation is reported beside it."""
    import torch
    from paper_1511_07800_gb300 import inputs, stp
    cfg = inputs.preset("les_paper")
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    stream = torch.cuda.current_stream()
    res = {}
    for zl in (0, 1):
        with stp.Channel(dict(cfg, zline=zl), precision="fp32", stream=stream.cuda_stream) as ch:
            ch.set_fields(*inputs.paper_les_initial(cfg, 1))
            ch.step(max(3, warmup))
            ch.stats_reset()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sweeps, conv = 0, True
            for _ in range(steps):
                st = ch.step(1)
                sweeps += st["sweeps"]
                conv = conv and st["converged"]
                ch.stats_accumulate()
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
        res[zl] = {"value": cells * steps / (ms / 1e3) / 1e6, "unit": "Mcell*steps/s", "ms_per_step": ms / steps,
                   "sweeps_per_step": sweeps / steps, "converged": conv}
    out = {"workload": "les_paper 240x140x120, Lx 8, Ly 4, Lz 1, Re_* 360, dt 1e-4, FP32 + FP64 refinement, "
                       "point SRJ (the paper's method), statistics every step", "steps": steps,
           "warmup": max(3, warmup), **res[0], "zline": res[1]}
    sweeps = res[0]["sweeps_per_step"] * steps
    if oracle_sample:
        import oracle
        cores = _oracle_threads()
        us = oracle_us_per_sweep(cfg, 0)
        o = oracle.Oracle(dict(cfg, omega=[0.8, 1.0] * 16, ptol=0.0, pmaxit=32))
        o.set_fields(*inputs.paper_les_initial(cfg, 1))
        t0 = time.perf_counter()
        o.step(1)
        t_step = time.perf_counter() - t0
        s_gpu = sweeps / steps
        t_proj = t_step + max(0.0, s_gpu - 32) * us * 1e-6
        out["cpu_baseline"] = {
            "kind": "oracle", "cores": cores, "value": cells / t_proj / 1e6, "unit": "Mcell*steps/s",
            "oracle_step_s_at_32_sweeps": t_step, "oracle_us_per_sweep": us,
            "sample": "one FP64 oracle step of the same workload from the same start with its solve held to 32 "
                      "sweeps (%.2f s), plus the oracle's measured time per sweep for the other %.0f of the "
                      "GPU's %.0f sweeps a step (projected; once-per-cycle residual checks not added)"
                      % (t_step, max(0.0, s_gpu - 32), s_gpu)}
    return out


def headline_config(args):
    from paper_1511_07800_gb300 import inputs
    cfg = inputs.preset(args.workload, zline=1 if args.solver == "zline" else 0, cn_zline=1)
    if args.grid:
        nx, ny, nz = (int(x) for x in args.grid.lower().split("x"))
        cfg.update(nx=nx, ny=ny, nz=nz)
    cfg["cn_sweeps"] = _auto_cn(cfg, args.precision)
    return cfg


def oracle_schedule(cfg):
    from oracle import srj
    om, _, _ = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"],
                                cfg.get("stretch", 0.0), line=bool(cfg.get("zline")))
    return om


def run_reference(args):
    """The oracle (plain FP64 C, OpenMP over z) stepping the headline
    workload on rank 0's host cores.  A whole step of the oracle takes
    about 15 s at this size, so each step is a bounded sample: first one
    complete untimed step, whose tolerance-driven solve gives the oracle's
    own sweeps per step, then every step (warm-up and timed) runs with its
    pressure solve held to 32 sweeps and is charged the measured time of
    the remaining sweeps (the oracle's time per sweep on the same grid)."""
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_1511_07800_gb300 import inputs
    cfg = headline_config(args)
    ncores = len(os.sched_getaffinity(0))
    oracle.set_threads(ncores)
    om = oracle_schedule(cfg)
    fields = inputs.initial_fields(args.workload, cfg, seed=1 if args.workload == "les_channel" else 0)
    full = oracle.Oracle(dict(cfg, omega=om))
    full.set_fields(*fields)
    t0 = time.perf_counter()
    st = full.step(1)
    t_full = time.perf_counter() - t0
    s_full = st["sweeps"]
    us = oracle_us_per_sweep(cfg, int(cfg.get("zline", 0)))
    o = oracle.Oracle(dict(cfg, omega=[0.8, 1.0] * 16, ptol=0.0, pmaxit=32))
    f = full.get_fields()
    o.set_fields(f["u"], f["v"], f["w"], f["p"])
    for _ in range(args.warmup):
        o.step(1)
    total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        o.step(1)
        total += time.perf_counter() - t0 + max(0, s_full - 32) * us * 1e-6
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    val = cells * args.steps / total / 1e6
    sample = ("each step: one FP64 oracle step with its solve held to 32 sweeps, plus %d x %.0f us for the rest "
              "of the %d sweeps the oracle's own tolerance-driven solve took in a complete first step (%.1f s; "
              "untimed); %s SRJ" % (max(0, s_full - 32), us, s_full, t_full,
                                    "z-line" if cfg.get("zline") else "point"))
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Mcell*steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC if args.workload == WORKLOAD else args.workload,
                                            "cells": cells, "srj_M": len(om), "cn_sweeps": cfg["cn_sweeps"]},
            "cpu_baseline": {"value": val, "unit": "Mcell*steps/s", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "Mcell*steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _auto_cn(cfg, precision="fp32"):
    """Crank-Nicolson Jacobi sweeps for the workload, by the library's rule
    (contraction hS/(1+hS) per sweep, down to the storage precision: 2^-24
    for FP32 fields, 1e-12 for FP64; S the largest diagonal weight for point
    sweeps, the x-y coupling weights alone for z-line sweeps); both arms
    get the count explicitly so they run the same sweeps."""
    from paper_1511_07800_gb300 import inputs
    zf = inputs.zfaces(cfg)
    dz = [zf[k + 1] - zf[k] for k in range(cfg["nz"])]
    zc = [0.5 * (zf[k] + zf[k + 1]) for k in range(cfg["nz"])]
    dzf = [dz[0]] + [zc[k] - zc[k - 1] for k in range(1, cfg["nz"])] + [dz[-1]]
    dx, dy = cfg["Lx"] / cfg["nx"], cfg["Ly"] / cfg["ny"]
    if cfg.get("cn_zline"):
        smax = 2 / dx**2 + 2 / dy**2
    else:
        smax = max(4 / dx**2 + 4 / dy**2 + 2 / (dzf[k] * dz[k]) + 2 / (dzf[k + 1] * dz[k])
                   for k in range(cfg["nz"]))
    hs = 0.5 * cfg["dt"] * cfg["nu"] * (4.0 if cfg.get("les") else 1.0) * smax
    rho = hs / (1 + hs)
    if rho <= 0:
        return 1
    lo = 1 if cfg.get("cn_zline") else 2
    target = 2.0 ** -24 if precision == "fp32" else 1e-12
    return max(lo, min(int(math.ceil(math.log(target) / math.log(rho))), 200))


def timed_steps(ch, steps, stream, flush):
    """`steps` projection steps, each bracketed by CUDA events on the
    library's stream, after an untimed write of a buffer larger than L2."""
    import torch
    ms, sweeps, launches, solve_ms, passes, conv = 0.0, 0, 0, 0.0, 0, True
    for _ in range(steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st = ch.step(1)
        e1.record(stream)
        e1.synchronize()
        ms += e0.elapsed_time(e1)
        sweeps += st["solve_sweeps"]
        passes += st["passes"]
        launches += st["launches"]
        solve_ms += st["solve_ms"]
        conv = conv and st["converged"]
    return dict(ms=ms, sweeps=sweeps, passes=passes, launches=launches, solve_ms=solve_ms, converged=conv)


def sweep_roofline(word, cells, r, kernel, peak, traffic_key):
    """HBM roofline of the SRJ sweep: 3 words a cell (read p and b, write
    p'), over the mean time per sweep of the solve graphs (GPU events around
    each solve, charged with its once-per-cycle checks and refinement
    kernels: a lower bound on the sweep's own rate)."""
    bytes_per_sweep = 3 * word * cells
    t = r["solve_ms"] / max(1, r["sweeps"]) / 1e3
    ach = bytes_per_sweep / t / 1e9 if r["sweeps"] else None
    tr = traffic_for(traffic_key)
    traffic = None
    if tr:
        traffic = tr["dram_bytes_per_launch"] * cells / tr["cells"]
    return {"bound": "hbm", "kernel": kernel, "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": ach / peak if ach else None, "traffic": traffic, "bytes_per_launch": bytes_per_sweep,
            "mean_launch_us": t * 1e6,
            "note": "achieved = algorithmic bytes (3 words a cell) / (solve-graph GPU time / sweeps), the "
                    "once-per-cycle residual checks and refinement kernels charged to the sweeps"}


def side_steps(stp, cfg, precision, fields, steps, warmup, stream, flush, peak, traffic_key):
    """Whole projection steps of another configuration (its own handle)."""
    word = 4 if precision == "fp32" else 8
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    with stp.Channel(cfg, precision=precision, stream=stream.cuda_stream) as ch:
        ch.set_fields(*fields)
        for _ in range(max(3, warmup)):
            ch.step(1)
        r = timed_steps(ch, steps, stream, flush)
        variant, _ = ch.sweep_tile()
        lk = ch.line_kernel()
    if cfg.get("zline"):
        kern = LINE_NAMES[lk] if precision == "fp32" else "k_line_sweep_vec<double> (z-line)"
    else:
        kern = (TILE_NAMES.get(variant, "k_sweep_f32") + " (autotuned tile variant %d)" % variant
                if precision == "fp32" else "k_sweep_f64_v2")
    out = {"value": cells * steps / (r["ms"] / 1e3) / 1e6, "unit": "Mcell*steps/s", "ms_per_step": r["ms"] / steps,
           "steps": steps, "warmup": max(3, warmup), "sweeps_per_step": r["sweeps"] / steps,
           "solve_ms_per_step": r["solve_ms"] / steps, "converged": r["converged"],
           "gpu_launches_per_step": r["launches"] / steps,
           "roofline": sweep_roofline(word, cells, r, kern, peak, traffic_key)}
    if precision == "fp64":
        out["roofline"]["note"] += ("; in FP64 the sweep is bound by GB300's FP64 pipe, not by HBM "
                                    "(profiles/srj_sweep_f64_os_instability.md)")
    return out


def sweeps_above_l2(stp, peak):
    """The SRJ sweeps on working sets larger than the 126 MB L2, so that
    their rate is an HBM rate: FP64 sweeps on the LES grid (p, p', b:
    151 MB) and FP32 inner sweeps on a 512 x 256 x 192 grid (d, d', r:
    302 MB); point and z-line sweeps each; a fixed number of sweeps from a
    seeded mean-free right-hand side, GPU events around the solve graph."""
    import numpy as np
    import torch
    from paper_1511_07800_gb300 import inputs
    out = {}
    cases = [("fp64_les_grid", "fp64", 256, 128, 192), ("fp32_512x256x192", "fp32", 512, 256, 192)]
    for name, prec, nx, ny, nz in cases:
        cfg = inputs.preset("les_channel", nx=nx, ny=ny, nz=nz)
        rng = np.random.default_rng(3)
        b = torch.from_numpy(rng.standard_normal((nz, ny, nx))).cuda()
        dz = torch.from_numpy(np.diff(inputs.zfaces(cfg))).cuda()[:, None, None]
        b -= (b * dz).sum() / (dz.sum() * nx * ny)
        word = 8 if prec == "fp64" else 4
        cells = nx * ny * nz
        res = {"grid": "%dx%dx%d" % (nx, ny, nz), "working_set_MB": 3 * word * cells / 1e6}
        for solver, zl in (("point", 0), ("zline", 1)):
            with stp.Channel(dict(cfg, zline=zl), precision=prec) as ch:
                M = len(stp.srj_schedule(dict(cfg, zline=zl))[0])
                p = torch.zeros_like(b)
                ch.poisson_solve(b, p, tol=0.0, maxit=M)  # warm-up (and the FP32 tile autotuner)
                p.zero_()
                st = ch.poisson_solve(b, p, tol=0.0, maxit=2 * M)
                variant, _ = ch.sweep_tile()
                lk = ch.line_kernel()
            t = st["solve_ms"] / max(1, st["sweeps"]) / 1e3
            ach = 3 * word * cells / t / 1e9
            res[solver] = {"sweeps": st["sweeps"], "us_per_sweep": t * 1e6, "achieved_GBs": ach,
                           "frac": ach / peak,
                           "kernel": (LINE_NAMES[lk].split(" ")[0] if zl and prec == "fp32" else
                                      "k_line_sweep_vec<double,RB>" if zl else
                                      (TILE_NAMES.get(variant, "k_sweep_f32") if prec == "fp32" else "k_sweep_f64_v2"))}
        out[name] = res
    out["note"] = ("time per sweep of a solve graph held to 2 cycles (its two residual checks and, in FP32, the "
                   "refinement kernels charged to the sweeps); achieved = 3 words a cell / that time")
    return out


def run_ours(args):
    import numpy as np
    import torch

    from paper_1511_07800_gb300 import build, inputs, stp
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl", init_method="env://")
    torch.cuda.set_device(local)
    build.build()
    cfg = headline_config(args)
    seed = 1 if args.workload == "les_channel" else 0
    fields = inputs.initial_fields(args.workload, cfg, seed=seed)
    stream = torch.cuda.current_stream()
    ch = stp.Channel(cfg, precision=args.precision, device=local, stream=stream.cuda_stream)
    ch.set_fields(*fields)
    cells = cfg["nx"] * cfg["ny"] * cfg["nz"]
    for _ in range(max(3, args.warmup)):
        ch.step(1)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clk = Clocks(local)
    clk.start()
    r = timed_steps(ch, args.steps, stream, flush)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms_max = reduce_max(r["ms"], "cuda")
    value = world * cells * args.steps / (ms_max / 1e3) / 1e6

    # end to end through the C ABI with pinned host buffers: every step the
    # whole stepper state (velocities, pressure, the two Adams-Bashforth
    # history levels, the step counter) goes in, one step runs, and the new
    # state comes out, so each step is the benchmarked AB3 step
    e2e = None
    if not args.no_e2e:
        n = ch.state_size()
        host = torch.empty(n, dtype=torch.float64).pin_memory()
        ch.get_state(host)
        torch.cuda.synchronize()
        ke = max(3, min(args.steps, 10))
        t0 = time.perf_counter()
        for _ in range(ke):
            ch.set_state(host)
            ch.step(1)
            ch.get_state(host)
        te = time.perf_counter() - t0
        te = reduce_max(te, "cuda")
        e2e = {"value": world * cells * ke / te / 1e6, "unit": "Mcell*steps/s", "h2d_bytes_per_step": 8 * n,
               "d2h_bytes_per_step": 8 * n, "host_memory": "pinned", "steps": ke,
               "api": "stp_set_state (host) -> stp_step(1) -> stp_get_state (host), wall clock"}

    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    word = 4 if args.precision == "fp32" else 8
    variant, _ = ch.sweep_tile()
    if cfg.get("zline"):
        kern = (LINE_NAMES[ch.line_kernel()] if args.precision == "fp32"
                else "k_line_sweep_vec<double,RB> (z-line SRJ sweep)")
        tkey = "zline_sweep_%s_%s" % (args.precision, args.workload)
    else:
        kern = (TILE_NAMES.get(variant, "k_sweep_f32") + " (SRJ sweep, autotuned tile variant %d)" % variant
                if args.precision == "fp32" else "k_sweep_f64_v2 (SRJ sweep)")
        tkey = "point_sweep_%s_%s" % (args.precision, args.workload)
    roof = sweep_roofline(word, cells, r, kern, peak, tkey)
    roof["peak_source"] = "MEASURED_PEAKS.json hbm_gbs (measured)" if "hbm_gbs" in peaks else "fallback"
    roof["l2_note"] = ("the FP32 inner solve's working set (d, d', r: 12 bytes a cell, %.0f MB) %s the 126 MB L2; "
                       "the sweeps' HBM rate on working sets above L2 is under srj_sweeps_above_l2"
                       % (12 * cells / 1e6, "fits in" if 12 * cells < 126e6 else "exceeds"))
    line = {
        "metric": METRIC, "value": value, "unit": "Mcell*steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": (WORKLOAD_DESC if args.workload == WORKLOAD else args.workload) +
                   (" at " + args.grid if args.grid else ""),
                   "cells": cells, "precision": args.precision, "solver": args.solver,
                   "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between timed steps (256 MB write, untimed); the step's fields (about "
                         "%.0f MB) exceed L2" % (cells * (4 * 17 + 8 * 4) / 1e6),
                   "srj_M": len(stp.srj_schedule(cfg)[0]), "cn_sweeps": cfg["cn_sweeps"]},
        "poisson": {"sweeps_per_step": r["sweeps"] / args.steps, "refine_passes_per_step": r["passes"] / args.steps,
                    "all_converged": r["converged"], "ms_per_step": r["solve_ms"] / args.steps},
        "roofline": roof,
        "gpu_launches": r["launches"],
        "clocks": clocks,
        "e2e": e2e,
    }
    side = rank == 0 and world == 1 and args.grid is None and not args.only_headline
    if side and not args.no_extra:
        try:
            pc = dict(cfg, zline=0)
            line["les_channel_point_srj"] = side_steps(stp, pc, "fp32", fields, max(3, min(args.steps, 5)), 3,
                                                       stream, flush, peak, "point_sweep_fp32_les_channel")
            line["les_channel_point_srj"]["note"] = "the same workload with the paper's point SRJ sweeps"
        except Exception as ex:  # report, never fake
            line["les_channel_point_srj"] = {"error": str(ex)[:300]}
        try:
            c2 = inputs.preset("os_instability")
            f2 = inputs.initial_fields("os_instability", c2, seed=0)
            line["os_instability"] = {
                "workload": "os_instability 128x64x128 Re 7500 dt 2e-3, Poiseuille + OS mode 1e-4 + noise 1e-6, "
                            "point SRJ to 1e-8",
                "fp32_refine": side_steps(stp, dict(c2, cn_sweeps=_auto_cn(c2, "fp32")), "fp32", f2,
                                          max(3, min(args.steps, 10)), 3, stream, flush, peak,
                                          "point_sweep_fp32_os_instability"),
                "fp64": side_steps(stp, dict(c2, cn_sweeps=_auto_cn(c2, "fp64")), "fp64", f2,
                                   max(3, min(args.steps, 5)), 3, stream, flush, peak,
                                   "point_sweep_fp64_os_instability")}
        except Exception as ex:  # report, never fake
            line["os_instability"] = {"error": str(ex)[:300]}
        try:
            line["srj_sweeps_above_l2"] = sweeps_above_l2(stp, peak)
        except Exception as ex:  # report, never fake
            line["srj_sweeps_above_l2"] = {"error": str(ex)[:300]}
    if side and not args.no_learned:
        try:
            c2 = inputs.preset("os_instability")  # cn_sweeps 0: the library's count for each precision
            line["poisson_learned_vs_plain"] = learned_comparison(c2, args.steps, not args.no_cpu_baseline)
        except Exception as ex:  # report, never fake
            line["poisson_learned_vs_plain"] = {"error": str(ex)[:200]}
    if side and not args.no_batch:
        try:
            line["batched_channels"] = batched_channels(max(3, min(args.steps, 10)), args.warmup, peak,
                                                        not args.no_cpu_baseline)
        except Exception as ex:  # report, never fake
            line["batched_channels"] = {"error": str(ex)[:200]}
    if side and not args.no_les:
        try:
            line["les_paper"] = les_paper_steps(10, 3, not args.no_cpu_baseline)
        except Exception as ex:  # report, never fake
            line["les_paper"] = {"error": str(ex)[:200]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.only_headline:
        try:
            line["cpu_baseline"] = cpu_baseline_sample(cfg, fields, r["sweeps"] / args.steps, oracle_schedule(cfg))
        except Exception as ex:  # report, never fake
            line["cpu_baseline"] = {"value": None, "error": str(ex)[:200]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    ch.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
