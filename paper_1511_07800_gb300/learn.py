"""Learned pressure guess: harvest training pairs from the solver, train the
U-Net, and compare solves with and without it.  Every arithmetic step runs
in the CUDA library (harvest in the solver, normalisation, forward,
backward and Adam in the network's kernels); this module only drives the
calls and holds the pairs in device memory.

A pair is (r, dp): r = b - L p_prev, the residual of the previous step's
pressure at the start of a solve, and dp = p - p_prev, the exact correction
the SRJ solve then finds.  The network maps r/s to dp/s (s = RMS(r)).
"""
import json
import math
import time

import numpy as np

from . import inputs, stp


def workload(name, grid=None, **over):
    cfg = inputs.preset(name, **over)
    if grid is not None:
        cfg.update(nx=grid[2], ny=grid[1], nz=grid[0])
    return cfg


def varied_fields(cfg, seed):
    """Instability-type initial state with a randomised mode amplitude and
    noise level (log-uniform), so that the harvested pressures vary."""
    rng = np.random.default_rng(10_000 + seed)
    Re = 1.0 / cfg["nu"]
    alpha = 2 * math.pi / cfg["Lx"] * (0.5 * cfg["Lz"])
    u0, v0, w0 = inputs.poiseuille(cfg, 1.0)
    amp = 10 ** rng.uniform(-5, -3)
    du, dv, dw, _ = inputs.os_mode(cfg, amp, Re, alpha)
    noise = 10 ** rng.uniform(-6, -2)
    return inputs.noise(cfg, noise, seed, (u0 + du, v0 + dv, w0 + dw))


def harvest(cfg, seeds, steps_per_seed, precision="fp32", skip=2, device=0):
    """Run one channel per seed and keep the pairs of every step after the
    first `skip` (the start-up solves begin from p = 0)."""
    import torch
    n = len(seeds) * steps_per_seed
    shape = (cfg["nz"], cfg["ny"], cfg["nx"])
    R = torch.zeros((n,) + shape, dtype=torch.float32, device="cuda")
    DP = torch.zeros_like(R)
    r = torch.zeros(shape, dtype=torch.float32, device="cuda")
    dp = torch.zeros_like(r)
    q = 0
    for seed in seeds:
        with stp.Channel(cfg, precision=precision, device=device) as ch:
            ch.set_fields(*varied_fields(cfg, seed))
            ch.step(skip)
            ch.set_harvest(r, dp)
            for _ in range(steps_per_seed):
                ch.step(1)
                R[q].copy_(r)
                DP[q].copy_(dp)
                q += 1
            ch.set_harvest(None, None)
    return R, DP


def output_scale(R, DP, nmax, shape, sample=64):
    """K = 1 / RMS(dp/s) over (a sample of) the pairs, measured with the
    network kernels: an all-zero network predicts 0, so its loss is the mean
    of (dp/s)^2."""
    zero = stp.UNet(nmax, *shape)
    zero.set_params(np.zeros(stp.UNet.param_count(), dtype=np.float32))
    n = min(R.shape[0], sample)
    tot, cnt = 0.0, 0
    for i in range(0, n, nmax):
        j = min(n, i + nmax)
        tot += zero.eval_pairs(R[i:j].contiguous(), DP[i:j].contiguous()) * (j - i)
        cnt += j - i
    zero.close()
    return 1.0 / math.sqrt(tot / cnt)


def train(net, R, DP, iters, batch, lr, seed=3, log_every=0):
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    n = R.shape[0]
    for it in range(iters):
        idx = torch.randint(0, n, (batch,), generator=g).cuda()
        loss = net.train_pairs(R[idx].contiguous(), DP[idx].contiguous(), lr)
        losses.append(loss)
        if log_every and it % log_every == 0:
            print("iter %d loss %.4g" % (it, loss), flush=True)
    return losses


def compare(cfg, net, seed, nsteps, precision="fp32", warm=2, device=0):
    """The same channel stepped twice from the same state, with the plain
    solve and with the learned guess: SRJ sweeps and solve time per step."""
    out = {}
    for mode in ("plain", "learned"):
        with stp.Channel(cfg, precision=precision, device=device) as ch:
            ch.set_fields(*varied_fields(cfg, seed))
            ch.step(warm)
            if mode == "learned":
                ch.set_learned_guess(net)
            sweeps, ms, passes = 0, 0.0, 0
            t0 = time.perf_counter()
            for _ in range(nsteps):
                st = ch.step(1)
                assert st["converged"]
                sweeps += st["sweeps"]
                passes += st["passes"]
                ms += st["solve_ms"]
            wall = time.perf_counter() - t0
            if mode == "learned":
                ch.set_learned_guess(None)
        out[mode] = dict(sweeps=sweeps / nsteps, solve_ms=ms / nsteps, passes=passes / nsteps, wall_s=wall)
    return out


def compare_modes(cfg, net, seed, nsteps, precision="fp32", warm=2, device=0):
    """Plain solves against the network as initial guess (mode 0) and as
    preconditioner (mode 1) on the same channel from the same state: SRJ
    sweeps, refinement passes and GPU solve time per step."""
    out = {}
    for mode in ("plain", "guess", "precond"):
        with stp.Channel(cfg, precision=precision, device=device) as ch:
            ch.set_fields(*varied_fields(cfg, seed))
            ch.step(warm)
            if mode != "plain":
                ch.set_learned_guess(net)
                ch.set_learned_mode(0 if mode == "guess" else 1)
            sweeps, ms, passes, conv = 0, 0.0, 0, True
            for _ in range(nsteps):
                st = ch.step(1)
                conv = conv and st["converged"]
                sweeps += st["sweeps"]
                passes += st["passes"]
                ms += st["solve_ms"]
            if mode != "plain":
                ch.set_learned_guess(None)
        out[mode] = dict(sweeps=sweeps / nsteps, solve_ms=ms / nsteps, passes=passes / nsteps, converged=conv)
    for mode in ("guess", "precond"):
        out[mode]["speedup"] = out["plain"]["solve_ms"] / out[mode]["solve_ms"]
    return out


def he_init(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, a small output
    layer, in the parameter order of the network."""
    rng = np.random.default_rng(seed)
    theta, cin, specs = [], 1, []
    for c in (16, 32, 64, 128):
        specs += [(cin, c, 27), (c, c, 27)]
        cin = c
    for lv in (2, 1, 0):
        c = (16, 32, 64, 128)[lv]
        specs += [((16, 32, 64, 128)[lv + 1] + c, c, 27), (c, c, 27)]
    specs.append((16, 1, 1))
    for i, (ci, co, taps) in enumerate(specs):
        std = math.sqrt(2.0 / (ci * taps)) if i < len(specs) - 1 else 0.1 / math.sqrt(ci)
        theta.append(rng.standard_normal(co * ci * taps) * std)
        theta.append(np.zeros(co))
    return np.concatenate(theta).astype(np.float32)


def config4(pairs=20000, seeds=200, grid=(128, 64, 128), eval_grids=((128, 64, 128), (192, 128, 256)),
            batch=4, iters=(3000, 1000), lrs=(1e-3, 3e-4), eval_steps=8, device=0, log=print):
    """The learned-guess experiment: `pairs` (residual, correction) pairs
    harvested from instability-workload channels (random mode amplitude and
    noise per seed, FP32 solves) at `grid` (nz, ny, nx), training with Adam
    in the library's kernels, then plain against learned solves (initial
    guess and preconditioner, FP32 and FP64) on an unseen seed at each of
    `eval_grids`.  Returns a dict of the measurements."""
    import torch
    t0 = time.perf_counter()
    cfg = workload("os_instability", grid=grid)
    per = max(1, pairs // seeds)
    R, DP = harvest(cfg, seeds=range(seeds), steps_per_seed=per)
    t_h = time.perf_counter() - t0
    log("harvested %d pairs in %.1f s" % (R.shape[0], t_h))
    Rv, DPv = harvest(cfg, seeds=[9000], steps_per_seed=16)
    K = output_scale(R, DP, batch, grid)
    net = stp.UNet(batch, *grid)
    theta0 = he_init(3)
    net.set_params(theta0)
    net.set_output_scale(K)
    losses = []
    t1 = time.perf_counter()
    for n, lr in zip(iters, lrs):
        losses += train(net, R, DP, n, batch, lr, seed=4 + len(losses), log_every=500)
    torch.cuda.synchronize()
    t_t = time.perf_counter() - t1
    val = float(np.mean([net.eval_pairs(Rv[i:i + batch].contiguous(), DPv[i:i + batch].contiguous())
                         for i in range(0, Rv.shape[0], batch)]))
    theta = net.get_params()
    net.close()
    del R, DP
    torch.cuda.empty_cache()
    out = {"pairs": int(per * seeds), "harvest_grid": "%dx%dx%d" % (grid[2], grid[1], grid[0]),
           "harvest_s": t_h, "train_s": t_t, "adam_steps": len(losses), "batch": batch,
           "final_train_loss": float(np.mean(losses[-50:])), "val_loss": val, "output_scale": K,
           "note": "losses in units where the all-zero network scores 1", "eval": {}}
    for eg in eval_grids:
        ecfg = workload("os_instability", grid=eg)
        enet = stp.UNet(1, *eg)
        enet.set_params(theta)
        enet.set_output_scale(K)
        res = {}
        for prec in ("fp32", "fp64"):
            res[prec] = compare_modes(ecfg, enet, seed=9001, nsteps=eval_steps, precision=prec)
        x = torch.randn((1,) + tuple(eg), device="cuda")
        y = torch.zeros_like(x)
        for _ in range(2):
            enet.forward(x, y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            enet.forward(x, y)
        e1.record()
        e1.synchronize()
        res["forward_ms"] = e0.elapsed_time(e1) / 5
        enet.close()
        out["eval"]["%dx%dx%d" % (eg[2], eg[1], eg[0])] = res
        log(json.dumps(res))
    return out


if __name__ == "__main__":
    import sys
    kw = {}
    if len(sys.argv) > 1:
        kw = json.loads(sys.argv[1])
    print(json.dumps(config4(**kw)), flush=True)
