"""Learned pressure guess: harvest training pairs from the solver, train the
U-Net, and compare solves with and without it.  Every arithmetic step runs
in the CUDA library (harvest in the solver, normalisation, forward,
backward and Adam in the network's kernels); this module only drives the
calls and holds the pairs in device memory.

A pair is (r, dp): r = b - L p_prev, the residual of the previous step's
pressure at the start of a solve, and dp = p - p_prev, the exact correction
the SRJ solve then finds.  The network maps r/s to dp/s (s = RMS(r)).
"""
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
