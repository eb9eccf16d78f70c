"""Physics checks of the GPU step against the oracle's Orr-Sommerfeld
eigenvalue (Sec. 4.2): the linear growth rate of ln ||w||_2 of a small
Orr-Sommerfeld mode on Poiseuille flow converges to the eigenvalue at
second order in the wall-normal spacing (the paper's 2-D trick ny = 3)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def growth_rate(stp_lib, Re, alpha, nx, nz, dt, nsteps, every=20, t_fit=0.8):
    from paper_1511_07800_gb300 import inputs
    cfg = inputs.preset("os_instability", nx=nx, ny=3, nz=nz, Lx=2 * math.pi / alpha, nu=1.0 / Re, fx=2.0 / Re,
                        dt=dt)
    u0, v0, w0 = inputs.poiseuille(cfg, 1.0)
    du, dv, dw, _ = inputs.os_mode(cfg, 1e-4, Re, alpha)
    zf = inputs.zfaces(cfg)
    hz = np.diff(np.concatenate([[zf[0]], 0.5 * (zf[1:] + zf[:-1]), [zf[-1]]]))
    t, L = [], []
    with stp_lib.Channel(cfg, precision="fp64") as ch:
        ch.set_fields(u0 + du, v0 + dv, w0 + dw)
        for n in range(0, nsteps + 1, every):
            if n > 0:
                assert ch.step(every)["converged"]
            w = ch.get_fields()["w"]
            L.append(math.sqrt(float(np.sum(hz[:, None, None] * w * w))))
            t.append(n * dt)
    t, L = np.array(t), np.array(L)
    m = t >= t_fit
    return np.polyfit(t[m], np.log(L[m]), 1)[0]


def test_orr_sommerfeld_growth_rate_converges(stp_lib, orc):
    """Re = 7500, alpha = 1 (the instability workload, 2-D slice): the error
    of the growth rate falls by more than 2.5x when nz doubles (second
    order), and is below 40 % at nz = 128."""
    from oracle import os_eig
    lam = os_eig.least_stable(7500.0, 1.0).real
    e = []
    for nz in (64, 128):
        g = growth_rate(stp_lib, 7500.0, 1.0, 128, nz, 2e-3, 2000)
        e.append(abs(g - lam) / lam)
    print("growth-rate errors nz=64, 128:", e)
    assert e[1] < e[0] / 2.5 and e[1] < 0.4
