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


def test_table1_orr_sommerfeld_case(stp_lib, orc):
    """The paper's Orr-Sommerfeld validation case (Sec. 4.2, its simulation
    table): Re_* = 500, alpha = 2 pi / 4, a channel one wavelength long,
    1200 x 3 x 300 cubic cells, dt = 1e-5 in the paper's units; in
    half-height centreline units Re = 31250, alpha = pi / 4, Lx = 8, Lz = 2,
    dt = 2.5e-3.  Started from the least-stable mode at max |du| = 1e-4 and
    run for 1600 steps (t = 4) in FP64, the three quantities of the paper's
    comparison are checked against the oracle's Chebyshev eigenvalue and
    eigenfunction and the paper's printed numbers:
      * the growth rate of L2^w(t) = ||dw||_2 (paper: 1.7293 simulated
        against 1.8056 theory, 4 % low): within 4 % of the eigenvalue;
      * the period T = 2 pi / omega of the oscillation, omega from the
        phase of the alpha Fourier mode of dw at mid-height (paper: 0.186
        +- 0.004 against 0.185): within 0.004 of the printed 0.185;
      * F(z) = du(x0, z) / max_z du(x0, z), x0 the location of the global
        maximum of du (the perturbation of u with its x-mean removed),
        against the eigenfunction's Re(psi' e^{i phi}) with phi putting the
        maximum at x0: within 1e-2 everywhere."""
    import json
    import os
    from numpy.polynomial import chebyshev as C
    from oracle import os_eig
    from paper_1511_07800_gb300 import inputs
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
    Re_s, a_p = gold["os_table"]["Re_star"], gold["os_table"]["alpha_over_pi"] * math.pi
    Re, alpha, _ = os_eig.paper_to_half_height(Re_s, a_p, 0.0)
    nx, ny, nz = 1200, 3, 300
    cfg = inputs.preset("os_instability", nx=nx, ny=ny, nz=nz, Lx=2 * math.pi / alpha, Ly=0.02,
                        nu=1.0 / Re, fx=2.0 / Re, dt=1e-5 * Re_s / 2)
    assert abs(cfg["Lx"] - 8.0) < 1e-12 and abs(cfg["dt"] - 2.5e-3) < 1e-15
    u0, v0, w0 = inputs.poiseuille(cfg, 1.0)
    du, dv, dw, _ = inputs.os_mode(cfg, 1e-4, Re, alpha)
    zf = inputs.zfaces(cfg)
    hz = np.diff(np.concatenate([[zf[0]], 0.5 * (zf[1:] + zf[:-1]), [zf[-1]]]))
    dx = cfg["Lx"] / nx
    xw = (np.arange(nx) + 0.5) * dx
    kmid = nz // 2  # the face at z = Lz / 2
    t, L, ph = [], [], []
    every, nsteps = 100, 1600
    with stp_lib.Channel(dict(cfg, zline=1), precision="fp64") as ch:
        ch.set_fields(u0 + du, v0 + dv, w0 + dw)
        for n in range(0, nsteps + 1, every):
            if n > 0:
                assert ch.step(every)["converged"]
            f = ch.get_fields()
            w = f["w"]
            L.append(math.sqrt(float(np.sum(hz[:, None, None] * w * w)) * dx * cfg["Ly"] / ny))
            ph.append(np.angle(np.sum(w[kmid, 1] * np.exp(-1j * alpha * xw))))
            t.append(n * cfg["dt"])
    t, L, ph = np.array(t), np.array(L), np.unwrap(np.array(ph))
    lam = os_eig.least_stable(Re, alpha)
    m = t >= 0.8
    growth = np.polyfit(t[m], np.log(L[m]), 1)[0]
    omega = -np.polyfit(t[m], ph[m], 1)[0]
    T_paper = 2 * math.pi / omega / (Re_s / 2)
    print("growth %.5e (eigenvalue %.5e, paper units %.4f), period %.4f paper units"
          % (growth, lam.real, growth * Re_s / 2, T_paper))
    assert abs(growth - lam.real) < 0.04 * lam.real
    assert abs(T_paper - gold["os_table"]["period"]) <= gold["os_simulated"]["period_uncertainty"]
    assert abs(omega - abs(lam.imag)) < 0.01 * abs(lam.imag)
    # F(z) at the final time
    uu = f["u"][:, 1, :]
    dU = uu - uu.mean(axis=1, keepdims=True)
    k0, i0 = np.unravel_index(np.argmax(dU), dU.shape)
    F_sim = dU[:, i0] / dU[:, i0].max()
    lams, vecs, xi = os_eig.os_spectrum(Re, alpha)
    nodes = np.concatenate([[1.0], xi, [-1.0]])
    psi = np.concatenate([[0.0], vecs[:, 0], [0.0]])
    coef = C.chebfit(nodes, psi.real, len(nodes) - 1) + 1j * C.chebfit(nodes, psi.imag, len(nodes) - 1)
    dcoef = C.chebder(coef)
    eta = 0.5 * (zf[1:] + zf[:-1]) - 1.0
    dpsi = C.chebval(eta, dcoef.real) + 1j * C.chebval(eta, dcoef.imag)
    fine = np.linspace(-1, 1, 4001)
    dfine = C.chebval(fine, dcoef.real) + 1j * C.chebval(fine, dcoef.imag)
    phi = -np.angle(dfine[np.argmax(np.abs(dfine))])
    F_th = np.real(dpsi * np.exp(1j * phi))
    F_th /= F_th.max()
    # the least-stable mode is even in psi, so |du| peaks equally near both
    # walls; x0 may hold either peak, which mirrors F about mid-height
    dev = min(np.abs(F_sim - F_th).max(), np.abs(F_sim - F_th[::-1]).max())
    print("F(z) max deviation %.2e" % dev)
    assert dev < 1e-2
