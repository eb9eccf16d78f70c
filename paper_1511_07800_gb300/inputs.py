"""Seeded synthetic inputs: workload presets and initial velocity fields.

This module holds no arithmetic of the projection step.  It builds the
channel set-ups (sizes, viscosity, time step, forcing) and initial fields
on the host with numpy, so that the CUDA path and the CPU oracle can start
from the same arrays.  Random numbers come from numpy's PCG64 generator
(`np.random.default_rng(seed)`).

Layouts (x fastest), cell (i, j, k):
  u[k, j, i] at x = i dx,       z = zc[k]     shape (nz,   ny, nx)
  v[k, j, i] at y = j dy,       z = zc[k]     shape (nz,   ny, nx)
  w[k, j, i] at z = zf[k]                     shape (nz+1, ny, nx), zero at k = 0, nz
  p[k, j, i] at the cell centre               shape (nz,   ny, nx)

Workloads (half-height units: Lz = 2, delta = 1):
  laminar_startup   32 x 16 x 32, Re = 100, at rest, -dp/dx = 2/Re, dt = 1e-3
  os_instability   128 x 64 x 128, Re = 7500, Poiseuille + Orr-Sommerfeld mode
                   (alpha = 1, Lx = 2 pi) of peak |du| 1e-4 + uniform noise 1e-6,
                   dt = 2e-3
  les_channel      256 x 128 x 192, Lx = 4 pi, Ly = 2 pi, tanh walls (gamma 2),
                   bulk Re 5600 (nu = 1/2800), Smagorinsky Cs = 0.1, van Driest
                   A = 25, Re_tau = 180, constant flux U_b = 1, laminar
                   1.5 z (2 - z) + uniform noise of 10 % of U_cl, dt = 1e-3
  les_paper        240 x 140 x 120, Lx = 8, Ly = 4, Lz = 1 (the paper's LES, its
                   units), Re_* = 360, -dp/dx = 2, Smagorinsky, dt = 1e-4,
                   u = U0/3 + a curl(f A) with random Fourier modes (5 per axis),
                   a setting the curl term's rms to 10 % of max U0/3
"""
import math

import numpy as np
import scipy.interpolate
import scipy.linalg

PI = math.pi


def preset(name, **over):
    """Channel set-up as a plain dict (the keys of the C-ABI config)."""
    base = dict(Lx=2 * PI, Ly=PI, Lz=2.0, forcing=0, fx=0.0, ubulk=0.0, les=0, cs=0.1,
                vd_a=25.0, re_tau=180.0, stretch=0.0, cn_sweeps=0, ptol=1e-8, pmaxit=200000)
    if name == "laminar_startup":
        Re = 100.0
        base.update(nx=32, ny=16, nz=32, nu=1 / Re, dt=1e-3, fx=2 / Re)
    elif name == "os_instability":
        Re = 7500.0
        base.update(nx=128, ny=64, nz=128, Lx=2 * PI / 1.0, nu=1 / Re, dt=2e-3, fx=2 / Re)
    elif name == "les_channel":
        base.update(nx=256, ny=128, nz=192, Lx=4 * PI, Ly=2 * PI, nu=1 / 2800.0, dt=1e-3,
                    forcing=1, ubulk=1.0, les=1, stretch=2.0)
    elif name == "les_paper":
        # the paper's LES in its own units: channel height 1, friction velocity
        # 1, Re_* = 360 (nu = 1/360), -dp/dx = 2 so that the laminar profile is
        # Re_* z (1 - z); van Driest d+ = z Re_* (re_tau is per half-height)
        base.update(nx=240, ny=140, nz=120, Lx=8.0, Ly=4.0, Lz=1.0, nu=1 / 360.0, dt=1e-4, fx=2.0,
                    les=1, re_tau=180.0)
    else:
        raise KeyError(name)
    base.update(over)
    return base


def zfaces(cfg):
    nz, Lz, g = cfg["nz"], cfg["Lz"], cfg.get("stretch", 0.0)
    s = np.arange(nz + 1) / nz
    zf = 0.5 * Lz * (1 + np.tanh(g * (2 * s - 1)) / np.tanh(g)) if g > 0 else Lz * s
    zf[0], zf[-1] = 0.0, Lz
    return zf


def zcentres(cfg):
    zf = zfaces(cfg)
    return 0.5 * (zf[1:] + zf[:-1])


def zeros(cfg):
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    return (np.zeros((nz, ny, nx)), np.zeros((nz, ny, nx)), np.zeros((nz + 1, ny, nx)))


def poiseuille(cfg, ucl=1.0):
    """u = ucl * z (2 - z) / (Lz/2)^2 scaled to the channel, v = w = 0."""
    u, v, w = zeros(cfg)
    zc = zcentres(cfg)
    d = 0.5 * cfg["Lz"]
    u[:] = (ucl * (zc / d) * (2 - zc / d))[:, None, None]
    return u, v, w


def noise(cfg, amp, seed, fields=None):
    """Add independent uniform noise on [-amp, amp] to every velocity value
    (wall faces of w excluded)."""
    rng = np.random.default_rng(seed)
    u, v, w = fields if fields is not None else zeros(cfg)
    u = u + rng.uniform(-amp, amp, u.shape)
    v = v + rng.uniform(-amp, amp, v.shape)
    dw = rng.uniform(-amp, amp, w.shape)
    dw[0] = 0.0
    dw[-1] = 0.0
    return u, v, w + dw


def random_state(cfg, seed, amp=1.0):
    """Random fields for operator-level checks: velocities, pressure and a
    positive viscosity field."""
    rng = np.random.default_rng(seed)
    u, v, w = noise(cfg, amp, seed)
    p = rng.uniform(-amp, amp, u.shape)
    nu = cfg["nu"] * (1.0 + rng.uniform(0.0, 4.0, u.shape))
    return u, v, w, p, nu


# --------------------------------------------------------------------------
# Orr-Sommerfeld mode for the instability workload.  The eigenfunction is
# found with second-order finite differences on a fine uniform grid in
# eta = z/delta - 1 (clamped ends by mirror ghosts); it only shapes the
# initial perturbation.
# --------------------------------------------------------------------------

def _os_mode_fd(Re, alpha, n=600):
    h = 2.0 / n
    eta = -1 + h * np.arange(1, n)
    m = n - 1
    D2 = (np.diag(np.full(m - 1, 1.0), -1) - 2 * np.eye(m) + np.diag(np.full(m - 1, 1.0), 1)) / h**2
    D4 = (np.diag(np.full(m - 2, 1.0), -2) + np.diag(np.full(m - 1, -4.0), -1) + 6 * np.eye(m) +
          np.diag(np.full(m - 1, -4.0), 1) + np.diag(np.full(m - 2, 1.0), 2))
    D4[0, 0] += 1.0          # psi_{-1} = psi_1 (psi' = 0 at the wall)
    D4[-1, -1] += 1.0
    D4 /= h**4
    I = np.eye(m)
    a2 = alpha * alpha
    U = 1 - eta**2
    L2 = D2 - a2 * I
    A = (D4 - 2 * a2 * D2 + a2 * a2 * I) / Re - 1j * alpha * (U[:, None] * L2) - 2j * alpha * I
    lam, vec = scipy.linalg.eig(A, L2)
    ok = np.isfinite(lam)
    lam, vec = lam[ok], vec[:, ok]
    q = int(np.argmax(lam.real))
    psi = np.concatenate([[0.0], vec[:, q], [0.0]])
    return complex(lam[q]), np.concatenate([[-1.0], eta, [1.0]]), psi


def os_mode(cfg, amp, Re, alpha):
    """Divergence-free 2-D perturbation (du, 0, dw) from the least-stable
    Orr-Sommerfeld mode, built from the streamfunction at the cell edges so
    that its discrete divergence vanishes.  Scaled so that max |du| = amp,
    with psi real where |psi| is largest.  Returns (du, dv, dw, lambda)."""
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    d = 0.5 * cfg["Lz"]
    lam, eta, psi = _os_mode_fd(Re, alpha)
    psi = psi * np.conj(psi[np.argmax(np.abs(psi))]) / np.abs(psi).max()
    sr = scipy.interpolate.CubicSpline(eta, psi.real)
    si = scipy.interpolate.CubicSpline(eta, psi.imag)
    zf = zfaces(cfg)
    dz = np.diff(zf)
    dx = cfg["Lx"] / nx
    x = dx * np.arange(nx + 1)
    ez = zf / d - 1
    ps = (sr(ez) + 1j * si(ez))
    ps[0] = ps[-1] = 0.0
    Psi = np.real(ps[:, None] * np.exp(1j * alpha * x / d)[None, :]) * d   # (nz+1, nx+1)
    du = (Psi[1:, :-1] - Psi[:-1, :-1]) / dz[:, None]                     # (nz, nx) at (i dx, zc)
    dw = -(Psi[:, 1:] - Psi[:, :-1]) / dx                                  # (nz+1, nx) at ((i+1/2)dx, zf)
    s = amp / np.abs(du).max()
    u = np.repeat((du * s)[:, None, :], ny, axis=1)
    w = np.repeat((dw * s)[:, None, :], ny, axis=1)
    w[0] = 0.0
    w[-1] = 0.0
    return u, np.zeros_like(u), w, lam


def batched_instances(count=64, seed=2, sizes=(32, 48, 64, 96, 128)):
    """Uneven-channel batch (sizes drawn per dimension from `sizes`, Re
    uniform in [5000, 10000], Orr-Sommerfeld amplitude log-uniform in
    [1e-5, 1e-3]); box 2 pi x pi x 2, dt 2e-3.  Instance i uses seed 1000 + i
    for its noise.  Returns a list of (cfg, (u, v, w))."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nx, ny, nz = (int(rng.choice(sizes)) for _ in range(3))
        Re = float(rng.uniform(5000.0, 10000.0))
        amp = float(10 ** rng.uniform(-5, -3))
        cfg = preset("os_instability", nx=nx, ny=ny, nz=nz, nu=1.0 / Re, fx=2.0 / Re)
        u0, v0, w0 = poiseuille(cfg, 1.0)
        du, dv, dw, _ = os_mode(cfg, amp, Re, 1.0)
        out.append((cfg, noise(cfg, 1e-6, 1000 + i, (u0 + du, v0 + dv, w0 + dw))))
    return out


def _paper_f(z, Lz):
    """Wall envelope of the perturbation, 1/2 + 1/2 sin(2 pi z/Lz - pi/2): zero
    with zero slope at both walls."""
    return 0.5 + 0.5 * np.sin(2 * PI * z / Lz - PI / 2)


def paper_les_initial(cfg, seed, modes=5, scale=1.0 / 3.0, intensity=0.1):
    """Turbulent-like start of the paper's LES: u = scale U0(z) + a curl(f(z) A(x)),
    U0 the laminar profile of the forcing (fx/(2 nu)) z (Lz - z), f the wall
    envelope above and A_i = sum over k_x, k_y, k_z = 1..modes of
    S_i(k) sin(k.x) + C_i(k) cos(k.x), k = 2 pi (k_x/Lx, k_y/Ly, k_z/Lz), with
    S and C uniform on [0, 1] (seeded).  The curl is taken discretely on the
    MAC grid from psi = f A placed on the cell edges, so the field has zero
    discrete divergence and w = 0 at the walls.  The paper gives no
    amplitude for the curl term: taken with a = 1 its rms exceeds the base
    flow and the advective CFL number at the paper's dt is about 2.  Here a
    scales it to an rms (over the three components) of `intensity` times the
    peak of scale U0 (a = 1 when intensity is None).  Returns (u, v, w)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    Lx, Ly, Lz = cfg["Lx"], cfg["Ly"], cfg["Lz"]
    dx, dy = Lx / nx, Ly / ny
    zf, zc = zfaces(cfg), zcentres(cfg)
    S = rng.uniform(0.0, 1.0, (3, modes, modes, modes))
    C = rng.uniform(0.0, 1.0, (3, modes, modes, modes))
    kk = np.arange(1, modes + 1)
    kx, ky, kz = 2 * PI * kk / Lx, 2 * PI * kk / Ly, 2 * PI * kk / Lz

    def A(comp, x, y, z):
        """A_comp on the grid spanned by 1-D coordinate arrays x, y, z -> [z][y][x].
        S sin(k.x) + C cos(k.x) = Re[(C - i S) e^{i k.x}], and e^{i k.x}
        factors by axis, so the sum is taken one axis at a time."""
        coef = C[comp] - 1j * S[comp]                                   # [a][b][c]
        g = np.einsum("abc,cz->abz", coef, np.exp(1j * np.outer(kz, z)))
        h = np.einsum("abz,by->azy", g, np.exp(1j * np.outer(ky, y)))
        return np.einsum("azy,ax->zyx", h, np.exp(1j * np.outer(kx, x))).real

    xi, xh = dx * np.arange(nx + 1), dx * (np.arange(nx + 1) + 0.5)
    yj, yh = dy * np.arange(ny + 1), dy * (np.arange(ny + 1) + 0.5)
    # psi on the edges: psi_x at (x_{i+1/2}, y_j, zf), psi_y at (x_i, y_{j+1/2}, zf),
    # psi_z at (x_i, y_j, zc); one extra point along x and y for the differences
    psx = _paper_f(zf, Lz)[:, None, None] * A(0, xh, yj, zf)
    psy = _paper_f(zf, Lz)[:, None, None] * A(1, xi, yh, zf)
    psz = _paper_f(zc, Lz)[:, None, None] * A(2, xi, yj, zc)
    dzc = np.diff(zf)[:, None, None]
    # u at (x_i, y_{j+1/2}, zc): d psi_z/dy - d psi_y/dz
    u = (psz[:, 1:, :nx] - psz[:, :ny, :nx]) / dy - (psy[1:, :ny, :nx] - psy[:nz, :ny, :nx]) / dzc
    # v at (x_{i+1/2}, y_j, zc): d psi_x/dz - d psi_z/dx
    v = (psx[1:, :ny, :nx] - psx[:nz, :ny, :nx]) / dzc - (psz[:, :ny, 1:] - psz[:, :ny, :nx]) / dx
    # w at (x_{i+1/2}, y_{j+1/2}, zf): d psi_y/dx - d psi_x/dy
    w = (psy[:, :ny, 1:] - psy[:, :ny, :nx]) / dx - (psx[:, 1:, :nx] - psx[:, :ny, :nx]) / dy
    w[0] = 0.0
    w[-1] = 0.0
    U0 = cfg["fx"] / (2.0 * cfg["nu"]) * zc * (Lz - zc)
    if intensity is not None:
        rms = np.sqrt((np.sum(u * u) + np.sum(v * v) + np.sum(w[1:-1] * w[1:-1])) /
                      (u.size + v.size + w[1:-1].size))
        a = intensity * scale * np.abs(U0).max() / rms
        u, v, w = a * u, a * v, a * w
    return u + scale * U0[:, None, None], v, w


def initial_fields(name, cfg=None, seed=0):
    """Initial (u, v, w) of a named workload."""
    cfg = cfg or preset(name)
    if name == "laminar_startup":
        return zeros(cfg)
    if name == "os_instability":
        Re = 1.0 / cfg["nu"]
        alpha = 2 * PI / cfg["Lx"] * (0.5 * cfg["Lz"])
        u0, v0, w0 = poiseuille(cfg, 1.0)
        du, dv, dw, _ = os_mode(cfg, 1e-4, Re, alpha)
        return noise(cfg, 1e-6, seed, (u0 + du, v0 + dv, w0 + dw))
    if name == "les_channel":
        u0, v0, w0 = poiseuille(cfg, 1.5)
        return noise(cfg, 0.15, seed, (u0, v0, w0))
    if name == "les_paper":
        return paper_les_initial(cfg, seed)
    raise KeyError(name)
