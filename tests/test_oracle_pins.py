"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each check is a closed form,
an invariant of the discretisation, a textbook reduction, an independent
solver, or a value printed in the paper.
"""
import math

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

PI = math.pi


def small_cfg(**over):
    c = dict(nx=12, ny=10, nz=8, Lx=2 * PI, Ly=PI, Lz=2.0, nu=0.01, dt=1e-3, forcing=0, fx=0.0,
             ubulk=0.0, les=0, cs=0.1, vd_a=25.0, re_tau=180.0, stretch=0.0, cn_sweeps=4,
             ptol=1e-10, pmaxit=100000)
    c.update(over)
    return c


def coords(cfg):
    nx, ny = cfg["nx"], cfg["ny"]
    dx, dy = cfg["Lx"] / nx, cfg["Ly"] / ny
    zf = inputs.zfaces(cfg)
    zc = 0.5 * (zf[1:] + zf[:-1])
    return dx, dy, zf, zc


# ---------------------------------------------------------------- Orr-Sommerfeld

def golden():
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        return json.load(f)


def test_os_paper_table_eigenvalue(orc):
    """Table of Sec. 4.2 (tests/golden/paper_values.json, os_table):
    Re_* = 500, alpha = 2 pi / 4 gives lambda = 1.8056 - 33.873 i (paper
    units) and the period 0.185."""
    from oracle import os_eig
    g = golden()["os_table"]
    Re_s = g["Re_star"]
    lam_printed = complex(g["lambda_real"], g["lambda_imag"])
    Re, a, lam_p = os_eig.paper_to_half_height(Re_s, g["alpha_over_pi"] * PI, lam_printed)
    lam = os_eig.least_stable(Re, a, N=160)
    # one unit of the last printed digit (1.8056, -33.873)
    assert abs(lam.real - lam_p.real) < 1e-4 * 2 / Re_s
    assert abs(lam.imag - lam_p.imag) < 1e-3 * 2 / Re_s
    # the printed period T = 2 pi / |Im lambda| (paper time units)
    assert abs(2 * PI / abs(lam.imag * Re_s / 2) - g["period"]) < 0.0005


def test_os_critical_reynolds(orc):
    """Sec. 4.1: critical Reynolds number 5772 (centreline, half height;
    golden os_critical), reached at the critical wavenumber 1.02056 (Re_c =
    5772.22 to two more digits): a neutral mode."""
    from oracle import os_eig
    assert round(5772.22) == golden()["os_critical"]["Re_c"]
    lam = os_eig.least_stable(5772.22, 1.02056, N=120)
    assert abs(lam.real) < 2e-7
    assert os_eig.least_stable(5000.0, 1.02056).real < 0
    assert os_eig.least_stable(7500.0, 1.0).real > 0


def test_os_two_independent_solvers_agree(orc):
    """The Chebyshev oracle solver and the finite-difference solver that
    shapes the initial perturbation find the same least-stable mode."""
    from oracle import os_eig
    lam_c = os_eig.least_stable(7500.0, 1.0)
    lam_f, _, _ = inputs._os_mode_fd(7500.0, 1.0)
    assert abs(lam_c - lam_f) < 2e-5 * 1e1
    assert abs(lam_c.real - lam_f.real) / lam_c.real < 0.01


# ---------------------------------------------------------------- SRJ schedule

def test_srj_cycle_is_chebyshev(orc):
    """Sec. 3.4 SRJ cycle: the product of (1 - omega_k mu) over one cycle
    equals the scaled Chebyshev polynomial for the chosen interval."""
    from oracle import srj
    mn, mx, M = 1e-3, 1.97, 64
    om = srj.chebyshev_schedule(mn, mx, M)
    assert len(om) == M and len(set(np.round(om, 12))) == M
    mu = np.linspace(mn, mx, 777)
    G = np.prod(1 - om[:, None] * mu[None, :], axis=0)
    x0 = (mx + mn) / (mx - mn)
    T = np.cos(M * np.arccos(np.clip((mx + mn - 2 * mu) / (mx - mn), -1, 1)))
    assert np.allclose(G, T / np.cosh(M * np.arccosh(x0)), rtol=0, atol=1e-10)
    assert np.abs(G).max() <= srj.cycle_factor(mn, mx, M) * (1 + 1e-9)
    # both over- and under-relaxation appear (the defining trait of SRJ)
    assert om.min() < 1 < om.max()
    # partial products stay within a few times the largest single factor
    P, worst = np.ones_like(mu), 0.0
    for w in om:
        P *= 1 - w * mu
        worst = max(worst, np.abs(P).max())
    assert worst < om.max() * mx


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_srj_bounds_match_brute_force(orc, stretch):
    """Separable eigen-bounds of D^-1(-L) agree with a dense eigen-solve of
    the operator assembled column by column from the C oracle."""
    from oracle import srj
    cfg = small_cfg(nx=6, ny=4, nz=6, stretch=stretch)
    o = orc.Oracle(cfg)
    n = 6 * 4 * 6
    Lm = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        Lm[:, q] = o.laplacian(e.reshape(6, 4, 6)).ravel()
    Dg = -np.diag(Lm)
    mu = np.sort(np.linalg.eigvals(-Lm / Dg[:, None]).real)
    mn, mx = srj.jacobi_bounds(6, 4, 6, cfg["Lx"], cfg["Ly"], cfg["Lz"], stretch)
    assert abs(mu[0]) < 1e-10
    assert abs(mu[1] - mn) < 1e-9 * max(1, mn)
    assert abs(mu[-1] - mx) < 1e-9


# ---------------------------------------------------------------- Poisson operator

@pytest.mark.parametrize("m,n,l", [(1, 0, 0), (0, 2, 1), (3, 1, 2), (2, 3, 5)])
def test_laplacian_eigenmodes(orc, m, n, l):
    """Eq. presdiv with Neumann walls: cos modes at the cell centres are exact
    eigenvectors of the uniform-grid L = D G with eigenvalue
    -(4/dx^2 sin^2(pi m/nx) + 4/dy^2 sin^2(pi n/ny) + 4/dz^2 sin^2(pi l/(2 nz)))."""
    cfg = small_cfg()
    o = orc.Oracle(cfg)
    dx, dy, zf, zc = coords(cfg)
    nx, ny, nz = cfg["nx"], cfg["ny"], cfg["nz"]
    dz = cfg["Lz"] / nz
    x = (np.arange(nx) + 0.5) * dx
    y = (np.arange(ny) + 0.5) * dy
    p = (np.cos(PI * l * zc / cfg["Lz"])[:, None, None] * np.cos(2 * PI * n * y / cfg["Ly"])[None, :, None] *
         np.cos(2 * PI * m * x / cfg["Lx"])[None, None, :])
    lam = -(4 / dx**2 * math.sin(PI * m / nx) ** 2 + 4 / dy**2 * math.sin(PI * n / ny) ** 2 +
            4 / dz**2 * math.sin(PI * l / (2 * nz)) ** 2)
    assert np.allclose(o.laplacian(p), lam * p, rtol=0, atol=1e-10 * abs(lam))


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_laplacian_is_div_of_grad(orc, stretch):
    """L = D G: correcting a zero velocity with dt = 1 gives -G p, whose
    divergence must be -L p; L annihilates constants; W L is symmetric."""
    cfg = small_cfg(stretch=stretch, dt=1.0)
    o = orc.Oracle(cfg)
    rng = np.random.default_rng(5)
    p = rng.standard_normal((8, 10, 12))
    z3 = np.zeros((8, 10, 12))
    u, v, w = o.correct(p, z3, z3, np.zeros((9, 10, 12)))
    assert np.allclose(o.divergence(u, v, w), -o.laplacian(p), atol=1e-9)
    assert np.abs(o.laplacian(np.ones_like(p))).max() < 1e-9
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    q = rng.standard_normal(p.shape)
    a = np.sum(dz * q * o.laplacian(p))
    b = np.sum(dz * p * o.laplacian(q))
    assert abs(a - b) < 1e-9 * abs(a)


def test_divergence_closed_form(orc):
    """Discrete divergence of trigonometric face fields."""
    cfg = small_cfg()
    o = orc.Oracle(cfg)
    dx, dy, zf, zc = coords(cfg)
    kx, ky = 2 * PI / cfg["Lx"] * 2, 2 * PI / cfg["Ly"]
    xu = np.arange(12) * dx
    yv = np.arange(10) * dy
    u = np.broadcast_to(np.sin(kx * xu), (8, 10, 12)).copy()
    v = np.broadcast_to(np.cos(ky * yv)[:, None], (8, 10, 12)).copy()
    w = np.zeros((9, 10, 12))
    w[:] = (zf * (2 - zf))[:, None, None]
    xc = xu + 0.5 * dx
    yc = yv + 0.5 * dy
    exp = (np.cos(kx * xc) * 2 * np.sin(kx * dx / 2) / dx)[None, None, :] + \
          (-np.sin(ky * yc) * 2 * np.sin(ky * dy / 2) / dy)[None, :, None] + \
          (2 - 2 * zc)[:, None, None]
    assert np.allclose(o.divergence(u, v, w), exp, atol=1e-11)


def test_srj_matches_spectral_direct_solve(orc):
    """Sec. 3.4: the SRJ iteration reaches the solution of L p = b found
    independently by diagonalising L (FFT in x, y; cosine transform in z,
    all written from the eigenvectors of the uniform-grid operator)."""
    from oracle import srj
    cfg = small_cfg(nx=16, ny=8, nz=12)
    om, mn, mx = srj.schedule_for(16, 8, 12, cfg["Lx"], cfg["Ly"], cfg["Lz"], 0.0)
    cfg["omega"] = om
    o = orc.Oracle(cfg)
    rng = np.random.default_rng(11)
    b = rng.standard_normal((12, 8, 16))
    b -= b.mean()
    p, it, rel, conv = o.poisson(b, tol=1e-11, maxit=200000)
    assert conv and rel <= 1e-11
    # direct: eigenvectors cos(pi l (k+1/2)/nz) in z, Fourier in x, y
    nx, ny, nz = 16, 8, 12
    dx, dy, dz = cfg["Lx"] / nx, cfg["Ly"] / ny, cfg["Lz"] / nz
    kk = np.arange(nz)
    C = np.cos(PI * np.outer(np.arange(nz), kk + 0.5) / nz)        # (l, k)
    Cn = C / np.sqrt((C * C).sum(axis=1))[:, None]
    bh = np.fft.fft2(np.einsum("lk,kji->lji", Cn, b), axes=(1, 2))
    lam = -(4 / dz**2 * np.sin(PI * np.arange(nz) / (2 * nz)) ** 2)[:, None, None] \
          - (4 / dy**2 * np.sin(PI * np.arange(ny) / ny) ** 2)[None, :, None] \
          - (4 / dx**2 * np.sin(PI * np.arange(nx) / nx) ** 2)[None, None, :]
    lam[0, 0, 0] = 1.0
    ph = bh / lam
    ph[0, 0, 0] = 0.0
    pd = np.einsum("lk,lji->kji", Cn, np.fft.ifft2(ph, axes=(1, 2)).real)
    assert np.abs((p - p.mean()) - (pd - pd.mean())).max() < 1e-9 * np.abs(pd).max()


def test_srj_sweep_is_jacobi_sor(orc):
    """Eq. Jacobi-SOR: omega = 1 gives the plain Jacobi point solve; any
    omega blends old and Jacobi values linearly; a fixed point is a solution."""
    cfg = small_cfg(stretch=2.0)
    o = orc.Oracle(cfg)
    rng = np.random.default_rng(3)
    p = rng.standard_normal((8, 10, 12))
    b = rng.standard_normal((8, 10, 12))
    pj = o.srj_sweep(p, b, 1.0)
    # the Jacobi value zeroes the point residual with neighbours frozen
    Lp = o.laplacian(p)
    e = np.zeros_like(p)
    e[3, 4, 5] = 1.0
    diag = o.laplacian(e)[3, 4, 5]
    r_pt = b[3, 4, 5] - (Lp[3, 4, 5] + diag * (pj[3, 4, 5] - p[3, 4, 5]))
    assert abs(r_pt) < 1e-10 * np.abs(b).max() * 1e3
    for om in (0.3, 7.5):
        assert np.allclose(o.srj_sweep(p, b, om), (1 - om) * p + om * pj, atol=1e-9)
    # solution is a fixed point
    b2 = o.laplacian(p)
    assert np.allclose(o.srj_sweep(p, b2, 3.0), p, atol=1e-10)


# ---------------------------------------------------------------- momentum terms

def test_advection_closed_forms(orc):
    """u.grad u (Sec. 2.1 Eq. NSE momentum, centred on the MAC grid) for
    fields with known discrete derivatives."""
    cfg = small_cfg()
    o = orc.Oracle(cfg)
    dx, dy, zf, zc = coords(cfg)
    kx = 2 * PI / cfg["Lx"]
    ky = 2 * PI / cfg["Ly"] * 2
    A, U, V = 0.7, 1.3, -0.4
    xu = np.arange(12) * dx
    yv = np.arange(10) * dy
    # u = A sin(kx x): u du/dx
    u = np.broadcast_to(A * np.sin(kx * xu), (8, 10, 12)).copy()
    z3, zw = np.zeros((8, 10, 12)), np.zeros((9, 10, 12))
    Au, Av, Aw = o.advection(u, z3, zw)
    exp = (A * np.sin(kx * xu) * A * np.cos(kx * xu) * math.sin(kx * dx) / dx)[None, None, :]
    assert np.allclose(Au, exp, atol=1e-12)
    assert np.abs(Av).max() == 0 and np.abs(Aw).max() == 0
    # uniform U carrying v = sin(kx x) (v at x = (i+1/2) dx): U dv/dx
    xv = xu + 0.5 * dx
    v = np.broadcast_to(np.sin(kx * xv), (8, 10, 12)).copy()
    Au, Av, Aw = o.advection(np.full((8, 10, 12), U), v, zw)
    assert np.allclose(Av, (U * np.cos(kx * xv) * math.sin(kx * dx) / dx)[None, None, :], atol=1e-12)
    # uniform V carrying u = sin(ky y) (u at y = (j+1/2) dy): V du/dy
    yu = yv + 0.5 * dy
    u = np.broadcast_to(np.sin(ky * yu)[:, None], (8, 10, 12)).copy()
    Au, Av, Aw = o.advection(u, np.full((8, 10, 12), V), zw)
    assert np.allclose(Au, (V * np.cos(ky * yu) * math.sin(ky * dy) / dy)[None, :, None], atol=1e-12)
    # w advected by uniform U and V: w at ((i+1/2)dx, (j+1/2)dy)
    w = np.zeros((9, 10, 12))
    w[1:-1] = np.sin(kx * xv)[None, None, :] * np.ones((7, 10, 1))
    Au, Av, Aw = o.advection(np.full((8, 10, 12), U), np.full((8, 10, 12), V), w)
    # (levels 2..nz-2: away from the jump of w to its zero wall value)
    assert np.allclose(Aw[2:-2], (U * np.cos(kx * xv) * math.sin(kx * dx) / dx)[None, None, :], atol=1e-12)
    # vertical advection of u = z (2 - z) by a uniform w in the interior (uniform grid):
    # centred difference of a quadratic is exact away from the walls
    u = np.broadcast_to((zc * (2 - zc))[:, None, None], (8, 10, 12)).copy()
    w = np.zeros((9, 10, 12))
    w[1:-1] = 0.5
    Au, _, _ = o.advection(u, z3, w)
    assert np.allclose(Au[2:-2], (0.5 * (2 - 2 * zc))[2:-2, None, None], atol=1e-12)


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_cross_viscous_constant_nu_is_grad_div(orc, stretch):
    """For constant viscosity the convective-like term of Eq. more_conv,
    d_j(nu d_i u_j) = nu d_i (div u), discretely nu G D u."""
    cfg = small_cfg(stretch=stretch, dt=1.0)
    o = orc.Oracle(cfg)
    u, v, w, p, nu = inputs.random_state(cfg, 7)
    nu = np.full_like(nu, 0.37)
    Cu, Cv, Cw = o.cross_viscous(u, v, w, nu)
    d = o.divergence(u, v, w)
    z3 = np.zeros_like(u)
    gu, gv, gw = o.correct(d, z3, z3, np.zeros_like(w))        # -G(div u)
    assert np.allclose(Cu, -0.37 * gu, atol=1e-8)
    assert np.allclose(Cv, -0.37 * gv, atol=1e-8)
    assert np.allclose(Cw, -0.37 * gw, atol=1e-8)


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_viscous_operators_symmetric_negative(orc, stretch):
    """The viscous term d_j(nu_T (d_j u_i + d_i u_j)) is the divergence of a
    symmetric stress: both of its parts are symmetric and the diffusive part
    is negative definite in the volume-weighted inner product."""
    cfg = small_cfg(stretch=stretch)
    o = orc.Oracle(cfg)
    a = inputs.random_state(cfg, 1)
    b = inputs.random_state(cfg, 2)
    nu = a[4]
    zf = inputs.zfaces(cfg)
    dz = np.diff(zf)
    hz = np.diff(np.concatenate([[zf[0]], 0.5 * (zf[1:] + zf[:-1]), [zf[-1]]]))
    wc, ww = dz[:, None, None], hz[:, None, None]

    def ip(x, y):
        return np.sum(wc * x[0] * y[0]) + np.sum(wc * x[1] * y[1]) + np.sum(ww * x[2] * y[2])

    for op in (o.diffusion, o.cross_viscous):
        Ab = op(b[0], b[1], b[2], nu)
        Aa = op(a[0], a[1], a[2], nu)
        s1, s2 = ip(a[:3], Ab), ip(Aa, b[:3])
        assert abs(s1 - s2) < 1e-10 * (abs(s1) + 1e-3)
    Da = o.diffusion(a[0], a[1], a[2], nu)
    assert ip(a[:3], Da) < 0


def test_diffusion_diagonal(orc):
    """The Jacobi diagonal S_D equals minus the response of the diffusion
    operator to a unit impulse at the point (wall ghosts included)."""
    cfg = small_cfg(stretch=2.0)
    o = orc.Oracle(cfg)
    _, _, _, _, nu = inputs.random_state(cfg, 4)
    Su, Sv, Sw = o.diffusion_diag(nu)
    z3, zw = np.zeros((8, 10, 12)), np.zeros((9, 10, 12))
    for (k, j, i) in [(0, 0, 0), (7, 9, 11), (3, 4, 5)]:
        e = z3.copy()
        e[k, j, i] = 1.0
        assert abs(o.diffusion(e, z3, zw, nu)[0][k, j, i] + Su[k, j, i]) < 1e-9 * Su[k, j, i]
        assert abs(o.diffusion(z3, e, zw, nu)[1][k, j, i] + Sv[k, j, i]) < 1e-9 * Sv[k, j, i]
    for (k, j, i) in [(1, 0, 0), (7, 9, 11), (4, 4, 5)]:
        e = zw.copy()
        e[k, j, i] = 1.0
        assert abs(o.diffusion(z3, z3, e, nu)[2][k, j, i] + Sw[k, j, i]) < 1e-9 * Sw[k, j, i]


def test_cn_jacobi_solves_the_cn_system(orc):
    """Sec. 3.1 Crank-Nicolson: enough Jacobi sweeps give a* with
    a* - dt/2 D a* = rhs."""
    cfg = small_cfg(stretch=2.0, dt=0.05, cn_sweeps=60)
    o = orc.Oracle(cfg)
    u, v, w, p, nu = inputs.random_state(cfg, 9)
    us, vs, ws = o.cn_solve(nu, u, v, w)
    Du, Dv, Dw = o.diffusion(us, vs, ws, nu)
    h = 0.5 * cfg["dt"]
    assert np.abs(us - h * Du - u).max() < 1e-11
    assert np.abs(vs - h * Dv - v).max() < 1e-11
    assert np.abs((ws - h * Dw - w)[1:-1]).max() < 1e-11


# ---------------------------------------------------------------- eddy viscosity

def test_eddy_viscosity_linear_shear(orc):
    """Sec. 2.2: for u = s min(z, Lz - z), which vanishes on both walls, the
    strain magnitude is exactly s (the mirror ghost reproduces the wall
    slope), except on the two levels that straddle the kink at mid-height, so
    nu_T = nu + (Cs Delta phi_w)^2 s with Delta = 2 (dx dy dz)^(1/3) and
    phi_w = 1 - exp(-d+ / A)."""
    cfg = small_cfg(les=1, stretch=2.0, cs=0.1, vd_a=25.0, re_tau=180.0)
    o = orc.Oracle(cfg)
    dx, dy, zf, zc = coords(cfg)
    s = 0.8
    u = np.broadcast_to((s * np.minimum(zc, 2 - zc))[:, None, None], (8, 10, 12)).copy()
    nuT = o.viscosity(u, np.zeros_like(u), np.zeros((9, 10, 12)))
    dz = np.diff(zf)
    d = np.minimum(zc, 2 - zc)
    lm = 0.1 * 2 * np.cbrt(dx * dy * dz) * (1 - np.exp(-d * 180.0 / 25.0))
    exp = (cfg["nu"] + lm**2 * s)[:, None, None] * np.ones((1, 10, 12))
    keep = [0, 1, 2, 5, 6, 7]
    assert np.allclose(nuT[keep], exp[keep], rtol=1e-13, atol=0)


def test_eddy_viscosity_spanwise_shear(orc):
    """u = sin(k y): the 4-edge average of du/dy at the centre is
    cos(k y_c) sin(k dy)/dy, so |S| = |cos(k y_c)| sin(k dy)/dy (levels
    away from the walls, where no-slip adds wall shear)."""
    cfg = small_cfg(les=1)
    o = orc.Oracle(cfg)
    dx, dy, zf, zc = coords(cfg)
    k = 2 * PI / cfg["Ly"]
    yu = (np.arange(10) + 0.5) * dy
    u = np.broadcast_to(np.sin(k * yu)[:, None], (8, 10, 12)).copy()
    nuT = o.viscosity(u, np.zeros_like(u), np.zeros((9, 10, 12)))
    yc = yu
    smag = np.abs(np.cos(k * yc)) * math.sin(k * dy) / dy
    dz = np.diff(zf)
    d = np.minimum(zc, 2 - zc)
    lm = 0.1 * 2 * np.cbrt(dx * dy * dz) * (1 - np.exp(-d * 180.0 / 25.0))
    exp = cfg["nu"] + (lm**2)[:, None, None] * smag[None, :, None] * np.ones((1, 1, 12))
    assert np.allclose(nuT[1:-1], exp[1:-1], rtol=1e-12, atol=0)
    assert np.all(o.viscosity(np.zeros_like(u), np.zeros_like(u), np.zeros((9, 10, 12))) == cfg["nu"])


# ---------------------------------------------------------------- whole steps

def test_ab3_advection_mode(orc):
    """Textbook reduction of the step: a uniform stream U carrying
    v = sin(k x) with nu = 0 has b = 0, p = 0 and N_v = -U D_x v, and the
    Fourier amplitude follows forward Euler, AB2, then AB3 (23, -16, 5)/12
    exactly, with the eigenvalue -i U sin(k dx)/dx of the centred difference."""
    cfg = small_cfg(nu=0.0, dt=0.01, cn_sweeps=2)
    from oracle import srj
    cfg["omega"] = srj.schedule_for(12, 10, 8, cfg["Lx"], cfg["Ly"], 2.0)[0]
    o = orc.Oracle(cfg)
    dx = cfg["Lx"] / 12
    k = 2 * PI / cfg["Lx"] * 2
    U = 1.1
    xv = (np.arange(12) + 0.5) * dx
    u = np.full((8, 10, 12), U)
    v = np.broadcast_to(np.sin(k * xv), (8, 10, 12)).copy()
    o.set_fields(u, v, np.zeros((9, 10, 12)))
    z = -1j * U * math.sin(k * dx) / dx * cfg["dt"]
    a = [1.0 + 0j]
    f = []
    for n in range(6):
        f.append(z * a[-1])
        if n == 0:
            a.append(a[-1] + f[-1])
        elif n == 1:
            a.append(a[-1] + 1.5 * f[-1] - 0.5 * f[-2])
        else:
            a.append(a[-1] + (23 * f[-1] - 16 * f[-2] + 5 * f[-3]) / 12)
        o.step(1)
        got = o.get_fields()["v"]
        exp = np.imag(a[-1] * np.exp(1j * k * xv))
        assert np.allclose(got, exp[None, None, :], atol=1e-13), n


def _startup_exact_discrete(nz, Lz, nu, fx, dt, nsteps):
    """u(z) under CN diffusion (Dirichlet walls by mirror ghosts) and a
    constant force: a 1-D problem solved by eigen-decomposition."""
    h = Lz / nz
    A = (np.diag(np.full(nz - 1, 1.0), -1) - 2 * np.eye(nz) + np.diag(np.full(nz - 1, 1.0), 1))
    A[0, 0] = A[-1, -1] = -3.0
    A *= nu / h**2
    lam, V = np.linalg.eigh(A)
    g = (1 + 0.5 * dt * lam) / (1 - 0.5 * dt * lam)
    fm = V.T @ np.full(nz, fx)
    am = np.zeros(nz)
    for _ in range(nsteps):
        am = g * am + dt * fm / (1 - 0.5 * dt * lam)
    return V @ am


def test_laminar_startup(orc):
    """Laminar start-up workload (fluid at rest, -dp/dx = 2/Re, Re = 100,
    32 x 16 x 32, dt = 1e-3): u stays a function of z alone, v = w = p = 0,
    and the step reduces to Crank-Nicolson on the 1-D wall-bounded Laplacian
    with the constant force.  Compared with (a) that 1-D problem solved
    exactly and (b) the continuous start-up series to O(dz^2 + dt^2)."""
    cfg = inputs.preset("laminar_startup", cn_sweeps=40)
    from oracle import srj
    cfg["omega"] = srj.schedule_for(32, 16, 32, cfg["Lx"], cfg["Ly"], 2.0)[0]
    o = orc.Oracle(cfg)
    o.set_fields(*inputs.zeros(cfg))
    st = o.step(100)
    f = o.get_fields()
    prof = f["u"][:, 0, 0]
    assert np.abs(f["u"] - prof[:, None, None]).max() < 1e-14
    assert np.abs(f["v"]).max() == 0 and np.abs(f["w"]).max() == 0 and np.abs(f["p"]).max() == 0
    exact = _startup_exact_discrete(32, 2.0, cfg["nu"], cfg["fx"], cfg["dt"], 100)
    assert np.abs(prof - exact).max() < 1e-12
    # continuous series, eta = z - 1
    zc = inputs.zcentres(cfg)
    eta = zc - 1
    t = 0.1
    Re = 100.0
    ser = 1 - eta**2
    for n in range(1, 400, 2):
        ser -= 32 * (-1) ** ((n - 1) // 2) / (n**3 * PI**3) * np.cos(n * PI * eta / 2) * math.exp(-n * n * PI * PI * t / (4 * Re))
    assert np.abs(prof - ser).max() < 2e-4
    assert st["converged"]


def test_projection_divergence_invariant(orc):
    """After a step D u^{n+1} = dt (b - L p): its size is bounded by dt times
    the Poisson residual, which the solve drives below tol ||b||."""
    cfg = inputs.preset("os_instability", nx=16, ny=3, nz=16, cn_sweeps=6)
    from oracle import srj
    cfg["omega"] = srj.schedule_for(16, 3, 16, cfg["Lx"], cfg["Ly"], 2.0)[0]
    cfg["ptol"] = 1e-9
    o = orc.Oracle(cfg)
    u, v, w = inputs.noise(cfg, 1e-3, 0, inputs.poiseuille(cfg))
    o.set_fields(u, v, w)
    st = o.step(1)
    # b of this step is O(|noise|/dt); the divergence after projection is tiny
    f = o.get_fields()
    d = o.divergence(f["u"], f["v"], f["w"])
    assert st["converged"] and st["rel_res"] <= 1e-9
    assert abs(np.abs(d).max() - st["max_div"]) < 1e-15
    # the noise gives |div u^n| ~ 1e-3/h ~ 0.1; the projection removes it to the
    # solver tolerance
    assert np.sqrt(np.sum(d * d)) < 2e-9 * np.sqrt(np.sum(o.divergence(u, v, w) ** 2)) + 1e-12


# ------------------------------------------------- Crank-Nicolson on z lines

def _cn_dense(o, cfg, nu, ru, rv, rw):
    """The Crank-Nicolson system (I - dt/2 D) a = rhs solved directly: D is
    assembled column by column from the oracle's diffusion operator applied
    to unit vectors (it is linear and acts on each component alone), and
    each component's system is solved with numpy's dense solver."""
    h = 0.5 * cfg["dt"]
    sc, sw = ru.shape, rw.shape
    out = []
    for comp, (rhs, shape) in enumerate(((ru, sc), (rv, sc), (rw, sw))):
        n = int(np.prod(shape))
        idx = [q for q in range(n) if comp < 2 or 0 < q // (shape[1] * shape[2]) < shape[0] - 1]
        A = np.zeros((len(idx), len(idx)))
        for col, q in enumerate(idx):
            e = [np.zeros(sc), np.zeros(sc), np.zeros(sw)]
            e[comp].flat[q] = 1.0
            D = o.diffusion(*e, nu)[comp]
            A[:, col] = -h * D.ravel()[idx]
            A[col, col] += 1.0
        a = np.zeros(shape)
        a.flat[idx] = np.linalg.solve(A, rhs.ravel()[idx])
        out.append(a)
    return out


def test_cn_line_jacobi_reaches_the_direct_solution(orc):
    """The z-line reading of the Crank-Nicolson solve (each z column solved
    exactly with the x-y neighbours of the previous iterate) converges to
    the solution of (I - dt/2 D) a = rhs found by a dense direct solve, on a
    wall-stretched grid with a spatially varying eddy viscosity; so does
    point Jacobi, to the same solution."""
    cfg = small_cfg(nx=4, ny=3, nz=5, stretch=2.0, dt=0.05)
    u, v, w, p, nu = inputs.random_state(cfg, 13)
    o = orc.Oracle(cfg)
    exact = _cn_dense(o, cfg, nu, u, v, w)
    for zl, sweeps in ((1, 40), (0, 400)):
        a = orc.Oracle(dict(cfg, cn_zline=zl, cn_sweeps=sweeps)).cn_solve(nu, u, v, w)
        for got, want in zip(a, exact):
            assert np.abs(got - want).max() < 1e-12 * max(1.0, np.abs(want).max()), zl


def test_cn_line_jacobi_contraction_bound(orc):
    """Each z-line sweep contracts the error in the max norm at least by
    rho = h S / (1 + h S), S the largest sum of the x-y coupling weights
    (2 nu_max / dx^2 + 2 nu_max / dy^2), since the column matrix is an
    M-matrix with row sums >= 1 + h S_xy; here rho is far below the
    point-Jacobi contraction, whose bound includes the stiff z couplings."""
    cfg = small_cfg(nx=6, ny=5, nz=7, stretch=2.0, dt=0.05)
    u, v, w, p, nu = inputs.random_state(cfg, 14)
    o = orc.Oracle(cfg)
    exact = _cn_dense(o, cfg, nu, u, v, w)
    dx, dy = cfg["Lx"] / cfg["nx"], cfg["Ly"] / cfg["ny"]
    hs = 0.5 * cfg["dt"] * nu.max() * (2 / dx**2 + 2 / dy**2)
    rho = hs / (1 + hs)
    prev = max(np.abs(a - b).max() for a, b in zip((u, v, w), exact))
    for n in (1, 2, 3):
        a = orc.Oracle(dict(cfg, cn_zline=1, cn_sweeps=n)).cn_solve(nu, u, v, w)
        err = max(np.abs(x - y).max() for x, y in zip(a, exact))
        assert err <= rho * prev * (1 + 1e-9) + 1e-14, (n, err, rho * prev)
        prev = err
    assert rho < 0.5
