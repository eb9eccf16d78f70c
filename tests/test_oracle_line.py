"""Pins of the oracle's z-line relaxation of the pressure solve (SRJ weights
applied to whole z columns solved exactly, Sec. 3.4 relaxation on lines).

Each check compares the C oracle's line sweep with something it does not
share code with: the spectrum of its own iteration matrix against the
separable enumeration of srj.line_bounds (scipy eigenvalues of the z
operator and the Fourier eigenvalues in x, y), a dense least-squares solve
of the Poisson problem, and the relaxation and fixed-point identities.
"""
import math

import numpy as np
import pytest

PI = math.pi


def cfg_of(nx, ny, nz, stretch, **over):
    c = dict(nx=nx, ny=ny, nz=nz, Lx=2 * PI, Ly=PI, Lz=2.0, nu=0.01, dt=1e-3, forcing=0, fx=0.0, ubulk=0.0,
             les=0, cs=0.1, vd_a=25.0, re_tau=180.0, stretch=stretch, cn_sweeps=4, ptol=1e-10, pmaxit=200000)
    c.update(over)
    return c


def dense_operator(fn, shape):
    n = int(np.prod(shape))
    M = np.zeros((n, n))
    for q in range(n):
        e = np.zeros(n)
        e[q] = 1.0
        M[:, q] = fn(e.reshape(shape)).ravel()
    return M


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_line_iteration_spectrum_is_separable(orc, stretch):
    """With b = 0 and omega = 1 a line sweep maps the error e to
    (I - A^-1(-L)) e.  The eigenvalues of A^-1(-L) taken from that dense
    iteration matrix equal, as a multiset, (tau + lam)/(tau + dxy) over the z
    eigenvalues tau and the x-y Fourier eigenvalues lam, and their extremes
    are the bounds srj.line_bounds returns."""
    from oracle import srj
    nx, ny, nz = 6, 4, 7
    cfg = cfg_of(nx, ny, nz, stretch)
    o = orc.Oracle(cfg)
    shape = (nz, ny, nx)
    zero = np.zeros(shape)
    G = dense_operator(lambda e: o.line_sweep(np.ascontiguousarray(e), zero, 1.0), shape)
    mu = np.sort(np.linalg.eigvals(np.eye(G.shape[0]) - G).real)
    # separable enumeration, from the z operator's own eigen-solve
    dz, cup, cdn, A0 = srj._z_operator(nz, cfg["Lz"], stretch)
    import scipy.linalg
    tau = scipy.linalg.eigh(A0, np.diag(dz), eigvals_only=True)
    dx, dy = cfg["Lx"] / nx, cfg["Ly"] / ny
    dxy = 2 / dx**2 + 2 / dy**2
    lam = ((4 / dx**2 * np.sin(PI * np.arange(nx) / nx) ** 2)[:, None] +
           (4 / dy**2 * np.sin(PI * np.arange(ny) / ny) ** 2)[None, :]).ravel()
    want = np.sort(((tau[:, None] + lam[None, :]) / (tau[:, None] + dxy)).ravel())
    want[0] = 0.0
    assert np.allclose(mu, want, atol=1e-9)
    mn, mx = srj.line_bounds(nx, ny, nz, cfg["Lx"], cfg["Ly"], cfg["Lz"], stretch)
    assert abs(mu[0]) < 1e-10
    assert abs(mu[1] - mn) < 1e-9 * max(1.0, mn) and abs(mu[-1] - mx) < 1e-9


def test_line_sweep_is_relaxation_with_fixed_point(orc):
    """p' = p + omega (p^L - p) for any omega, and a solution of L p = b is
    left unchanged by every sweep."""
    cfg = cfg_of(10, 6, 9, 2.0)
    o = orc.Oracle(cfg)
    rng = np.random.default_rng(5)
    p = rng.standard_normal((9, 6, 10))
    b = rng.standard_normal((9, 6, 10))
    pl = o.line_sweep(p, b, 1.0)
    for om in (0.25, 3.0, 40.0):
        assert np.allclose(o.line_sweep(p, b, om), p + om * (pl - p), atol=1e-9 * max(1.0, om))
    b2 = o.laplacian(p)
    for om in (1.0, 17.0):
        assert np.allclose(o.line_sweep(p, b2, om), p, atol=1e-10)


def test_line_srj_matches_dense_solve_and_beats_point_srj(orc):
    """Line SRJ with its Chebyshev schedule reaches the least-squares
    solution of the dense Poisson system (assembled from the oracle's
    Laplacian, solved by numpy), and on a wall-stretched grid it needs far
    fewer sweeps than point SRJ to the same tolerance."""
    from oracle import srj
    nx, ny, nz = 8, 6, 12
    base = cfg_of(nx, ny, nz, 2.0)
    o0 = orc.Oracle(base)
    shape = (nz, ny, nx)
    Lm = dense_operator(lambda e: o0.laplacian(np.ascontiguousarray(e)), shape)
    rng = np.random.default_rng(9)
    b = rng.standard_normal(shape)
    dz = np.diff(srj.z_grid(nz, base["Lz"], 2.0))
    w = np.broadcast_to(dz[:, None, None], shape).ravel()
    bv = b.ravel() - (b.ravel() * w).sum() / w.sum()       # volume-mean-free right-hand side
    pd = np.linalg.lstsq(Lm, bv, rcond=None)[0].reshape(shape)
    res = {}
    for line in (True, False):
        om, mn, mx = srj.schedule_for(nx, ny, nz, base["Lx"], base["Ly"], base["Lz"], 2.0, line=line)
        o = orc.Oracle(dict(base, omega=om, zline=int(line)))
        p, it, rel, conv = o.poisson(bv.reshape(shape), tol=1e-10, maxit=400000)
        assert conv and rel <= 1e-10
        vm = lambda a: a - (a * dz[:, None, None]).sum() / (dz.sum() * nx * ny)
        assert np.abs(vm(p) - vm(pd)).max() < 1e-7 * np.abs(pd).max()
        res[line] = it
    assert res[True] * 4 <= res[False], res      # sweep counts are whole cycles
