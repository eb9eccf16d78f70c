"""Pins of the oracle's LES statistics (Sec. 6) against closed forms, and
the library's bulk post-processing against the same closed forms."""
import math

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs, les

PI = math.pi


def test_moments_and_correlation_of_cosine_modes():
    """u = U(z) + a cos(2 pi m x/Lx): the centre value carries the mode with
    amplitude a cos(pi m/nx); R_uu(d) = (a^2/2) cos(2 pi m d/nx) on the faces."""
    from oracle import les_stats
    nx, ny, nz, m, a = 24, 6, 5, 3, 0.7
    x = np.arange(nx)
    U = np.linspace(1.0, 2.0, nz)
    u = U[:, None, None] + a * np.cos(2 * PI * m * x / nx)[None, None, :] * np.ones((nz, ny, nx))
    v = np.zeros((nz, ny, nx))
    w = np.zeros((nz + 1, ny, nx))
    mom = les_stats.plane_moments(u, v, w)
    ac = a * math.cos(PI * m / nx)
    assert np.allclose(mom[0], U, atol=1e-13)
    assert np.allclose(mom[3], U ** 2 + ac * ac / 2, atol=1e-12)
    assert np.allclose(mom[[1, 2, 4, 5, 6, 7, 8]], 0.0, atol=1e-14)
    c = les_stats.corr_x(u, v, w, 2)
    R = c[0] - U[2] ** 2
    assert np.allclose(R, a * a / 2 * np.cos(2 * PI * m * x / nx), atol=1e-12)


@pytest.mark.parametrize("which", ["oracle", "library"])
def test_bulk_of_the_laminar_profile(which):
    """The laminar profile of the paper's units, Re_* z (1 - z): bulk velocity
    Re_*/6 and wall shear nu Re_* = 1 (u_tau = 1), to the grid's accuracy.
    The same closed forms pin the oracle's bulk quantities and the library's
    host post-processing (les.bulk), each on its own."""
    from oracle import les_stats
    cfg = inputs.preset("les_paper")
    zc = inputs.zcentres(cfg)
    re = 1.0 / cfg["nu"]
    prof = re * zc * (1 - zc)
    b = les_stats.bulk(prof, inputs.zfaces(cfg), cfg["nu"]) if which == "oracle" else les.bulk(cfg, prof)
    dz = 1.0 / cfg["nz"]
    assert abs(b["U_mean"] - re / 6) < re * dz * dz
    assert abs(b["u_tau"] - 1.0) < dz
    assert abs(b["U_max"] - re / 4) < re * dz * dz
    assert abs(b["Cf"] - 2 / b["U_mean"] ** 2) < 4 * dz / b["U_mean"] ** 2
    assert abs(b["pope_Umax_over_utau"] - (math.log(b["Re_tau"]) / 0.4 + 3.47)) < 1e-12
    assert abs(b["dean_Cf"] - 0.073 * (b["U_mean"] / cfg["nu"]) ** -0.25) < 1e-15
    # on a stretched grid the midpoint rule is still exact for the linear
    # part of a profile: a constant profile has U_mean = U_max = the constant
    cs = inputs.preset("les_paper", stretch=1.5)
    flat = np.full(cs["nz"], 3.25)
    bs = les_stats.bulk(flat, inputs.zfaces(cs), cs["nu"]) if which == "oracle" else les.bulk(cs, flat)
    assert abs(bs["U_mean"] - 3.25) < 1e-13 and bs["U_max"] == 3.25


def test_paper_initial_condition_is_divergence_free(orc):
    """The paper's turbulent-like start: zero discrete divergence (the curl of
    an edge potential), w = 0 at the walls, plane mean of u exactly U0/3."""
    cfg = inputs.preset("les_paper", nx=24, ny=14, nz=12)
    u, v, w = inputs.paper_les_initial(cfg, 3)
    o = orc.Oracle(dict(cfg, omega=[1.0]))
    scale = np.abs(u).max() / (cfg["Lx"] / cfg["nx"])
    assert np.abs(o.divergence(u, v, w)).max() < 1e-13 * scale
    assert np.abs(w[0]).max() == 0.0 and np.abs(w[-1]).max() == 0.0
    zc = inputs.zcentres(cfg)
    U0 = cfg["fx"] / (2 * cfg["nu"]) * zc * (cfg["Lz"] - zc)
    assert np.allclose(u.mean(axis=(1, 2)), U0 / 3, atol=1e-12 * U0.max())
    assert np.abs(v.mean(axis=(1, 2))).max() < 1e-12 * np.abs(v).max()
    assert (u - u.mean(axis=(1, 2), keepdims=True)).std() > 1.0


def _paper_like_profile(nz, nu, U_mean, U_cl):
    """A symmetric mean profile on nz (odd) uniform cells over height 1:
    linear at the wall with friction velocity 1 (u = z/nu at the first
    centre), a parabolic core peaking at U_cl on the centre cell, its
    curvature chosen (bisection) so that the volume mean is U_mean."""
    zc = (np.arange(nz) + 0.5) / nz
    d = np.minimum(zc, 1.0 - zc)

    def prof(A):
        return np.minimum(d / nu, U_cl - A * (0.5 - d) ** 2)

    lo, hi = 0.0, 1e4
    for _ in range(200):
        A = 0.5 * (lo + hi)
        if prof(A).mean() > U_mean:
            lo = A
        else:
            hi = A
    u = prof(0.5 * (lo + hi))
    assert abs(u.mean() - U_mean) < 1e-9 and u[0] == d[0] / nu and u.max() == U_cl
    return u


def test_bulk_definitions_reproduce_the_paper_numbers():
    """Sec. 6 prints U_mean = 15.39, Re_mean = U_mean H/nu = 5542, U_cl =
    18.30, the Pope estimate (1/0.4) log Re_* + 3.47 = 18.18, U_max/U_mean =
    1.19, C_f = 2 u_*^2/U_mean^2 = 8.44e-3 and Dean's 0.073 Re_mean^-0.25 =
    8.46e-3 (tests/golden/paper_values.json, les_bulk).  A mean profile with
    friction velocity 1, the printed U_mean and U_cl, on the paper's height 1
    and nu = 1/Re_* = 1/360, gives every derived number to its last printed
    digit through the oracle's and the library's bulk definitions (a height
    of 2 in Re_mean, a missing factor 2 in C_f or a half-cell wall distance
    taken as a whole cell would each fail)."""
    import json
    import os
    from oracle import les_stats
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")) as f:
        g = json.load(f)["les_bulk"]
    nu = 1.0 / g["Re_star"]
    nz = 201
    u = _paper_like_profile(nz, nu, g["U_mean"], g["U_cl"])
    zf = np.linspace(0.0, 1.0, nz + 1)
    cfg = inputs.preset("les_paper", nz=nz)
    assert cfg["Lz"] == 1.0 and cfg["nu"] == nu and cfg.get("stretch", 0.0) == 0.0
    for b in (les_stats.bulk(u, zf, nu), les.bulk(cfg, u)):
        assert abs(b["u_tau"] - 1.0) < 1e-12
        assert abs(b["Re_tau"] - g["Re_star"]) < 1e-9
        # Re_mean to half a unit of U_mean's last printed digit (0.005 x 360)
        assert abs(b["Re_mean"] - g["Re_mean"]) <= 0.005 * g["Re_star"]
        assert abs(b["U_max"] - g["U_cl"]) < 1e-12
        assert abs(b["Umax_over_Umean"] - g["Umax_over_Umean"]) <= 0.005
        assert abs(b["Cf"] - g["Cf"]) <= 0.005e-3
        assert abs(b["dean_Cf"] - g["dean_Cf"]) <= 0.005e-3
        # the paper truncates 18.187 to 18.18
        assert 0.0 <= b["pope_Umax_over_utau"] - g["pope_U_max"] < 0.01
