"""LES statistics (Sec. 6) -- TEST INFRASTRUCTURE ONLY (part of the oracle).

Plain numpy definitions of what the library's statistics kernels and its
bulk post-processing compute, written from the paper's definitions:
* the space average over x and y of a quantity at each level (the time
  average is the mean over the accumulated samples);
* the velocities at the cell centres: the mean of the two faces of each
  component on the MAC grid;
* the two-point correlation R(d) = <q(x + d) q(x)> - <q>^2 along x at one
  level (y offset 0);
* the bulk velocity U_mean = (1/Lz) int <u> dz, the centreline (largest)
  mean velocity, the friction velocity from the wall shear of the mean
  profile, C_f = 2 u*^2 / U_mean^2, and the two literature correlations the
  paper compares with: U_max/u* = (1/0.4) ln Re_* + 3.47 and
  C_f = 0.073 Re_mean^(-1/4).
"""
import numpy as np


def centres(u, v, w):
    """Cell-centre values of the three components (periodic x, y)."""
    uc = 0.5 * (u + np.roll(u, -1, axis=2))
    vc = 0.5 * (v + np.roll(v, -1, axis=1))
    wc = 0.5 * (w[:-1] + w[1:])
    return uc, vc, wc


def plane_moments(u, v, w):
    """[9][nz]: plane means of uc, vc, wc, uc^2, vc^2, wc^2, uc vc, uc wc, vc wc."""
    uc, vc, wc = centres(u, v, w)
    qs = [uc, vc, wc, uc * uc, vc * vc, wc * wc, uc * vc, uc * wc, vc * wc]
    return np.array([q.mean(axis=(1, 2)) for q in qs])


def corr_x(u, v, w, kc):
    """[3][nx]: <q(x + d dx) q(x)> over the plane at level kc, for q = u, v (on
    their faces) and wc, before the mean is subtracted."""
    wc = 0.5 * (w[:-1] + w[1:])
    out = []
    for q in (u[kc], v[kc], wc[kc]):
        nx = q.shape[1]
        out.append(np.array([(np.roll(q, -d, axis=1) * q).mean() for d in range(nx)]))
    return np.array(out)


def bulk(umean, zf, nu):
    """Bulk quantities of a mean profile <u>(z) at the cell centres."""
    dz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    Lz = zf[-1] - zf[0]
    U_mean = float((umean * dz).sum() / Lz)
    U_max = float(umean.max())
    # wall shear: the no-slip wall lies half a cell below the first centre
    tau = 0.5 * nu * (umean[0] / (zc[0] - zf[0]) + umean[-1] / (zf[-1] - zc[-1]))
    u_tau = float(np.sqrt(max(tau, 0.0)))
    re_tau = u_tau * Lz / nu
    re_mean = U_mean * Lz / nu
    return dict(U_mean=U_mean, U_max=U_max, u_tau=u_tau, Re_tau=re_tau, Re_mean=re_mean,
                Cf=2 * u_tau ** 2 / U_mean ** 2, Umax_over_utau=U_max / u_tau,
                Umax_over_Umean=U_max / U_mean,
                pope_Umax_over_utau=np.log(re_tau) / 0.4 + 3.47, dean_Cf=0.073 * re_mean ** -0.25)
