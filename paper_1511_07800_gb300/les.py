"""Bulk quantities of the LES (Sec. 6) from the mean profile the library's
statistics kernels accumulate (Channel.stats_read): host post-processing of
a few numbers, not part of the time step.

  U_mean   (1/Lz) int <u> dz                bulk velocity
  U_max    largest <u>, at the centreline
  u_tau    sqrt(nu d<u>/dz) at the walls     (the no-slip wall half a cell
                                              below the first centre; mean of
                                              both walls)
  C_f      2 u_tau^2 / U_mean^2              skin friction
and the literature correlations the paper compares with:
  U_max/u_tau = (1/0.4) ln Re_* + 3.47,  C_f = 0.073 Re_mean^(-1/4),
  Re_* = u_tau Lz / nu, Re_mean = U_mean Lz / nu.
"""
import math

import numpy as np

from . import inputs


def bulk(cfg, umean):
    zf = inputs.zfaces(cfg)
    nu = cfg["nu"]
    Lz = cfg["Lz"]
    dz = np.diff(zf)
    zc = 0.5 * (zf[1:] + zf[:-1])
    U_mean = float(np.dot(umean, dz) / Lz)
    U_max = float(np.max(umean))
    wall = 0.5 * nu * (umean[0] / (zc[0] - zf[0]) + umean[-1] / (zf[-1] - zc[-1]))
    u_tau = math.sqrt(max(wall, 0.0))
    re_tau, re_mean = u_tau * Lz / nu, U_mean * Lz / nu
    return dict(U_mean=U_mean, U_max=U_max, u_tau=u_tau, Re_tau=re_tau, Re_mean=re_mean,
                Cf=2 * u_tau * u_tau / (U_mean * U_mean), Umax_over_utau=U_max / u_tau,
                Umax_over_Umean=U_max / U_mean, pope_Umax_over_utau=math.log(re_tau) / 0.4 + 3.47,
                dean_Cf=0.073 * re_mean ** -0.25)
