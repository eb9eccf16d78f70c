"""Oracle for the projection step -- TEST INFRASTRUCTURE ONLY.

Plain, slow FP64 CPU implementation of the simplified-TPLS projection step
(arXiv 1511.07800, Sec. 2-3) used to check the CUDA path.  Only the tests,
the smoke check and the CPU-baseline leg of the benchmark may import this
package; the product path never does.  It shares no code with the CUDA
library: the C source `stp_oracle.c` is compiled on its own into
`liboracle.so` and driven through ctypes here.

Modules:
  this file   -- ctypes wrapper of the C oracle (step and its building blocks)
  srj.py      -- SRJ relaxation schedule (Sec. 3.4) and the eigenvalue bounds
                 it is built from (point and z-line Jacobi)
  os_eig.py   -- Orr-Sommerfeld eigenvalue solver (Sec. 4.1)
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")


def build(force=False):
    """Compile the C oracle (gcc, FP64, no FMA contraction, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", _SRC, "-o", _LIB + ".tmp", "-lm"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("nu", ctypes.c_double), ("dt", ctypes.c_double),
        ("forcing", ctypes.c_int), ("fx", ctypes.c_double), ("ubulk", ctypes.c_double),
        ("les", ctypes.c_int), ("cs", ctypes.c_double), ("vd_a", ctypes.c_double),
        ("re_tau", ctypes.c_double), ("stretch", ctypes.c_double),
        ("cn_sweeps", ctypes.c_int), ("srj_m", ctypes.c_int),
        ("srj_omega", ctypes.POINTER(ctypes.c_double)),
        ("ptol", ctypes.c_double), ("pmaxit", ctypes.c_int), ("zline", ctypes.c_int),
        ("cn_zline", ctypes.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(Params)
        L.orc_create.restype = ctypes.c_void_p
        L.orc_create.argtypes = [pp]
        L.orc_destroy.argtypes = [ctypes.c_void_p]
        L.orc_set_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp]
        L.orc_get_fields.argtypes = [ctypes.c_void_p, dp, dp, dp, dp, dp]
        L.orc_step.argtypes = [ctypes.c_void_p, ctypes.c_int, dp]
        L.orc_step.restype = ctypes.c_int
        L.orc_zfaces.argtypes = [pp, dp]
        for name in ("orc_explicit", "orc_cross_viscous", "orc_diffusion"):
            getattr(L, name).argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_advection.argtypes = [pp, dp, dp, dp, dp, dp, dp]
        L.orc_viscosity.argtypes = [pp, dp, dp, dp, dp]
        L.orc_diffusion_diag.argtypes = [pp, dp, dp, dp, dp]
        L.orc_cn_solve.argtypes = [pp, dp, dp, dp, dp, dp, dp, dp]
        L.orc_divergence.argtypes = [pp, dp, dp, dp, dp]
        L.orc_laplacian.argtypes = [pp, dp, dp]
        L.orc_srj_sweep.argtypes = [pp, dp, dp, ctypes.c_double, dp]
        L.orc_line_sweep.argtypes = [pp, dp, dp, ctypes.c_double, dp]
        L.orc_poisson.argtypes = [pp, dp, dp, ctypes.c_double, ctypes.c_int, dp]
        L.orc_poisson.restype = ctypes.c_int
        L.orc_correct.argtypes = [pp, dp, dp, dp, dp]
        L.orc_set_threads.argtypes = [ctypes.c_int]
        L.orc_get_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Oracle:
    """One channel on the CPU.  `cfg` is a dict with the keys of `Params`
    (omega: the SRJ schedule as a float64 array)."""

    KEYS = ("nx", "ny", "nz", "Lx", "Ly", "Lz", "nu", "dt", "forcing", "fx", "ubulk", "les", "cs",
            "vd_a", "re_tau", "stretch", "cn_sweeps", "ptol", "pmaxit", "zline", "cn_zline")

    def __init__(self, cfg):
        self.cfg = dict(cfg)
        self.omega = np.ascontiguousarray(np.asarray(cfg.get("omega", [1.0]), dtype=np.float64))
        self.P = Params()
        for k in self.KEYS:
            setattr(self.P, k, type(getattr(self.P, k))(cfg.get(k, 0)))
        self.P.srj_m = len(self.omega)
        self.P.srj_omega = _ptr(self.omega)
        self.nx, self.ny, self.nz = cfg["nx"], cfg["ny"], cfg["nz"]
        self.shape_c = (self.nz, self.ny, self.nx)
        self.shape_w = (self.nz + 1, self.ny, self.nx)
        self._h = None

    # -- building blocks ----------------------------------------------------
    def zfaces(self):
        zf = np.zeros(self.nz + 1)
        lib().orc_zfaces(ctypes.byref(self.P), _ptr(zf))
        return zf

    def _c(self):
        return np.zeros(self.shape_c)

    def _w(self):
        return np.zeros(self.shape_w)

    def viscosity(self, u, v, w):
        nu = self._c()
        lib().orc_viscosity(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(nu))
        return nu

    def explicit(self, u, v, w, nu):
        a, b, c = self._c(), self._c(), self._w()
        lib().orc_explicit(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(nu), _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def advection(self, u, v, w):
        a, b, c = self._c(), self._c(), self._w()
        lib().orc_advection(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def cross_viscous(self, u, v, w, nu):
        a, b, c = self._c(), self._c(), self._w()
        lib().orc_cross_viscous(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(nu),
                                _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def diffusion(self, u, v, w, nu):
        a, b, c = self._c(), self._c(), self._w()
        lib().orc_diffusion(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(nu), _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def diffusion_diag(self, nu):
        a, b, c = self._c(), self._c(), self._w()
        lib().orc_diffusion_diag(ctypes.byref(self.P), _ptr(nu), _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def cn_solve(self, nu, ru, rv, rw):
        a, b, c = self._c(), self._c(), self._w()
        ru, rv, rw = (np.ascontiguousarray(x, dtype=np.float64).copy() for x in (ru, rv, rw))
        lib().orc_cn_solve(ctypes.byref(self.P), _ptr(nu), _ptr(ru), _ptr(rv), _ptr(rw), _ptr(a), _ptr(b), _ptr(c))
        return a, b, c

    def divergence(self, u, v, w):
        d = self._c()
        lib().orc_divergence(ctypes.byref(self.P), _ptr(u), _ptr(v), _ptr(w), _ptr(d))
        return d

    def laplacian(self, p):
        out = self._c()
        lib().orc_laplacian(ctypes.byref(self.P), _ptr(np.ascontiguousarray(p)), _ptr(out))
        return out

    def srj_sweep(self, p, b, omega):
        out = self._c()
        lib().orc_srj_sweep(ctypes.byref(self.P), _ptr(p), _ptr(b), float(omega), _ptr(out))
        return out

    def line_sweep(self, p, b, omega):
        """One z-line Jacobi-SOR sweep (each z column solved exactly)."""
        out = self._c()
        lib().orc_line_sweep(ctypes.byref(self.P), _ptr(p), _ptr(b), float(omega), _ptr(out))
        return out

    def poisson(self, b, p0=None, tol=1e-8, maxit=100000):
        """SRJ solve of L p = b.  Returns (p, sweeps, relative residual, converged)."""
        p = np.zeros(self.shape_c) if p0 is None else np.array(p0, dtype=np.float64, order="C")
        rel = ctypes.c_double(0.0)
        b = np.ascontiguousarray(b, dtype=np.float64)
        it = lib().orc_poisson(ctypes.byref(self.P), _ptr(p), _ptr(b), float(tol), int(maxit), ctypes.byref(rel))
        conv = it >= 0
        return p, (it if conv else -1 - it), rel.value, conv

    def correct(self, p, u, v, w):
        u, v, w = (np.array(x, dtype=np.float64, order="C") for x in (u, v, w))
        lib().orc_correct(ctypes.byref(self.P), _ptr(np.ascontiguousarray(p)), _ptr(u), _ptr(v), _ptr(w))
        return u, v, w

    # -- time stepping --------------------------------------------------------
    def set_fields(self, u, v, w, p=None):
        if self._h is None:
            self._h = lib().orc_create(ctypes.byref(self.P))
        arr = [np.ascontiguousarray(x, dtype=np.float64) for x in (u, v, w)]
        pa = None if p is None else np.ascontiguousarray(p, dtype=np.float64)
        lib().orc_set_fields(self._h, _ptr(arr[0]), _ptr(arr[1]), _ptr(arr[2]), _ptr(pa))

    def get_fields(self):
        u, v, p, nu = self._c(), self._c(), self._c(), self._c()
        w = self._w()
        lib().orc_get_fields(self._h, _ptr(u), _ptr(v), _ptr(w), _ptr(p), _ptr(nu))
        return dict(u=u, v=v, w=w, p=p, nu=nu)

    def step(self, n=1):
        """Advance n steps.  Returns the stats of the last step:
        (sweeps, rel residual, max|div u|, bulk u, max|u|, implied -dp/dx), and
        whether every pressure solve converged."""
        st = np.zeros(6)
        rc = lib().orc_step(self._h, int(n), _ptr(st))
        return dict(sweeps=int(st[0]), rel_res=st[1], max_div=st[2], ubulk=st[3], umax=st[4],
                    dpdx=st[5], converged=(rc == 0))

    def __del__(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None


def set_threads(n):
    lib().orc_set_threads(int(n))


def get_threads():
    return lib().orc_get_threads()
