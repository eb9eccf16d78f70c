"""Python binding of the C ABI in include/stp.h (argument marshalling only).

Every step of the method runs in the CUDA library libstp.so; this module
converts dicts and arrays to the C structures and pointers.  It refuses to
work when the library is missing: there is no CPU path.

Arrays: numpy float64 arrays are passed as host memory (STP_HOST); objects
with `data_ptr()` and `is_cuda` (torch CUDA float64 tensors) as device memory
(STP_DEVICE).  Layouts are those of the header: u, v, p [nz][ny][nx],
w [nz+1][ny][nx], x fastest.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libstp.so")

STP_OK = 0
STP_EINVAL = -1
STP_ENOMEM = -2
STP_ECUDA = -3
STP_ENOTCONVERGED = -4
STP_EDIVERGED = -5
STP_ECFL = -6
STP_ETIMEOUT = -7
STP_HOST, STP_DEVICE = 0, 1
STP_FP64, STP_FP32_REFINE = 0, 1
TERMS = {"viscosity": 1, "explicit": 2, "diffusion": 3, "divergence": 4, "laplacian": 5}


class StpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("stp error %d: %s" % (code, msg))
        self.code = code


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("Lx", ctypes.c_double), ("Ly", ctypes.c_double), ("Lz", ctypes.c_double),
        ("nu", ctypes.c_double), ("dt", ctypes.c_double),
        ("forcing", ctypes.c_int), ("fx", ctypes.c_double), ("ubulk", ctypes.c_double),
        ("les", ctypes.c_int), ("cs", ctypes.c_double), ("vd_a", ctypes.c_double),
        ("re_tau", ctypes.c_double), ("stretch", ctypes.c_double),
        ("precision", ctypes.c_int), ("ptol", ctypes.c_double), ("pmaxit", ctypes.c_int),
        ("cn_sweeps", ctypes.c_int), ("srj_m", ctypes.c_int),
        ("srj_omega", ctypes.POINTER(ctypes.c_double)),
        ("inner_tol", ctypes.c_double), ("cfl_check", ctypes.c_int),
        ("device", ctypes.c_int), ("stream", ctypes.c_void_p), ("zline", ctypes.c_int),
        ("cn_zline", ctypes.c_int),
    ]


class StepStats(ctypes.Structure):
    _fields_ = [("poisson_sweeps", ctypes.c_int), ("refine_passes", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("ubulk", ctypes.c_double), ("umax", ctypes.c_double), ("dpdx", ctypes.c_double),
                ("step", ctypes.c_longlong), ("launches", ctypes.c_longlong),
                ("solve_sweeps", ctypes.c_longlong), ("solve_ms", ctypes.c_double)]


class BatchStats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("cells", ctypes.c_longlong), ("sweeps", ctypes.c_longlong),
                ("converged", ctypes.c_int), ("gpu_ms", ctypes.c_double), ("kernels", ctypes.c_longlong)]


class BatchGroup(ctypes.Structure):
    _fields_ = [("channels", ctypes.c_int), ("M", ctypes.c_int), ("variant", ctypes.c_int),
                ("cells", ctypes.c_longlong), ("sweep_us", ctypes.c_float)]


class SolveStats(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int), ("refine_passes", ctypes.c_int),
                ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]


EXPORTS = ("stp_config_defaults", "stp_init", "stp_destroy", "stp_last_error", "stp_set_fields",
           "stp_get_fields", "stp_step", "stp_poisson_solve", "stp_eval", "stp_srj_schedule",
           "stp_poisson_residual_noalloc", "stp_unet_param_count", "stp_unet_create", "stp_unet_destroy",
           "stp_unet_last_error", "stp_unet_set_params", "stp_unet_get_params", "stp_unet_forward",
           "stp_unet_gradient", "stp_unet_train_step", "stp_unet_train_pairs", "stp_unet_eval_pairs",
           "stp_set_learned_guess", "stp_set_harvest", "stp_unet_set_output_scale", "stp_state_size",
           "stp_get_state", "stp_set_state", "stp_batch_create", "stp_batch_destroy", "stp_batch_last_error",
           "stp_batch_step", "stp_batch_groups", "stp_sweep_tile", "stp_stats_reset",
           "stp_stats_accumulate", "stp_stats_read", "stp_unet_layer", "stp_set_learned_mode",
           "stp_line_kernel")

_lib = None


def lib():
    """Load libstp.so (built by build.py).  Raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libstp.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    dp = ctypes.POINTER(ctypes.c_double)
    vp = ctypes.c_void_p
    L.stp_config_defaults.argtypes = [ctypes.POINTER(Config)]
    L.stp_config_defaults.restype = None
    L.stp_init.argtypes = [ctypes.POINTER(Config), ctypes.POINTER(vp)]
    L.stp_destroy.argtypes = [vp]
    L.stp_destroy.restype = None
    L.stp_last_error.argtypes = [vp]
    L.stp_last_error.restype = ctypes.c_char_p
    L.stp_set_fields.argtypes = [vp, vp, vp, vp, vp, ctypes.c_int]
    L.stp_get_fields.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int]
    L.stp_step.argtypes = [vp, ctypes.c_int, ctypes.POINTER(StepStats)]
    L.stp_poisson_solve.argtypes = [vp, vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.POINTER(SolveStats)]
    L.stp_eval.argtypes = [vp, ctypes.c_int, vp, vp, vp, ctypes.c_int]
    L.stp_srj_schedule.argtypes = [ctypes.POINTER(Config), ctypes.c_int, dp, ctypes.POINTER(ctypes.c_int),
                                   dp, dp]
    L.stp_poisson_residual_noalloc.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, ctypes.c_double, vp, vp, vp,
                                               ctypes.POINTER(ctypes.c_double), vp]
    L.stp_unet_param_count.restype = ctypes.c_longlong
    L.stp_unet_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.stp_unet_destroy.argtypes = [vp]
    L.stp_unet_destroy.restype = None
    L.stp_unet_last_error.argtypes = [vp]
    L.stp_unet_last_error.restype = ctypes.c_char_p
    L.stp_unet_set_params.argtypes = [vp, vp, ctypes.c_int]
    L.stp_unet_get_params.argtypes = [vp, vp, ctypes.c_int]
    L.stp_unet_forward.argtypes = [vp, vp, vp, ctypes.c_int]
    L.stp_unet_gradient.argtypes = [vp, vp, vp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_float)]
    L.stp_unet_train_step.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
    L.stp_unet_train_pairs.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_float)]
    L.stp_unet_eval_pairs.argtypes = [vp, vp, vp, ctypes.c_int, ctypes.POINTER(ctypes.c_float)]
    L.stp_set_learned_guess.argtypes = [vp, vp]
    L.stp_batch_create.argtypes = [ctypes.POINTER(vp), ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.stp_batch_destroy.argtypes = [vp]
    L.stp_batch_destroy.restype = None
    L.stp_batch_last_error.argtypes = [vp]
    L.stp_batch_last_error.restype = ctypes.c_char_p
    L.stp_batch_step.argtypes = [vp, ctypes.c_int, ctypes.POINTER(BatchStats), ctypes.POINTER(StepStats)]
    L.stp_batch_groups.argtypes = [vp, ctypes.c_int, ctypes.POINTER(BatchGroup)]
    L.stp_sweep_tile.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    L.stp_line_kernel.argtypes = [vp]
    L.stp_stats_reset.argtypes = [vp, ctypes.c_int]
    L.stp_stats_accumulate.argtypes = [vp]
    L.stp_stats_read.argtypes = [vp, dp, dp, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]
    L.stp_state_size.argtypes = [vp]
    L.stp_state_size.restype = ctypes.c_longlong
    L.stp_get_state.argtypes = [vp, vp]
    L.stp_set_state.argtypes = [vp, vp]
    L.stp_unet_set_output_scale.argtypes = [vp, ctypes.c_float]
    L.stp_set_harvest.argtypes = [vp, vp, vp]
    L.stp_unet_layer.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, ctypes.c_int]
    L.stp_set_learned_mode.argtypes = [vp, ctypes.c_int]
    _lib = L
    return L


def make_config(cfg, precision="fp64", device=0, stream=None, omega=None):
    """stp_config from a workload dict (keys as in inputs.preset)."""
    c = Config()
    lib().stp_config_defaults(ctypes.byref(c))
    for k in ("nx", "ny", "nz", "Lx", "Ly", "Lz", "nu", "dt", "forcing", "fx", "ubulk", "les", "cs", "vd_a",
              "re_tau", "stretch", "ptol", "pmaxit", "cn_sweeps", "srj_m", "inner_tol", "cfl_check", "zline",
              "cn_zline"):
        if k in cfg and cfg[k] is not None:
            setattr(c, k, type(getattr(c, k))(cfg[k]))
    c.precision = STP_FP64 if precision in ("fp64", 0) else STP_FP32_REFINE
    c.device = int(device)
    c.stream = stream
    keep = None
    if omega is not None:
        keep = np.ascontiguousarray(omega, dtype=np.float64)
        c.srj_m = len(keep)
        c.srj_omega = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    return c, keep


def srj_schedule(cfg, M=0):
    """(omega, mu_min, mu_max) of the library's Chebyshev SRJ schedule."""
    c, _ = make_config(cfg)
    om = np.zeros(1024)
    m = ctypes.c_int(0)
    mn, mx = ctypes.c_double(0), ctypes.c_double(0)
    rc = lib().stp_srj_schedule(ctypes.byref(c), int(M), om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                ctypes.byref(m), ctypes.byref(mn), ctypes.byref(mx))
    if rc != STP_OK:
        raise StpError(rc, lib().stp_last_error(None).decode())
    return om[:m.value].copy(), mn.value, mx.value


def poisson_residual_noalloc(cfg, p, b, r_out=None, stream=None):
    """||b - L p||_2 for device arrays p, b (torch CUDA float64 tensors)
    through the allocation-free entry point; r_out optionally receives b - Lp."""
    norm = ctypes.c_double(0.0)
    rc = lib().stp_poisson_residual_noalloc(int(cfg["nx"]), int(cfg["ny"]), int(cfg["nz"]), float(cfg["Lx"]),
                                            float(cfg["Ly"]), float(cfg["Lz"]), float(cfg.get("stretch", 0.0)),
                                            ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(b.data_ptr()),
                                            ctypes.c_void_p(r_out.data_ptr()) if r_out is not None else None,
                                            ctypes.byref(norm), stream)
    if rc != STP_OK:
        raise StpError(rc, lib().stp_last_error(None).decode())
    return norm.value


def _addr(a):
    """(pointer, where) for a numpy array or a CUDA tensor."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        if not getattr(a, "is_cuda", False):
            a = a.numpy()
        else:
            return ctypes.c_void_p(a.data_ptr()), STP_DEVICE
    assert a.dtype == np.float64 and a.flags.c_contiguous, "need C-contiguous float64"
    return ctypes.c_void_p(a.ctypes.data), STP_HOST


class Channel:
    """One channel on one GPU (a handle of the C ABI)."""

    def __init__(self, cfg, precision="fp64", device=0, stream=None, omega=None):
        self.cfg = dict(cfg)
        self.nx, self.ny, self.nz = cfg["nx"], cfg["ny"], cfg["nz"]
        c, self._omega = make_config(cfg, precision, device, stream, omega)
        h = ctypes.c_void_p()
        rc = lib().stp_init(ctypes.byref(c), ctypes.byref(h))
        if rc != STP_OK:
            raise StpError(rc, lib().stp_last_error(None).decode())
        self._h = h

    # ------------------------------------------------------------------
    def _check(self, rc, allow=()):
        if rc != STP_OK and rc not in allow:
            raise StpError(rc, lib().stp_last_error(self._h).decode())
        return rc

    def _where(self, *arrays):
        ws = {w for (p, w) in (_addr(a) for a in arrays if a is not None)}
        if len(ws) != 1:
            raise ValueError("mix of host and device arrays")
        return ws.pop()

    def set_fields(self, u, v, w, p=None):
        where = self._where(u, v, w, p)
        ptr = [_addr(a)[0] for a in (u, v, w, p)]
        self._check(lib().stp_set_fields(self._h, ptr[0], ptr[1], ptr[2], ptr[3], where))

    def get_fields(self, out=None):
        """Copy the fields out: into `out` (dict of arrays/tensors) or new numpy arrays."""
        if out is None:
            sc, sw = (self.nz, self.ny, self.nx), (self.nz + 1, self.ny, self.nx)
            out = dict(u=np.zeros(sc), v=np.zeros(sc), w=np.zeros(sw), p=np.zeros(sc), nu=np.zeros(sc))
        where = self._where(*[out[k] for k in ("u", "v", "w", "p", "nu") if out.get(k) is not None])
        ptr = [_addr(out.get(k))[0] for k in ("u", "v", "w", "p", "nu")]
        self._check(lib().stp_get_fields(self._h, *ptr, where))
        return out

    def step(self, n=1):
        st = StepStats()
        rc = self._check(lib().stp_step(self._h, int(n), ctypes.byref(st)), allow=(STP_ENOTCONVERGED, STP_ECFL))
        return dict(sweeps=st.poisson_sweeps, passes=st.refine_passes, converged=bool(st.converged),
                    rel_res=st.rel_residual, ubulk=st.ubulk, umax=st.umax, dpdx=st.dpdx, step=st.step,
                    launches=st.launches, solve_sweeps=st.solve_sweeps, solve_ms=st.solve_ms, status=rc)

    def poisson_solve(self, rhs, p0, tol=1e-8, maxit=0):
        """Solve L p = rhs from p0 (updated in place)."""
        where = self._where(rhs, p0)
        st = SolveStats()
        rc = self._check(lib().stp_poisson_solve(self._h, _addr(rhs)[0], _addr(p0)[0], float(tol), int(maxit), where,
                                                 ctypes.byref(st)), allow=(STP_ENOTCONVERGED,))
        return dict(sweeps=st.sweeps, passes=st.refine_passes, converged=bool(st.converged),
                    rel_res=st.rel_residual, solve_ms=st.solve_ms, status=rc)

    def eval(self, term, out=None):
        """A term of the step on the current fields (see stp_eval)."""
        t = TERMS[term]
        sc, sw = (self.nz, self.ny, self.nx), (self.nz + 1, self.ny, self.nx)
        if out is None:
            if t in (2, 3):
                out = (np.zeros(sc), np.zeros(sc), np.zeros(sw))
            else:
                out = (np.zeros(sc),)
        where = self._where(*out)
        ptr = [_addr(a)[0] for a in out] + [None] * (3 - len(out))
        self._check(lib().stp_eval(self._h, t, ptr[0], ptr[1], ptr[2], where))
        return out if len(out) > 1 else out[0]

    def state_size(self):
        return int(lib().stp_state_size(self._h))

    def get_state(self, out=None):
        """The whole time-stepper state as a float64 host array (checkpoint);
        `out` may be a host float64 tensor (e.g. pinned) of state_size()."""
        if out is None:
            out = np.zeros(self.state_size())
        ptr = out.data_ptr() if hasattr(out, "data_ptr") else out.ctypes.data
        self._check(lib().stp_get_state(self._h, ctypes.c_void_p(ptr)))
        return out

    def set_state(self, buf):
        if hasattr(buf, "data_ptr"):
            self._check(lib().stp_set_state(self._h, ctypes.c_void_p(buf.data_ptr())))
            return
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        self._check(lib().stp_set_state(self._h, ctypes.c_void_p(buf.ctypes.data)))

    def set_learned_guess(self, net):
        """Start every pressure solve from the network's guess (None: off)."""
        self._net = net
        self._check(lib().stp_set_learned_guess(self._h, net._h if net is not None else None))

    def set_learned_mode(self, mode):
        """0: the network's guess once per solve; 1: as a preconditioner at
        every refinement pass (FP32) or SRJ cycle (FP64)."""
        self._check(lib().stp_set_learned_mode(self._h, int(mode)))

    def set_harvest(self, r_out, dp_out):
        """Record (residual, correction) pairs of each solve into two CUDA
        float32 tensors [nz][ny][nx] (None, None: stop)."""
        self._harvest = (r_out, dp_out)
        a = ctypes.c_void_p(r_out.data_ptr()) if r_out is not None else None
        b = ctypes.c_void_p(dp_out.data_ptr()) if dp_out is not None else None
        self._check(lib().stp_set_harvest(self._h, a, b))

    def stats_reset(self, kc=-1):
        """Clear the LES statistics; kc: level of the two-point correlations (-1: nz/2)."""
        self._check(lib().stp_stats_reset(self._h, int(kc)))

    def stats_accumulate(self):
        """Add the current fields to the statistics (asynchronous)."""
        self._check(lib().stp_stats_accumulate(self._h))

    def stats_read(self):
        """(moments [9][nz], correlations [3][nx], samples, kc): means over x, y
        and the samples of uc, vc, wc, uc^2, vc^2, wc^2, uc vc, uc wc, vc wc,
        and R(d) of u, v, wc at level kc."""
        mom = np.zeros((9, self.nz))
        cor = np.zeros((3, self.nx))
        n = ctypes.c_longlong(0)
        kc = ctypes.c_int(0)
        self._check(lib().stp_stats_read(self._h, mom.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                         cor.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(n),
                                         ctypes.byref(kc)))
        return mom, cor, n.value, kc.value

    def sweep_tile(self):
        """(variant, microseconds per sweep) picked by the FP32 sweep autotuner."""
        us = ctypes.c_float()
        v = lib().stp_sweep_tile(self._h, ctypes.byref(us))
        return v, us.value

    def line_kernel(self):
        """z-line sweep kernel: 1 register-chunked (FP32), 0 shared-memory
        lock step, -1 point sweeps."""
        return lib().stp_line_kernel(self._h)

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.stp_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class UNet:
    """The learned-guess network (see stp_unet_* in the header).  Arrays are
    torch CUDA float32 tensors [n][nz][ny][nx]; parameters a flat float32
    vector (numpy for host, tensor for device)."""

    def __init__(self, nmax, nz, ny, nx, stream=None):
        h = ctypes.c_void_p()
        rc = lib().stp_unet_create(int(nmax), int(nz), int(ny), int(nx), stream, ctypes.byref(h))
        if rc != STP_OK:
            raise StpError(rc, "stp_unet_create failed (sizes must be multiples of 8)")
        self._h = h
        self.shape = (nz, ny, nx)
        self.nmax = nmax

    @staticmethod
    def param_count():
        return int(lib().stp_unet_param_count())

    def _check(self, rc):
        if rc != STP_OK:
            raise StpError(rc, lib().stp_unet_last_error(self._h).decode())

    def set_params(self, theta):
        if hasattr(theta, "data_ptr"):
            self._check(lib().stp_unet_set_params(self._h, ctypes.c_void_p(theta.data_ptr()), STP_DEVICE))
        else:
            a = np.ascontiguousarray(theta, dtype=np.float32)
            self._check(lib().stp_unet_set_params(self._h, ctypes.c_void_p(a.ctypes.data), STP_HOST))

    def get_params(self):
        a = np.zeros(self.param_count(), dtype=np.float32)
        self._check(lib().stp_unet_get_params(self._h, ctypes.c_void_p(a.ctypes.data), STP_HOST))
        return a

    def forward(self, x, y):
        self._check(lib().stp_unet_forward(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr()),
                                           int(x.shape[0])))

    def gradient(self, x, t, grad=None):
        loss = ctypes.c_float(0)
        g = ctypes.c_void_p(grad.data_ptr()) if grad is not None else None
        self._check(lib().stp_unet_gradient(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                            int(x.shape[0]), g, ctypes.byref(loss)))
        return loss.value

    def train_step(self, x, t, lr):
        loss = ctypes.c_float(0)
        self._check(lib().stp_unet_train_step(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                              int(x.shape[0]), float(lr), ctypes.byref(loss)))
        return loss.value

    def set_output_scale(self, k):
        self._check(lib().stp_unet_set_output_scale(self._h, float(k)))

    def train_pairs(self, r, dp, lr):
        """One Adam step on (residual, correction) pairs, each scaled by its RMS(r)."""
        loss = ctypes.c_float(0)
        self._check(lib().stp_unet_train_pairs(self._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(dp.data_ptr()),
                                               int(r.shape[0]), float(lr), ctypes.byref(loss)))
        return loss.value

    def eval_pairs(self, r, dp):
        loss = ctypes.c_float(0)
        self._check(lib().stp_unet_eval_pairs(self._h, ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(dp.data_ptr()),
                                              int(r.shape[0]), ctypes.byref(loss)))
        return loss.value

    def layer(self, index, mode, a, b, out):
        """One convolution on its own (stp_unet_layer): mode "forward",
        "data_grad" or "weight_grad"; a, b, out torch CUDA float32 tensors
        (b may be None), channels last."""
        m = {"forward": 0, "data_grad": 1, "weight_grad": 2}[mode]
        bp = ctypes.c_void_p(b.data_ptr()) if b is not None else None
        self._check(lib().stp_unet_layer(self._h, int(index), m, ctypes.c_void_p(a.data_ptr()), bp,
                                         ctypes.c_void_p(out.data_ptr()), int(a.shape[0])))

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.stp_unet_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()


class Batch:
    """Many channels advanced together by one graph launch (stp_batch_*)."""

    def __init__(self, channels, stream=None):
        self.channels = list(channels)
        arr = (ctypes.c_void_p * len(self.channels))(*[c._h.value for c in self.channels])
        h = ctypes.c_void_p()
        rc = lib().stp_batch_create(arr, len(self.channels), stream, ctypes.byref(h))
        if rc != STP_OK:
            raise StpError(rc, lib().stp_last_error(None).decode())
        self._h = h

    def step(self, n=1):
        st = BatchStats()
        per = (StepStats * len(self.channels))()
        rc = lib().stp_batch_step(self._h, int(n), ctypes.byref(st), per)
        if rc not in (STP_OK, STP_ENOTCONVERGED):
            raise StpError(rc, lib().stp_batch_last_error(self._h).decode())
        return dict(steps=st.steps, cells=st.cells, sweeps=st.sweeps, converged=bool(st.converged),
                    gpu_ms=st.gpu_ms, kernels=st.kernels, status=rc,
                    channels=[dict(sweeps=p.poisson_sweeps, converged=bool(p.converged), rel_res=p.rel_residual,
                                   ubulk=p.ubulk, umax=p.umax, step=p.step) for p in per])

    def groups(self):
        """Lock-step groups (known after the first step): channels, M, sweep
        variant, cells and the measured grouped sweep time."""
        n = lib().stp_batch_groups(self._h, 0, None)
        arr = (BatchGroup * max(1, n))()
        lib().stp_batch_groups(self._h, n, arr)
        return [dict(channels=g.channels, M=g.M, variant=g.variant, cells=g.cells, sweep_us=g.sweep_us)
                for g in arr[:n]]

    def close(self):
        if getattr(self, "_h", None) is not None and _lib is not None:
            _lib.stp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()
