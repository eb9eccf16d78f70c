"""The C-ABI library loads and exports what include/stp.h declares; its
host-only parts (configuration checks, SRJ schedule) work without a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "stp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stp_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(stp_lib):
    names = declared()
    assert len(names) >= 10
    lib = stp_lib.lib()
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(stp_lib.EXPORTS)


def test_config_struct_layout(stp_lib):
    """The ctypes mirror has the size the library's defaults fill."""
    c = stp_lib.Config()
    stp_lib.lib().stp_config_defaults(ctypes.byref(c))
    assert c.nx == 32 and c.ptol == 1e-8 and c.cs == 0.1 and c.vd_a == 25.0 and c.inner_tol == 1e-3
    assert c.stream is None and c.srj_m == 0


@pytest.mark.parametrize("bad", [dict(nx=2), dict(nz=1), dict(dt=0.0), dict(precision=7), dict(Lz=-1.0),
                                 dict(srj_m=6), dict(cn_zline=1, nx=4, ny=70000, nz=2)])
def test_init_rejects_bad_config(stp_lib, bad):
    cfg = inputs.preset("laminar_startup")
    prec = bad.pop("precision", 0)
    cfg.update(bad)
    c, _ = stp_lib.make_config(cfg)
    c.precision = prec
    h = ctypes.c_void_p()
    rc = stp_lib.lib().stp_init(ctypes.byref(c), ctypes.byref(h))
    assert rc == stp_lib.STP_EINVAL and not h.value
    assert len(stp_lib.lib().stp_last_error(None)) > 0


@pytest.mark.parametrize("name,stretch", [("laminar_startup", 0.0), ("os_instability", 0.0), ("les_channel", 2.0)])
def test_schedule_matches_oracle(stp_lib, orc, name, stretch):
    """The library's SRJ schedule (Sturm bisection in C++) and the oracle's
    (scipy eigen-solves in Python) agree."""
    from oracle import srj
    cfg = inputs.preset(name)
    om, mn, mx = stp_lib.srj_schedule(cfg)
    om2, mn2, mx2 = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"], stretch)
    assert abs(mn - mn2) < 1e-9 * mn2 and abs(mx - mx2) < 1e-12
    assert len(om) == len(om2)
    assert np.allclose(om, om2, rtol=1e-8)


@pytest.mark.parametrize("name,stretch", [("os_instability", 0.0), ("les_channel", 2.0)])
def test_line_schedule_matches_oracle(stp_lib, orc, name, stretch):
    """z-line SRJ: the library's bounds (closed-form extremes of
    (tau + lam)/(tau + dxy), Sturm bisection for tau) equal the oracle's
    enumeration of every eigenvalue pair, and the schedules agree."""
    from oracle import srj
    cfg = dict(inputs.preset(name), zline=1)
    om, mn, mx = stp_lib.srj_schedule(cfg)
    om2, mn2, mx2 = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"], stretch,
                                     line=True)
    assert abs(mn - mn2) < 1e-9 * mn2 and abs(mx - mx2) < 1e-12
    assert len(om) == len(om2)
    assert np.allclose(om, om2, rtol=1e-8)
    # on the wall-stretched grid the line spectrum is far better conditioned
    if stretch > 0:
        _, pmn, pmx = stp_lib.srj_schedule(inputs.preset(name))
        assert (mx / mn) * 10 < pmx / pmn
