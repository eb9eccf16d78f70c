"""Checkpoint/resume and failure detection of the step through the C ABI.
Failures are made on the host (a sweep cap that cannot be met, NaN in the
initial fields, a velocity that breaks the CFL rule); nothing faults the GPU."""
import math

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

from .test_gpu_parity import case, schedule, turbulent_like

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume_bitwise(stp_lib, precision):
    """N steps, save, restore into a new handle, N more steps == 2N steps."""
    cfg = case(stretch=2.0, les=1, forcing=1, nu=1 / 500.0)
    om = schedule(cfg, 16)
    with stp_lib.Channel(cfg, precision=precision, omega=om) as a:
        a.set_fields(*turbulent_like(cfg, 21))
        a.step(6)
        ref = a.get_fields()
    with stp_lib.Channel(cfg, precision=precision, omega=om) as b:
        b.set_fields(*turbulent_like(cfg, 21))
        b.step(3)
        state = b.get_state()
    with stp_lib.Channel(cfg, precision=precision, omega=om) as c:
        c.set_state(state)
        st = c.step(3)
        assert st["step"] == 6
        got = c.get_fields()
    for k in ("u", "v", "w", "p", "nu"):
        assert np.array_equal(got[k], ref[k]), k


def test_not_converged_is_reported(stp_lib):
    cfg = case(ptol=1e-14, pmaxit=16)
    with stp_lib.Channel(cfg, omega=schedule(cfg, 16)) as ch:
        ch.set_fields(*turbulent_like(cfg, 2))
        st = ch.step(1)
        assert st["status"] == stp_lib.STP_ENOTCONVERGED and not st["converged"] and st["sweeps"] == 16


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nan_is_detected(stp_lib, precision):
    cfg = case()
    u, v, w = turbulent_like(cfg, 3)
    u[3, 4, 5] = float("nan")
    with stp_lib.Channel(cfg, precision=precision, omega=schedule(cfg, 16)) as ch:
        ch.set_fields(u, v, w)
        with pytest.raises(stp_lib.StpError) as e:
            ch.step(1)
        assert e.value.code == stp_lib.STP_EDIVERGED


def test_cfl_violation_is_reported(stp_lib):
    """Eq. cfl_cond: U_max dt <= 0.1 dx."""
    cfg = case(cfl_check=1, dt=0.05)
    u, v, w = turbulent_like(cfg, 4)
    with stp_lib.Channel(cfg, omega=schedule(cfg, 16)) as ch:
        ch.set_fields(u * 3.0, v, w)
        st = ch.step(1)
        assert st["status"] == stp_lib.STP_ECFL
        assert st["umax"] * cfg["dt"] > 0.1 * cfg["Lx"] / cfg["nx"]
