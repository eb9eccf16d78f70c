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
    # the buffer keeps the handle's precision: FP32 fields packed two to a
    # double (p stays FP64), refused by a handle of the other precision
    other = "fp64" if precision == "fp32" else "fp32"
    with stp_lib.Channel(cfg, precision=other, omega=om) as d:
        if precision == "fp32":
            nc = cfg["nx"] * cfg["ny"] * cfg["nz"]
            assert len(state) < 0.6 * d.state_size() and len(state) >= 5.5 * nc
        with pytest.raises(stp_lib.StpError) as e:
            d.set_state(state)
        assert e.value.code == stp_lib.STP_EINVAL


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


def _equal(a, b):
    return np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_diverged_step_keeps_last_good_fields(stp_lib, precision):
    """A run whose time step is far beyond the CFL limit blows up: the step
    that produces NaN/Inf returns STP_EDIVERGED and is undone, so the
    fields, the pressure and the step counter are those of the last good
    step; the handle then takes new fields and steps normally."""
    cfg = case(dt=0.5, nu=1e-4, forcing=0, fx=0.0)
    om = schedule(cfg, 16)
    u, v, w = turbulent_like(cfg, 5)
    with stp_lib.Channel(cfg, precision=precision, omega=om) as ch:
        ch.set_fields(u * 20.0, v * 20.0, w * 20.0)
        last, state, code = None, None, None
        for n in range(400):
            last = ch.get_fields()
            state = ch.get_state()
            try:
                ch.step(1)
            except stp_lib.StpError as e:
                code = e.code
                break
        assert code == stp_lib.STP_EDIVERGED, "the run did not blow up"
        assert n > 1  # a mid-run failure: the Adams-Bashforth history is in use
        got = ch.get_fields()
        for k in ("u", "v", "w", "p"):
            assert _equal(got[k], last[k]), k
        assert _equal(ch.get_state(), state)
        ch.set_fields(u, v, w)
        st = ch.step(2)
        assert st["status"] in (stp_lib.STP_OK, stp_lib.STP_ENOTCONVERGED) and st["step"] == 2


def test_barrier_timeout_is_reported_and_recovered(stp_lib, monkeypatch):
    """The persistent SRJ cycle (STP_PERSISTENT=1) waits at a grid barrier
    between sweeps, each wait bounded by STP_BARRIER_WAIT clock cycles.  A
    limit of one cycle makes the waits run out: the step returns
    STP_ETIMEOUT, leaves the fields of the last good step, and the barrier
    state is cleared on the next call, whose steps then equal those of a
    fresh handle bit for bit."""
    cfg = case(nx=64, ny=20, nz=24, stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=4)
    om = schedule(cfg, 32)
    monkeypatch.setenv("STP_PERSISTENT", "1")
    f0 = turbulent_like(cfg, 12)
    with stp_lib.Channel(cfg, precision="fp32", omega=om) as ref:
        ref.set_fields(*f0)
        ref.step(3)
        want = ref.get_fields()
    with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
        ch.set_fields(*f0)
        before = ch.get_fields()
        monkeypatch.setenv("STP_BARRIER_WAIT", "1")
        with pytest.raises(stp_lib.StpError) as e:
            ch.step(1)
        assert e.value.code == stp_lib.STP_ETIMEOUT
        after = ch.get_fields()
        for k in ("u", "v", "w", "p"):
            assert np.array_equal(after[k], before[k]), k
        monkeypatch.delenv("STP_BARRIER_WAIT")
        st = ch.step(3)
        assert st["converged"] and st["step"] == 3
        got = ch.get_fields()
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(got[k], want[k]), k


def test_poisson_rhs_with_mean_is_rejected(stp_lib):
    """L p = b has a solution only if the volume integral of b vanishes
    (Neumann walls, periodic x and y): a right-hand side with a mean is
    refused with STP_EINVAL before any sweep; a mean-free one solves and
    the solution comes back with zero volume-weighted mean."""
    cfg = case(nx=40, ny=12, nz=16, stretch=2.0)
    rng = np.random.default_rng(9)
    b = rng.standard_normal((16, 12, 40))
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    vol = dz * np.ones_like(b)
    b -= np.sum(b * dz) / np.sum(vol)
    with stp_lib.Channel(cfg, omega=schedule(cfg, 16)) as ch:
        with pytest.raises(stp_lib.StpError) as e:
            ch.poisson_solve(b + 1e-3, np.zeros_like(b), tol=1e-8)
        assert e.value.code == stp_lib.STP_EINVAL
        p = rng.standard_normal(b.shape) + 5.0
        st = ch.poisson_solve(b, p, tol=1e-8)
        assert st["converged"]
        assert abs(np.sum(p * dz)) / np.sum(np.abs(p) * vol) < 1e-13
