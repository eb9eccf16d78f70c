"""Batched channels: one graph launch advances several channels of
different sizes and configurations; each ends exactly where it ends when
stepped on its own."""
import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

from .test_gpu_parity import case, schedule, turbulent_like

pytestmark = pytest.mark.gpu


def _channels():
    return [
        (case(nx=32, ny=16, nz=32, nu=1 / 500.0), "fp64"),
        (case(nx=48, ny=24, nz=32, stretch=2.0, les=1, forcing=1, nu=1 / 500.0), "fp32"),
        (case(nx=64, ny=32, nz=48, nu=1 / 800.0, cn_sweeps=3), "fp32"),
        (case(nx=40, ny=19, nz=14, nu=1 / 300.0), "fp64"),
    ]


def test_batch_matches_individual_steps(stp_lib):
    specs = _channels()
    ref = []
    for i, (cfg, prec) in enumerate(specs):
        with stp_lib.Channel(cfg, precision=prec, omega=schedule(cfg, 16)) as ch:
            ch.set_fields(*turbulent_like(cfg, 30 + i))
            ch.step(5)
            ref.append(ch.get_fields())
    chans = []
    for i, (cfg, prec) in enumerate(specs):
        ch = stp_lib.Channel(cfg, precision=prec, omega=schedule(cfg, 16))
        ch.set_fields(*turbulent_like(cfg, 30 + i))
        chans.append(ch)
    b = stp_lib.Batch(chans)
    st = b.step(2)
    st = b.step(3)
    assert st["converged"] and st["steps"] == 3
    for i, ch in enumerate(chans):
        got = ch.get_fields()
        assert st["channels"][i]["step"] == 5
        for k in ("u", "v", "w", "p"):
            assert np.array_equal(got[k], ref[i][k]), (i, k)
    b.close()
    for ch in chans:
        ch.close()


def test_batch_uneven_instability_channels(stp_lib):
    """Instances drawn like the uneven-channel workload (here 8 instances of
    sizes from {32, 48, 64}^3): all solves converge; the OS perturbation
    stays small and the bulk flow stays laminar."""
    inst = inputs.batched_instances(count=8, seed=2, sizes=(32, 48, 64))
    chans = []
    for cfg, f in inst:
        ch = stp_lib.Channel(cfg, precision="fp32")
        ch.set_fields(*f)
        chans.append(ch)
    b = stp_lib.Batch(chans)
    st = b.step(20)
    assert st["converged"] and st["sweeps"] > 0
    for c in st["channels"]:
        assert 0.6 < c["ubulk"] < 0.7 and c["umax"] < 1.01
    b.close()
    for ch in chans:
        ch.close()


@pytest.mark.parametrize("env", [{"STP_SWEEP_VARIANT": "0"}, {"STP_SWEEP_VARIANT": "7"},
                                 {"STP_SWEEP_VARIANT": "5", "STP_BATCH_GROUP_CELLS": "60000"},
                                 {"STP_BATCH_GROUP_CHAIN": "1"}])
def test_grouped_solves_match_own_solves(stp_lib, monkeypatch, env):
    """Lock-step groups (one launch per solve kernel over all channels of a
    group), with a forced sweep tile, split into parts, or chained, leave
    every channel bitwise where its own solve leaves it.  The channels share
    M = 32 but differ in size, stretching and LES, so their solves stop after
    different numbers of cycles and passes."""
    specs = [case(nx=32, ny=16, nz=32, nu=1 / 500.0),
             case(nx=48, ny=24, nz=32, stretch=2.0, les=1, forcing=1, nu=1 / 500.0),
             case(nx=64, ny=32, nz=48, nu=1 / 800.0, cn_sweeps=3),
             case(nx=32, ny=32, nz=16, nu=1 / 300.0)]
    res = []
    monkeypatch.setenv("STP_BATCH_GROUP_MAX_CHANNEL", "-1")
    for groups in ("0", "1"):
        monkeypatch.setenv("STP_BATCH_GROUPS", groups)
        for k, v in env.items():
            monkeypatch.setenv(k, v)
        chans = []
        for i, cfg in enumerate(specs):
            ch = stp_lib.Channel(cfg, precision="fp32", omega=schedule(cfg, 32))
            ch.set_fields(*turbulent_like(cfg, 50 + i))
            chans.append(ch)
        b = stp_lib.Batch(chans)
        st = b.step(4)
        assert st["converged"] and st["kernels"] > 0
        grp = b.groups()
        if groups == "1":
            assert sum(g["channels"] for g in grp) >= 2
            assert all(g["M"] == 32 for g in grp)
        else:
            assert grp == []
        res.append(([ch.get_fields() for ch in chans], [c["sweeps"] for c in st["channels"]]))
        b.close()
        for ch in chans:
            ch.close()
    (fa, sa), (fb, sb) = res
    assert sa == sb
    for i in range(len(specs)):
        for k in ("u", "v", "w", "p"):
            assert np.array_equal(fa[i][k], fb[i][k]), (env, i, k)
