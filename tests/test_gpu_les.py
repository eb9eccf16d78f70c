"""The paper's LES workload (Sec. 6) on the GPU: its turbulent-like start,
whole steps against the oracle, and the statistics kernels (plane moments,
two-point correlations) against the oracle's plain definitions."""
import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs, les

from .conftest import rel_err
from .test_gpu_parity import schedule

pytestmark = pytest.mark.gpu


def small_paper_cfg(**over):
    return inputs.preset("les_paper", nx=48, ny=28, nz=24, **over)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-6)])
def test_statistics_match_oracle(stp_lib, orc, precision, tol):
    """Moments per level and streamwise correlations accumulated over two
    states (before and after two steps) equal the oracle's averages of the
    same two states."""
    from oracle import les_stats
    cfg = small_paper_cfg(cn_sweeps=4, ptol=1e-8)
    f0 = inputs.paper_les_initial(cfg, 4)
    kc = 7
    with stp_lib.Channel(cfg, precision=precision, omega=schedule(cfg, 32)) as ch:
        ch.set_fields(*f0)
        ch.stats_reset(kc)
        states = []
        for _ in range(2):
            ch.stats_accumulate()
            fg = ch.get_fields()
            states.append((fg["u"], fg["v"], fg["w"]))
            ch.step(2)
        mom, cor, n, k = ch.stats_read()
    assert n == 2 and k == kc
    mo = np.mean([les_stats.plane_moments(*s) for s in states], axis=0)
    co = np.mean([les_stats.corr_x(*s, kc) for s in states], axis=0) - mo[:3, kc][:, None] ** 2
    scale = np.abs(mo).max(axis=1, keepdims=True)
    assert np.abs(mom - mo).max() < tol * max(1.0, np.abs(mo).max()), np.abs(mom - mo).max()
    assert np.all(np.abs(mom - mo) <= tol * np.maximum(scale, 1.0))
    assert np.abs(cor - co).max() < tol * np.abs(mo[3:6]).max()


def test_paper_les_steps_match_oracle(stp_lib, orc):
    """Whole LES steps of the paper's workload (its units, its random
    Fourier-curl start, Smagorinsky with van Driest) with the solves held to
    two cycles: every field agrees with the oracle to 1e-10 (FP64)."""
    cfg = small_paper_cfg(cn_sweeps=6, ptol=0.0, pmaxit=2 * 16)
    om = schedule(cfg, 16)
    f0 = inputs.paper_les_initial(cfg, 5)
    o = orc.Oracle(dict(cfg, omega=om))
    o.set_fields(*f0)
    so = o.step(3)
    fo = o.get_fields()
    with stp_lib.Channel(cfg, omega=om) as ch:
        ch.set_fields(*f0)
        sg = ch.step(3)
        fg = ch.get_fields()
    assert sg["sweeps"] == so["sweeps"] == 32
    for key in ("u", "v", "w", "p", "nu"):
        e = rel_err(fg[key], fo[key]) if key != "p" else rel_err(fg[key] - fg[key].mean(), fo[key] - fo[key].mean())
        assert e < 1e-10, (key, e)


def test_paper_les_short_run(stp_lib, orc):
    """Twenty FP32 steps of the paper's workload from its start: every solve
    converges, the velocity stays divergence-free to the solver tolerance,
    and the bulk post-processing of the accumulated mean profile gives
    finite, positive values."""
    cfg = small_paper_cfg()
    f0 = inputs.paper_les_initial(cfg, 6)
    o = orc.Oracle(dict(cfg, omega=[1.0]))
    with stp_lib.Channel(cfg, precision="fp32") as ch:
        ch.set_fields(*f0)
        ch.stats_reset()
        for _ in range(20):
            st = ch.step(1)
            assert st["converged"]
            ch.stats_accumulate()
        fg = ch.get_fields()
        mom, cor, n, kc = ch.stats_read()
    div = o.divergence(fg["u"], fg["v"], fg["w"])
    assert np.abs(div).max() < 1e-3 * np.abs(fg["u"]).max() / (cfg["Lx"] / cfg["nx"])
    b = les.bulk(cfg, mom[0])
    assert n == 20 and all(np.isfinite(list(b.values())))
    assert b["U_mean"] > 0 and b["u_tau"] > 0 and b["Cf"] > 0
