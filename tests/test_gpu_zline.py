"""z-line relaxation of the pressure solve on the GPU: each z column solved
exactly per sweep (Thomas), SRJ weights from the line-Jacobi spectrum.
Parity with the oracle's line sweep (a plain Thomas solve per column)."""
import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

from .conftest import gauge, rel_err
from .test_gpu_parity import case, turbulent_like

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


def line_schedule(cfg, M):
    from oracle import srj
    om, _, _ = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"],
                                cfg.get("stretch", 0.0), M, line=True)
    return om


def mean_free_rhs(cfg, seed):
    rng = np.random.default_rng(seed)
    b = rng.standard_normal((cfg["nz"], cfg["ny"], cfg["nx"]))
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    return b - np.sum(b * dz) / np.sum(dz * np.ones_like(b)), rng


@pytest.mark.parametrize("stretch,nx,ny,nz", [(0.0, 48, 20, 18), (2.0, 48, 20, 18), (2.0, 37, 21, 18),
                                              (2.0, 64, 21, 18), (0.0, 96, 8, 30), (2.0, 8, 5, 400)])
def test_line_fixed_sweeps_parity(stp_lib, orc, stretch, nx, ny, nz):
    """The same line schedule applied for the same number of sweeps gives
    the same pressure as the oracle's column-by-column Thomas solves (FP64;
    ragged rows and row blocks; rows of a multiple of 32 cells take the
    vector kernel; 400 levels take the kernel that keeps the columns in
    global memory)."""
    cfg = case(nx=nx, ny=ny, nz=nz, stretch=stretch, zline=1)
    om = line_schedule(cfg, 32)
    cfg["omega"] = om
    b, rng = mean_free_rhs(cfg, 5)
    p0 = rng.standard_normal(b.shape) * 0.1
    o = orc.Oracle(cfg)
    p_o, it_o, rel_o, conv_o = o.poisson(b, p0, tol=0.0, maxit=3 * 32)
    with stp_lib.Channel(cfg, omega=om) as ch:
        p_g = p0.copy()
        st = ch.poisson_solve(b, p_g, tol=0.0, maxit=3 * 32)
    assert st["sweeps"] == it_o == 96 and not st["converged"] and not conv_o
    assert rel_err(p_g, gauge(p_o, cfg)) < TOL64
    # residuals near 1e-12 of ||b|| are FP64 rounding of L p: an absolute floor
    assert abs(st["rel_res"] - rel_o) < 1e-9 * rel_o + 1e-11


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_line_solve_converges_to_tolerance(stp_lib, orc, precision):
    """Tolerance-driven line solves stop at ||b - Lp|| <= 1e-8 ||b||,
    checked with the oracle's operator, and take fewer sweeps than point
    sweeps on the wall-stretched grid."""
    cfg = case(nx=64, ny=24, nz=32, stretch=2.0)
    b, _ = mean_free_rhs(cfg, 7)
    o = orc.Oracle(cfg)
    sweeps = {}
    for zl in (1, 0):
        with stp_lib.Channel(dict(cfg, zline=zl), precision=precision) as ch:
            p = np.zeros_like(b)
            st = ch.poisson_solve(b, p, tol=1e-8)
        r = b - o.laplacian(p)
        rel = np.sqrt(np.sum(r * r) / np.sum(b * b))
        assert st["converged"] and rel <= 1e-8 * 1.0001, (zl, rel)
        sweeps[zl] = st["sweeps"]
    assert sweeps[1] < sweeps[0], sweeps


@pytest.mark.parametrize("stretch,les,forcing", [(0.0, 0, 0), (2.0, 1, 1)])
def test_line_step_parity_fp64(stp_lib, orc, stretch, les, forcing):
    """Whole projection steps with line relaxation and the solves forced to
    two cycles: every field agrees with the oracle to 1e-10."""
    cfg = case(stretch=stretch, les=les, forcing=forcing, ptol=0.0, pmaxit=2 * 16, nu=1 / 500.0, zline=1)
    om = line_schedule(cfg, 16)
    o = orc.Oracle(dict(cfg, omega=om))
    f0 = turbulent_like(cfg, 3)
    o.set_fields(*f0)
    so = o.step(5)
    fo = o.get_fields()
    with stp_lib.Channel(cfg, omega=om) as ch:
        ch.set_fields(*f0)
        sg = ch.step(5)
        fg = ch.get_fields()
    assert sg["sweeps"] == so["sweeps"] == 32
    for k in ("u", "v", "w", "p", "nu"):
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < TOL64, (k, e)


@pytest.mark.parametrize("nx", [40, 64])
def test_line_step_fp32_vs_fp64_oracle(stp_lib, orc, nx):
    """FP32 line sweeps inside the FP64 refinement: per-field error against
    the FP64 oracle (converged 1e-8 solves) within the bounds stated for the
    FP32 point-sweep path (64: the vector kernel)."""
    cfg = case(nx=nx, stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=6, zline=1)
    om = line_schedule(cfg, 32)
    o = orc.Oracle(dict(cfg, omega=om))
    f0 = turbulent_like(cfg, 6)
    o.set_fields(*f0)
    o.step(5)
    fo = o.get_fields()
    with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
        ch.set_fields(*f0)
        sg = ch.step(5)
        fg = ch.get_fields()
    assert sg["converged"] and sg["rel_res"] <= 1e-8
    bounds = dict(u=2e-6, v=2e-6, w=2e-6, p=1e-3, nu=2e-6)
    for k, bd in bounds.items():
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < bd, (k, e)


@pytest.mark.parametrize("nz", [2, 3, 5])
@pytest.mark.parametrize("nx", [37, 64])
def test_line_short_columns_parity(stp_lib, orc, nx, nz):
    """Columns of 2, 3 and 5 levels: the twist level t = nz/2 sits next to
    a wall (nz = 2 leaves the upper chain empty), on the cell kernel (37)
    and the vector kernel (64).  An explicit schedule, 8 sweeps, FP64,
    against the oracle's plain Thomas solves to 1e-10."""
    cfg = case(nx=nx, ny=6, nz=nz, stretch=2.0, zline=1)
    om = [0.6, 0.9, 0.7, 1.0]  # all below 2/mu_max: a contracting iteration
    cfg["omega"] = om
    b, rng = mean_free_rhs(cfg, 11)
    p0 = rng.standard_normal(b.shape) * 0.1
    o = orc.Oracle(cfg)
    p_o, it_o, _, _ = o.poisson(b, p0, tol=0.0, maxit=8)
    with stp_lib.Channel(cfg, omega=om) as ch:
        p_g = p0.copy()
        st = ch.poisson_solve(b, p_g, tol=0.0, maxit=8)
    assert st["sweeps"] == it_o == 8
    assert rel_err(p_g, gauge(p_o, cfg)) < TOL64


@pytest.mark.parametrize("nz", [120, 200])
@pytest.mark.parametrize("nx", [37, 64])
def test_line_rows_per_block_fp64(stp_lib, orc, nx, nz):
    """FP64 blocks of two rows (96 < nz <= 192) and of one row (192 < nz <=
    384), on the cell and the vector kernel: fixed sweeps of the line
    schedule against the oracle to 1e-10."""
    cfg = case(nx=nx, ny=5, nz=nz, stretch=2.0, zline=1)
    om = line_schedule(cfg, 16)
    cfg["omega"] = om
    b, rng = mean_free_rhs(cfg, 13)
    p0 = rng.standard_normal(b.shape) * 0.1
    o = orc.Oracle(cfg)
    p_o, it_o, _, _ = o.poisson(b, p0, tol=0.0, maxit=32)
    with stp_lib.Channel(cfg, omega=om) as ch:
        p_g = p0.copy()
        st = ch.poisson_solve(b, p_g, tol=0.0, maxit=32)
    assert st["sweeps"] == it_o == 32
    assert rel_err(p_g, gauge(p_o, cfg)) < TOL64


@pytest.mark.parametrize("nz", [300, 500])
@pytest.mark.parametrize("nx", [37, 64])
def test_line_rows_per_block_fp32(stp_lib, orc, nx, nz):
    """FP32 blocks of two rows (192 < nz <= 384) and of one row (384 < nz <=
    768), cell and vector kernel: the refined solve reaches 1e-8 measured
    with the oracle's operator."""
    cfg = case(nx=nx, ny=5, nz=nz, stretch=2.0, zline=1)
    b, _ = mean_free_rhs(cfg, 17)
    o = orc.Oracle(cfg)
    with stp_lib.Channel(cfg, precision="fp32") as ch:
        p = np.zeros_like(b)
        st = ch.poisson_solve(b, p, tol=1e-8)
    r = b - o.laplacian(p)
    rel = np.sqrt(np.sum(r * r) / np.sum(b * b))
    assert st["converged"] and rel <= 1e-8 * 1.0001, rel


@pytest.mark.parametrize("nz", [2, 3, 5, 17, 64, 191, 192])
@pytest.mark.parametrize("nx", [64, 96])
def test_line_sweeps_fp32_both_kernels(stp_lib, orc, monkeypatch, nx, nz):
    """FP32 line sweeps of both kernels (the register-chunked one, variant
    1, for rows of a multiple of 32 cells and columns of up to 192 levels;
    the shared-memory lock-step one, STP_LINE_VARIANT=0): one refinement
    pass of 4 sweeps with an explicit schedule solves L d = b - L p0 from
    d = 0 in FP32, which in exact arithmetic is the oracle's 4 FP64 sweeps
    from p0.  Per element, |p - p_oracle| <= 5e-5 max|d|: the FP32
    rounding of r, of each sweep's residual (differences of wall-stretched
    couplings) and of the column solve over 4 sweeps with weights below 1
    (a contraction) reaches about 1e-5 on 192 levels, while a wrong term of
    the recurrences is of order one; and the chunked kernel's error stays
    within twice the lock-step kernel's.  With chunks of two levels or
    more (from 64 levels) the two kernels round differently, so their
    results must differ (the variant is live); chunks of one level
    reproduce the sequential elimination exactly."""
    cfg = case(nx=nx, ny=5, nz=nz, stretch=2.0, zline=1)
    om = [0.6, 0.9, 0.7, 1.0]
    cfg["omega"] = om
    b, rng = mean_free_rhs(cfg, 19)
    p0 = rng.standard_normal(b.shape) * 0.1
    p_o, it_o, _, _ = orc.Oracle(cfg).poisson(b, p0, tol=0.0, maxit=4)
    want = gauge(p_o, cfg)
    scale = np.abs(want - gauge(p0, cfg)).max()
    got, err = {}, {}
    for variant in ("0", "1"):
        monkeypatch.setenv("STP_LINE_VARIANT", variant)
        with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
            p_g = p0.copy()
            st = ch.poisson_solve(b, p_g, tol=0.0, maxit=4)
        assert st["sweeps"] == it_o == 4 and st["passes"] == 1, st
        err[variant] = np.abs(p_g - want).max() / scale
        assert err[variant] < 5e-5, (variant, err[variant])
        got[variant] = p_g
    print(f"line sweeps fp32 {nx}x5x{nz}: error/max|d| lock-step {err['0']:.3g}, chunked {err['1']:.3g}")
    assert err["1"] <= 2 * err["0"] + 1e-7, err
    if nz >= 64:
        assert not np.array_equal(got["0"], got["1"])


@pytest.mark.parametrize("shape", [(256, 24, 40), (96, 13, 64), (64, 8, 200)])
def test_persistent_line_cycle_bitwise(stp_lib, monkeypatch, shape):
    """FP32 z-line cycles as one cooperative launch (STP_LINE_PERSISTENT=1;
    each tile waits for its x-y neighbour tiles' previous sweep instead of
    a kernel boundary) give bitwise the fields of the one-launch-per-sweep
    path on the shared-memory lock-step kernel (STP_LINE_VARIANT=0), whose
    tile it runs: same arithmetic per cell, the same values read.  Grids
    with rows per tile of 4, 4 (a partial last tile row) and 2 (tall
    columns)."""
    nx, ny, nz = shape
    cfg = case(nx=nx, ny=ny, nz=nz, stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=4, zline=1)
    om = line_schedule(cfg, 32)
    monkeypatch.setenv("STP_LINE_VARIANT", "0")
    out = []
    for mode in ("0", "1"):
        monkeypatch.setenv("STP_LINE_PERSISTENT", mode)
        with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
            ch.set_fields(*turbulent_like(cfg, 14))
            st = ch.step(3)
            assert st["converged"]
            out.append((ch.get_fields(), st))
    (fa, sa), (fb, sb) = out
    assert sa["sweeps"] == sb["sweeps"] and sa["passes"] == sb["passes"]
    assert sb["launches"] < sa["launches"]
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(fa[k], fb[k]), k


def test_persistent_line_cycle_timeout_recovers(stp_lib, monkeypatch):
    """Tiles of the persistent line cycle that wait for a sweep count no
    neighbour reaches (STP_WAIT_SKEW=1, set on the host) give up after
    STP_BARRIER_WAIT clock cycles (here 1e6, about half a millisecond):
    STP_ETIMEOUT, the fields of the last good step kept, and the next call
    (flags cleared, no skew) steps as a fresh handle does."""
    cfg = case(nx=128, ny=16, nz=32, stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=4, zline=1)
    om = line_schedule(cfg, 32)
    monkeypatch.setenv("STP_LINE_PERSISTENT", "1")
    f0 = turbulent_like(cfg, 15)
    with stp_lib.Channel(cfg, precision="fp32", omega=om) as ref:
        ref.set_fields(*f0)
        ref.step(2)
        want = ref.get_fields()
    with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
        ch.set_fields(*f0)
        before = ch.get_fields()
        monkeypatch.setenv("STP_BARRIER_WAIT", "1000000")
        monkeypatch.setenv("STP_WAIT_SKEW", "1")
        with pytest.raises(stp_lib.StpError) as e:
            ch.step(1)
        assert e.value.code == stp_lib.STP_ETIMEOUT
        after = ch.get_fields()
        for k in ("u", "v", "w", "p"):
            assert np.array_equal(after[k], before[k]), k
        monkeypatch.delenv("STP_BARRIER_WAIT")
        monkeypatch.delenv("STP_WAIT_SKEW")
        st = ch.step(2)
        assert st["converged"]
        got = ch.get_fields()
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(got[k], want[k]), k
