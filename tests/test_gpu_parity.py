"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

FP64: element-wise agreement to 1e-10 relative (max-norm over max |field|)
on identical seeded inputs, with the pressure solves forced to the same
number of SRJ sweeps where a solve is involved.  FP32 sweeps with FP64
refinement: the error against the FP64 oracle is bounded per field.
Grids are chosen to span several 32 x 8 thread tiles with ragged tails.
"""
import math

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

from .conftest import gauge, rel_err

pytestmark = pytest.mark.gpu

PI = math.pi
TOL64 = 1e-10


def case(nx=40, ny=19, nz=14, stretch=0.0, les=0, nu=0.01, **over):
    c = dict(nx=nx, ny=ny, nz=nz, Lx=2 * PI, Ly=PI, Lz=2.0, nu=nu, dt=2e-3, forcing=0, fx=0.02, ubulk=1.0,
             les=les, cs=0.1, vd_a=25.0, re_tau=180.0, stretch=stretch, cn_sweeps=4, ptol=1e-8, pmaxit=100000)
    c.update(over)
    return c


def schedule(cfg, M=16):
    from oracle import srj
    om, _, _ = srj.schedule_for(cfg["nx"], cfg["ny"], cfg["nz"], cfg["Lx"], cfg["Ly"], cfg["Lz"],
                                cfg.get("stretch", 0.0), M)
    return om


def turbulent_like(cfg, seed):
    """Laminar profile plus strong noise: exercises every term."""
    u, v, w = inputs.noise(cfg, 0.2, seed, inputs.poiseuille(cfg, 1.0))
    return u, v, w


@pytest.mark.parametrize("stretch,les", [(0.0, 0), (2.0, 0), (0.0, 1), (2.0, 1)])
def test_terms_parity(stp_lib, orc, stretch, les):
    """nu_T (Sec. 2.2), explicit terms and diffusion (Sec. 3.1), divergence
    and Laplacian (Eq. presdiv) evaluated on the same fields."""
    cfg = case(stretch=stretch, les=les)
    u, v, w = turbulent_like(cfg, 1)
    p = np.random.default_rng(2).standard_normal(u.shape)
    o = orc.Oracle(cfg)
    with stp_lib.Channel(cfg, omega=schedule(cfg)) as ch:
        ch.set_fields(u, v, w, p)
        nu_g = ch.eval("viscosity")
        nu_o = o.viscosity(u, v, w)
        assert rel_err(nu_g, nu_o) < 1e-12
        for term, fn in (("explicit", lambda: o.explicit(u, v, w, nu_o)),
                         ("diffusion", lambda: o.diffusion(u, v, w, nu_o))):
            got = ch.eval(term)
            exp = fn()
            for a, b in zip(got, exp):
                assert rel_err(a, b) < 1e-12, term
        assert rel_err(ch.eval("divergence"), o.divergence(u, v, w)) < 1e-12
        assert rel_err(ch.eval("laplacian"), o.laplacian(p)) < 1e-12


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_divergence_fp32_fields(stp_lib, orc, stretch):
    """Eq. presdiv with FP32 fields: the kernel keeps each face difference
    and its product with the (FP32) metric as exact two-float sums, so b
    equals the FP64 evaluation of the same FP32 numbers to FP64 rounding
    (1e-13 against a numpy FP64 evaluation with the metric rounded to FP32
    as the library rounds it); against the oracle's FP64 divergence of the
    rounded fields, which uses the FP64 metric, the metric's FP32 rounding
    remains (below 1e-6)."""
    cfg = case(stretch=stretch, nx=40, ny=19, nz=14)
    u, v, w = turbulent_like(cfg, 4)
    u32, v32, w32 = (np.asarray(a, np.float32).astype(np.float64) for a in (u, v, w))
    zf = inputs.zfaces(cfg)
    idx = float(np.float32(1.0 / (cfg["Lx"] / cfg["nx"])))
    idy = float(np.float32(1.0 / (cfg["Ly"] / cfg["ny"])))
    idz = (1.0 / np.diff(zf)).astype(np.float32).astype(np.float64)[:, None, None]
    want = ((np.roll(u32, -1, axis=2) - u32) * idx + (np.roll(v32, -1, axis=1) - v32) * idy +
            (w32[1:] - w32[:-1]) * idz)
    with stp_lib.Channel(cfg, precision="fp32") as ch:
        ch.set_fields(u, v, w)
        got = ch.eval("divergence")
    assert rel_err(got, want) < 1e-13
    assert rel_err(got, orc.Oracle(cfg).divergence(u32, v32, w32)) < 1e-6


@pytest.mark.parametrize("stretch", [0.0, 2.0])
def test_srj_fixed_sweeps_parity(stp_lib, orc, stretch):
    """Sec. 3.4: the same schedule applied for the same number of sweeps
    gives the same pressure."""
    cfg = case(nx=48, ny=20, nz=18, stretch=stretch)
    om = schedule(cfg, 32)
    cfg["omega"] = om
    rng = np.random.default_rng(5)
    b = rng.standard_normal((18, 20, 48))
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    b -= np.sum(b * dz) / np.sum(dz * np.ones_like(b))
    p0 = rng.standard_normal(b.shape) * 0.1
    o = orc.Oracle(cfg)
    p_o, it_o, rel_o, conv_o = o.poisson(b, p0, tol=0.0, maxit=3 * 32)
    with stp_lib.Channel(cfg, omega=om) as ch:
        p_g = p0.copy()
        st = ch.poisson_solve(b, p_g, tol=0.0, maxit=3 * 32)
    assert st["sweeps"] == it_o == 96 and not st["converged"] and not conv_o
    assert rel_err(p_g, gauge(p_o, cfg)) < TOL64
    assert abs(st["rel_res"] - rel_o) < 1e-9 * rel_o


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_poisson_converges_to_tolerance(stp_lib, orc, precision):
    """The solve stops with ||b - Lp|| <= tol ||b||, checked with the
    oracle's operator, from a zero guess."""
    cfg = case(nx=64, ny=24, nz=32, stretch=2.0)
    rng = np.random.default_rng(7)
    b = rng.standard_normal((32, 24, 64))
    dz = np.diff(inputs.zfaces(cfg))[:, None, None]
    b -= np.sum(b * dz) / np.sum(dz * np.ones_like(b))
    o = orc.Oracle(cfg)
    with stp_lib.Channel(cfg, precision=precision) as ch:
        p = np.zeros_like(b)
        st = ch.poisson_solve(b, p, tol=1e-8)
    r = b - o.laplacian(p)
    rel = np.sqrt(np.sum(r * r) / np.sum(b * b))
    assert st["converged"] and rel <= 1e-8 * 1.0001
    assert abs(rel - st["rel_res"]) < 1e-3 * rel + 1e-15
    if precision == "fp32":
        assert st["passes"] >= 2


def run_both(stp_lib, orc, cfg, fields, nsteps, omega, precision="fp64"):
    o = orc.Oracle(dict(cfg, omega=omega))
    o.set_fields(*fields)
    so = o.step(nsteps)
    with stp_lib.Channel(cfg, precision=precision, omega=omega) as ch:
        ch.set_fields(*fields)
        sg = ch.step(nsteps)
        fg = ch.get_fields()
    return o.get_fields(), so, fg, sg


@pytest.mark.parametrize("stretch,les,forcing", [(0.0, 0, 0), (2.0, 1, 1), (2.0, 0, 0), (0.0, 1, 1)])
def test_step_parity_fp64(stp_lib, orc, stretch, les, forcing):
    """Whole projection steps (Sec. 3.1) with the pressure solves forced to
    two SRJ cycles each: every field agrees to 1e-10 relative."""
    cfg = case(stretch=stretch, les=les, forcing=forcing, ptol=0.0, pmaxit=2 * 16, nu=1 / 500.0)
    om = schedule(cfg, 16)
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, turbulent_like(cfg, 3), 6, om)
    assert sg["sweeps"] == so["sweeps"] == 32
    for k in ("u", "v", "w", "p", "nu"):
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < TOL64, (k, e)
    assert abs(sg["ubulk"] - so["ubulk"]) < 1e-12
    if forcing == 1:
        assert abs(sg["ubulk"] - 1.0) < 1e-12


@pytest.mark.parametrize("stretch,les,forcing,sweeps,shape", [(2.0, 1, 1, 2, None), (0.0, 0, 0, 3, None),
                                                               (2.0, 0, 0, 1, None), (1.0, 1, 0, 4, None),
                                                               (2.0, 1, 0, 2, (33, 5, 210)),
                                                               (2.0, 1, 1, 2, (9, 3, 2))])
def test_step_parity_cn_zline_fp64(stp_lib, orc, stretch, les, forcing, sweeps, shape):
    """Whole steps with the Crank-Nicolson system solved by z-line Jacobi
    sweeps (Thomas on every column, x-y neighbours from the previous
    iterate), held to a few sweeps so that every sweep's exact arithmetic
    matters: every field agrees with the oracle's line sweeps to 1e-10.
    Also tall columns (210 levels) and two levels, where each w column has
    a single unknown."""
    extra = {} if shape is None else dict(nx=shape[0], ny=shape[1], nz=shape[2])
    cfg = case(stretch=stretch, les=les, forcing=forcing, ptol=0.0, pmaxit=2 * 16, nu=1 / 300.0, dt=4e-3,
               cn_zline=1, cn_sweeps=sweeps, **extra)
    om = schedule(cfg, 16)
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, turbulent_like(cfg, 3), 4, om)
    for k in ("u", "v", "w", "p", "nu"):
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < TOL64, (k, e)


@pytest.mark.parametrize("shape", [(40, 19, 14), (33, 7, 9), (64, 24, 32)])
def test_step_cn_zline_fp32_and_converged(stp_lib, orc, shape):
    """FP32 steps with z-line Crank-Nicolson sweeps and converged pressure
    solves stay within the FP32 bounds of the FP64 oracle; with the automatic
    sweep count (contraction below 1e-12) the z-line and point solves of the
    Crank-Nicolson system give the same step to 1e-10 in FP64."""
    nx, ny, nz = shape
    base = case(nx=nx, ny=ny, nz=nz, stretch=2.0, les=1, nu=1 / 500.0, cn_zline=1, cn_sweeps=5)
    om = schedule(base, 16)
    fo, so, fg, sg = run_both(stp_lib, orc, base, turbulent_like(base, 6), 3, om, precision="fp32")
    assert sg["converged"]
    scale = max(np.abs(fo[k]).max() for k in ("u", "v", "w"))
    for k in ("u", "v", "w"):
        assert np.abs(fg[k] - fo[k]).max() / scale < 2e-6, k
    out = {}
    for zl in (0, 1):
        # fixed pressure sweeps, so that the solves stay linear in b and the
        # two runs differ only by the Crank-Nicolson solutions (1e-12)
        with stp_lib.Channel(dict(base, cn_zline=zl, cn_sweeps=0, ptol=0.0, pmaxit=32), precision="fp64",
                             omega=om) as ch:
            ch.set_fields(*turbulent_like(base, 6))
            ch.step(3)
            out[zl] = ch.get_fields()
    for k in ("u", "v", "w"):
        assert rel_err(out[1][k], out[0][k]) < 1e-10, k


def test_cn_auto_count_fp32_reaches_storage_precision(stp_lib):
    """With FP32 fields the automatic Crank-Nicolson count stops at a 2^-24
    contraction bound instead of 1e-12: 3 z-line sweeps on the LES channel's
    x-y spacing, where FP64 fields take 5.  Three steps of a channel with
    that spacing give the same fields with the automatic count as with 12
    sweeps, to FP32 rounding (2e-6 of the velocity scale, 1e-3 of the
    pressure)."""
    import math
    import bench
    cfg = inputs.preset("les_channel", nx=64, ny=32, nz=48, Lx=math.pi, Ly=math.pi / 2, zline=1, cn_zline=1)
    assert bench._auto_cn(cfg, "fp32") == 3 and bench._auto_cn(cfg, "fp64") == 5
    f0 = inputs.initial_fields("les_channel", cfg, seed=3)
    out = {}
    for n in (0, 12):
        with stp_lib.Channel(dict(cfg, cn_sweeps=n), precision="fp32") as ch:
            ch.set_fields(*f0)
            st = ch.step(3)
            assert st["converged"]
            out[n] = ch.get_fields()
    scale = max(np.abs(out[12][k]).max() for k in ("u", "v", "w"))
    for k in ("u", "v", "w"):
        assert np.abs(out[0][k] - out[12][k]).max() / scale < 2e-6, k
    assert rel_err(out[0]["p"] - out[0]["p"].mean(), out[12]["p"] - out[12]["p"].mean()) < 1e-3


def test_step_parity_converged_solves(stp_lib, orc):
    """Steps with tolerance-driven solves take the same sweep counts and
    agree to 1e-10 (instability workload shape on a 2-D slice)."""
    cfg = inputs.preset("os_instability", nx=64, ny=3, nz=48, cn_sweeps=0)
    om = schedule(cfg, 64)
    cfg["cn_sweeps"] = 6
    u, v, w = inputs.initial_fields("os_instability", cfg, seed=0)
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, (u, v, w), 5, om)
    assert so["converged"] and sg["converged"]
    assert sg["sweeps"] == so["sweeps"]
    for k in ("u", "v", "w"):
        assert rel_err(fg[k], fo[k]) < TOL64, k
    assert rel_err(fg["w"] - w, fo["w"] - w) < 1e-7


def test_laminar_startup_workload(stp_lib, orc):
    """The laminar start-up workload (32 x 16 x 32, Re 100, 100 steps): GPU
    against the oracle and against the exact 1-D reduction."""
    from .test_oracle_pins import _startup_exact_discrete
    cfg = inputs.preset("laminar_startup", cn_sweeps=8)
    om = schedule(cfg, 64)
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, inputs.zeros(cfg), 100, om)
    assert rel_err(fg["u"], fo["u"]) < TOL64
    exact = _startup_exact_discrete(32, 2.0, cfg["nu"], cfg["fx"], cfg["dt"], 100)
    assert np.abs(fg["u"][:, 3, 5] - exact).max() < 1e-12
    assert np.abs(fg["v"]).max() < 1e-14 and np.abs(fg["w"]).max() < 1e-14


def test_edge_shapes(stp_lib, orc):
    """Smallest legal grid, odd sizes and the 2-D trick ny = 3."""
    for (nx, ny, nz) in [(3, 3, 2), (33, 3, 5), (31, 9, 3)]:
        cfg = case(nx=nx, ny=ny, nz=nz, ptol=0.0, pmaxit=8, les=1, stretch=1.0)
        om = schedule(cfg, 8)
        fo, so, fg, sg = run_both(stp_lib, orc, cfg, turbulent_like(cfg, 9), 3, om)
        for k in ("u", "v", "w"):
            assert rel_err(fg[k], fo[k]) < TOL64, (nx, ny, nz, k)


@pytest.mark.parametrize("zline", [0, 1])
@pytest.mark.parametrize("shape", [(3, 3, 2), (33, 3, 5), (31, 9, 3), (42, 7, 9), (66, 10, 13)])
def test_edge_shapes_fp32(stp_lib, orc, shape, zline):
    """FP32 sweeps with FP64 refinement on ragged grids: rows that are not
    a multiple of 4 cells (the scalar sweep kernel, no float4 tiles, no
    autotuner), odd level counts and the 2-D trick ny = 3; point and z-line
    sweeps.  Both sides solve the pressure to 1e-8; every field is within
    the per-field FP32 bounds of the FP64 oracle."""
    nx, ny, nz = shape
    cfg = case(nx=nx, ny=ny, nz=nz, les=1, stretch=1.0, nu=1 / 500.0, cn_sweeps=6, zline=zline)
    from oracle import srj
    om, _, _ = srj.schedule_for(nx, ny, nz, cfg["Lx"], cfg["Ly"], cfg["Lz"], cfg["stretch"], 16, line=bool(zline))
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, turbulent_like(cfg, 9), 3, om, precision="fp32")
    assert sg["converged"] and so["converged"]
    bounds = dict(u=2e-6, v=2e-6, w=2e-6, p=1e-3, nu=2e-6)
    for k, bd in bounds.items():
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < bd, (shape, zline, k, e)


def test_bad_wall_rejected(stp_lib):
    cfg = case()
    u, v, w = inputs.zeros(cfg)
    w[0, 1, 1] = 1.0
    with stp_lib.Channel(cfg) as ch:
        with pytest.raises(stp_lib.StpError) as e:
            ch.set_fields(u, v, w)
        assert e.value.code == stp_lib.STP_EINVAL


def test_device_pointers_roundtrip(stp_lib):
    """Fields passed and returned as device memory (torch tensors)."""
    torch = pytest.importorskip("torch")
    cfg = case()
    u, v, w = turbulent_like(cfg, 4)
    with stp_lib.Channel(cfg, omega=schedule(cfg)) as ch:
        tu, tv, tw = (torch.from_numpy(a).cuda() for a in (u, v, w))
        ch.set_fields(tu, tv, tw)
        out = {k: torch.zeros_like(tu) for k in ("u", "v", "p", "nu")}
        out["w"] = torch.zeros_like(tw)
        ch.get_fields(out)
        torch.cuda.synchronize()
        assert np.array_equal(out["u"].cpu().numpy(), u) and np.array_equal(out["w"].cpu().numpy(), w)


@pytest.mark.parametrize("stretch,les", [(0.0, 0), (2.0, 1)])
def test_fp32_refine_error_vs_fp64_oracle(stp_lib, orc, stretch, les):
    """FP32 sweeps with FP64 refinement: per-field error against the FP64
    oracle after 5 steps with converged (1e-8) pressure solves.  The
    pressure carries the FP32 rounding of u* amplified by 1/(dt dx) through
    b = D u*/dt, so its bound is the loosest."""
    cfg = case(stretch=stretch, les=les, nu=1 / 500.0, cn_sweeps=6)
    om = schedule(cfg, 32)
    fo, so, fg, sg = run_both(stp_lib, orc, cfg, turbulent_like(cfg, 6), 5, om, precision="fp32")
    assert sg["converged"] and sg["rel_res"] <= 1e-8
    bounds = dict(u=2e-6, v=2e-6, w=2e-6, p=1e-3, nu=2e-6)
    for k, bd in bounds.items():
        e = rel_err(fg[k], fo[k]) if k != "p" else rel_err(fg[k] - fg[k].mean(), fo[k] - fo[k].mean())
        assert e < bd, (k, e)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_host_driven_solve_matches_graph(stp_lib, monkeypatch, precision):
    """The host-driven solve (STP_HOST_SOLVE=1, for profilers) runs the same
    kernels in the same order as the device-steered graph: identical fields."""
    cfg = case(stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=4)
    om = schedule(cfg, 16)
    out = []
    for mode in ("0", "1"):
        monkeypatch.setenv("STP_HOST_SOLVE", mode)
        with stp_lib.Channel(cfg, precision=precision, omega=om) as ch:
            ch.set_fields(*turbulent_like(cfg, 8))
            st = ch.step(3)
            out.append((ch.get_fields(), st))
    (fa, sa), (fb, sb) = out
    assert sa["sweeps"] == sb["sweeps"] and sa["passes"] == sb["passes"]
    for k in ("u", "v", "w", "p"):
        assert np.array_equal(fa[k], fb[k]), k


def test_persistent_cycle_matches_per_sweep_kernels(stp_lib, monkeypatch):
    """FP32 SRJ cycles as one persistent cooperative kernel (grid barriers
    between sweeps) give the fields of the one-kernel-per-sweep path."""
    cfg = case(nx=64, ny=20, nz=24, stretch=2.0, les=1, nu=1 / 500.0, cn_sweeps=4)
    om = schedule(cfg, 32)
    out = []
    for mode in ("0", "1"):
        monkeypatch.setenv("STP_PERSISTENT", mode)
        with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
            ch.set_fields(*turbulent_like(cfg, 12))
            st = ch.step(3)
            assert st["converged"]
            out.append((ch.get_fields(), st))
    (fa, sa), (fb, sb) = out
    assert sa["sweeps"] == sb["sweeps"]
    for k in ("u", "v", "w", "p"):
        assert rel_err(fb[k] - fb[k].mean() * (k == "p"), fa[k] - fa[k].mean() * (k == "p")) < 1e-6, k


@pytest.mark.parametrize("shape", [(64, 24, 32), (32, 12, 16)])
def test_sweep_variants_identical(stp_lib, monkeypatch, shape):
    """Every FP32 sweep tile shape the autotuner may pick computes the same
    values (z levels per thread, rows per block, warps packed along the
    plane, and two sweeps per launch on a shared-memory tile only change the
    mapping).  The second grid has rows of 8 float4 units, so a packed warp
    holds four rows and wraps x inside the warp."""
    nx, ny, nz = shape
    cfg = case(nx=nx, ny=ny, nz=nz, stretch=2.0, les=0, nu=1 / 500.0, cn_sweeps=4)
    om = schedule(cfg, 32)
    ref = None
    ran = set()
    for v in range(12):
        monkeypatch.setenv("STP_SWEEP_VARIANT", str(v))
        with stp_lib.Channel(cfg, precision="fp32", omega=om) as ch:
            ch.set_fields(*turbulent_like(cfg, 13))
            ch.step(2)
            f = ch.get_fields()
            ran.add(ch.sweep_tile()[0])
        if ref is None:
            ref = f
        else:
            for k in ("u", "v", "w", "p"):
                assert np.array_equal(f[k], ref[k]), (v, k)
    # the pair tiles (two sweeps per launch) that fit these grids did run
    assert ({10, 11} | ({9} if ny % 8 == 0 else set())) <= ran, ran
