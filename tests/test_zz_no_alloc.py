"""The allocation-free residual entry point (stp_poisson_residual_noalloc).

It is meant for callers that hold their own device buffers but may not
allocate device memory; its scratch is a fixed array inside the library
shared by every call.  Here it is called through the C ABI twice in a row,
on different inputs, and each result is compared with the residual built
from the existing entry point stp_eval(laplacian) on the same p and b."""
import math

import numpy as np
import pytest

from paper_1511_07800_gb300 import inputs

pytestmark = pytest.mark.gpu


def _reference_residual(stp_lib, cfg, p, b):
    """b - L p from the existing entry point (stp_eval with the Laplacian)."""
    with stp_lib.Channel(cfg) as ch:
        u, v, w = inputs.zeros(cfg)
        ch.set_fields(u, v, w, p)
        return b - ch.eval("laplacian")


@pytest.mark.parametrize("stretch,shape", [(0.0, (40, 19, 14)), (2.0, (64, 24, 32))])
def test_noalloc_residual_matches_existing_entry_point(stp_lib, stretch, shape):
    torch = pytest.importorskip("torch")
    nx, ny, nz = shape
    cfg = dict(nx=nx, ny=ny, nz=nz, Lx=2 * math.pi, Ly=math.pi, Lz=2.0, nu=0.01, dt=1e-3, stretch=stretch)
    rng = np.random.default_rng(21)
    for call in range(2):
        p = rng.standard_normal((nz, ny, nx))
        b = rng.standard_normal((nz, ny, nx)) * (1 + call)
        r_ref = _reference_residual(stp_lib, cfg, p, b)
        n_ref = float(np.sqrt(np.sum(r_ref * r_ref)))
        tp, tb = torch.from_numpy(p).cuda(), torch.from_numpy(b).cuda()
        tr = torch.full_like(tp, float("nan"))
        n = stp_lib.poisson_residual_noalloc(cfg, tp, tb, tr)
        assert abs(n - n_ref) <= 1e-12 * n_ref, (call, n, n_ref)
        r = tr.cpu().numpy()
        assert np.abs(r - r_ref).max() <= 1e-12 * np.abs(r_ref).max(), call


def test_noalloc_rejects_oversized_grid(stp_lib):
    torch = pytest.importorskip("torch")
    cfg = dict(nx=8, ny=8, nz=5000, Lx=1.0, Ly=1.0, Lz=2.0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(stp_lib.StpError) as e:
        stp_lib.poisson_residual_noalloc(cfg, t, t)
    assert e.value.code == stp_lib.STP_EINVAL and "scratch" in str(e.value)
