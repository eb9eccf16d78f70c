"""The learned-guess U-Net on the GPU (BF16 tensor-core kernels: tcgen05
with TMEM accumulators where the level's shape allows, mma.sync elsewhere) against
the FP64 oracle, with the oracle's storage points rounded to bfloat16 where
the CUDA path stores in bfloat16: forward pass, the gradient of the MSE
loss, and one Adam step."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _setup(seed, shape=(2, 8, 8, 16)):
    from oracle import unet
    rng = np.random.default_rng(seed)
    theta = unet.init_params(seed).astype(np.float32).astype(np.float64)
    x = rng.standard_normal(shape)
    t = rng.standard_normal(shape) * 0.1
    return unet, theta, x, t


def test_unet_param_count(stp_lib, orc):
    from oracle import unet
    assert stp_lib.UNet.param_count() == unet.n_params()


# (2, 8, 8, 16): every level on the mma.sync kernels; (1, 8, 16, 16): the
# full-resolution level on the tcgen05 kernel (w % 8 == 0, h % 16 == 0)
SHAPES = [(2, 8, 8, 16), (1, 8, 16, 16)]


@pytest.mark.parametrize("shape", SHAPES)
def test_unet_forward_parity(stp_lib, orc, shape):
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(1, shape)
    n, d, h, w = x.shape
    net = stp_lib.UNet(n, d, h, w)
    net.set_params(theta.astype(np.float32))
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    ty = torch.zeros_like(tx)
    net.forward(tx, ty)
    y = ty.cpu().numpy().astype(np.float64)
    y_b = unet.forward(theta, x[..., None], rnd=unet.bf16)[..., 0]
    y_e = unet.forward(theta, x[..., None])[..., 0]
    scale = np.abs(y_b).max()
    # against the bfloat16-storage oracle: FP32 accumulation order only
    assert np.abs(y - y_b).max() < 2e-2 * scale
    # against exact FP64: the size of bfloat16 storage itself
    assert np.abs(y - y_e).max() < 6e-2 * np.abs(y_e).max()
    net.close()


@pytest.mark.parametrize("shape", SHAPES)
def test_unet_gradient_parity(stp_lib, orc, shape):
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(2, shape)
    n, d, h, w = x.shape
    net = stp_lib.UNet(n, d, h, w)
    net.set_params(theta.astype(np.float32))
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    g = torch.zeros(stp_lib.UNet.param_count(), dtype=torch.float32, device="cuda")
    loss = net.gradient(tx, tt, g)
    L_o, g_o = unet.loss_and_grad(theta, x[..., None], t[..., None], rnd=unet.bf16)
    gg = g.cpu().numpy().astype(np.float64)
    assert abs(loss - L_o) < 1e-2 * L_o
    rel = np.linalg.norm(gg - g_o) / np.linalg.norm(g_o)
    cos = gg @ g_o / (np.linalg.norm(gg) * np.linalg.norm(g_o))
    assert rel < 5e-2 and cos > 0.998, (rel, cos)
    # per layer: every layer's gradient block agrees
    q = 0
    for (name, ci, co, taps) in unet.layer_specs():
        m = co * ci * taps + co
        a, b = gg[q:q + m], g_o[q:q + m]
        assert np.linalg.norm(a - b) < 0.1 * np.linalg.norm(b) + 1e-9, name
        q += m
    net.close()


def test_unet_adam_step(stp_lib, orc):
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(3)
    n, d, h, w = x.shape
    net = stp_lib.UNet(n, d, h, w)
    net.set_params(theta.astype(np.float32))
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    lr = 1e-3
    net.train_step(tx, tt, lr)
    th1 = net.get_params().astype(np.float64)
    _, g_o = unet.loss_and_grad(theta, x[..., None], t[..., None], rnd=unet.bf16)
    t_o, _, _ = unet.adam_step(theta, g_o, np.zeros_like(theta), np.zeros_like(theta), 1, lr)
    big = np.abs(g_o) > 1e-3 * np.abs(g_o).max()
    # the first Adam step moves each parameter by about lr * sign(g)
    agree = np.mean(np.sign(th1 - theta)[big] == np.sign(t_o - theta)[big])
    assert agree > 0.98, agree
    assert np.abs(th1 - theta).max() <= lr * 1.001
    net.close()


def test_unet_training_reduces_loss(stp_lib, orc):
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(4)
    n, d, h, w = x.shape
    net = stp_lib.UNet(n, d, h, w)
    net.set_params(theta.astype(np.float32))
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    l0 = net.train_step(tx, tt, 1e-3)
    for _ in range(30):
        l1 = net.train_step(tx, tt, 1e-3)
    assert l1 < 0.5 * l0
    net.close()


def test_tensor_core_conv_matches_mma_sync(stp_lib, orc, monkeypatch):
    """The tcgen05 convolutions (TMEM accumulator, operands read from a
    shared-memory halo) and the mma.sync ones compute the same network:
    forward output and gradient agree to the rounding of the FP32
    accumulation order (levels 1-3 of this shape run on tcgen05; level 1 has
    all taps' weights resident, the 192- and 64-channel layers of level 3
    stream them through the stage ring)."""
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(4, (1, 8, 64, 32))
    n, d, h, w = x.shape
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    out = {}
    for tc in ("0", "1"):
        monkeypatch.setenv("STP_UNET_TC", tc)
        net = stp_lib.UNet(n, d, h, w)
        net.set_params(theta.astype(np.float32))
        ty = torch.zeros_like(tx)
        net.forward(tx, ty)
        g = torch.zeros(stp_lib.UNet.param_count(), dtype=torch.float32, device="cuda")
        loss = net.gradient(tx, tt, g)
        out[tc] = (ty.cpu().numpy().astype(np.float64), g.cpu().numpy().astype(np.float64), loss)
        net.close()
    (y0, g0, l0), (y1, g1, l1) = out["0"], out["1"]
    assert np.abs(y1 - y0).max() < 2e-2 * np.abs(y0).max()
    assert abs(l1 - l0) < 1e-2 * l0
    assert np.linalg.norm(g1 - g0) < 5e-2 * np.linalg.norm(g0)
    assert g1 @ g0 / (np.linalg.norm(g1) * np.linalg.norm(g0)) > 0.998


@pytest.mark.parametrize("planes", ["2", "4"])
def test_tensor_core_planes_per_block(stp_lib, orc, monkeypatch, planes):
    """tcgen05 blocks computing 2 or 4 z planes (one halo of planes + 2, one
    weight load, one accumulator per plane in tensor memory) give the same
    network as one plane a block: each plane's accumulator sees the same
    sequence of MMAs, so the forward output is bitwise equal; the gradient
    (its weight part accumulated with atomics) agrees to rounding.  Level 3
    of this shape is 2 deep, so a forced 4 falls back to 2 there."""
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(4, (1, 8, 64, 32))
    n, d, h, w = x.shape
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    out = {}
    monkeypatch.setenv("STP_UNET_TC", "1")
    for pl in ("1", planes):
        monkeypatch.setenv("STP_UNET_TC_PLANES", pl)
        net = stp_lib.UNet(n, d, h, w)
        net.set_params(theta.astype(np.float32))
        ty = torch.zeros_like(tx)
        net.forward(tx, ty)
        g = torch.zeros(stp_lib.UNet.param_count(), dtype=torch.float32, device="cuda")
        net.gradient(tx, tt, g)
        out[pl] = (ty.cpu().numpy(), g.cpu().numpy().astype(np.float64))
        net.close()
    (y1, g1), (yp, gp) = out["1"], out[planes]
    assert np.array_equal(y1, yp)
    assert np.linalg.norm(gp - g1) < 1e-5 * np.linalg.norm(g1)


def test_mma_sync_widths_bitwise(stp_lib, orc, monkeypatch):
    """The mma.sync convolutions with 64, 32, 16 or 8 output channels a
    block (forced; the library picks by grid size) compute every output
    with the same sequence of MMAs: forward outputs are bitwise equal; the
    loss and the gradient, which sum with atomics, agree to rounding."""
    torch = pytest.importorskip("torch")
    unet, theta, x, t = _setup(5, (1, 8, 64, 32))
    n, d, h, w = x.shape
    tx = torch.from_numpy(x.astype(np.float32)).cuda()
    tt = torch.from_numpy(t.astype(np.float32)).cuda()
    monkeypatch.setenv("STP_UNET_TC", "0")
    out = {}
    for nt in ("8", "4", "2", "1"):
        monkeypatch.setenv("STP_UNET_MMA_NT", nt)
        net = stp_lib.UNet(n, d, h, w)
        net.set_params(theta.astype(np.float32))
        ty = torch.zeros_like(tx)
        net.forward(tx, ty)
        g = torch.zeros(stp_lib.UNet.param_count(), dtype=torch.float32, device="cuda")
        loss = net.gradient(tx, tt, g)
        out[nt] = (ty.cpu().numpy(), g.cpu().numpy().astype(np.float64), loss)
        net.close()
    y8, g8, l8 = out["8"]
    for nt in ("4", "2", "1"):
        y, g, l = out[nt]
        assert np.array_equal(y, y8), nt
        assert abs(l - l8) <= 1e-6 * l8, nt
        assert np.linalg.norm(g - g8) < 1e-5 * np.linalg.norm(g8), nt
