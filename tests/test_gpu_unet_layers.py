"""Every convolution kernel of the learned-guess U-Net against the FP64
oracle, element by element, with a bound derived from the arithmetic.

Each 3x3x3 layer runs on its own through stp_unet_layer, on the kernel the
network uses for it (tcgen05 with resident or streamed weights, 1, 2 or 4 z
planes a block; mma.sync at the sizes tcgen05 does not take), at a network
shape of 1 x 16 x 64 x 64 whose levels reach every one of those paths.
Inputs and weights are BF16 on both sides, so the only differences are:

* FP32 accumulation of K products (K = 27 c_in + 1 for a forward, 27 c_out
  for a data gradient, the voxel count for a weight gradient): at most
  gamma_K * S with S the same sum over absolute values and
  gamma_K = K u / (1 - K u).  u is taken as 2^-22, four times the FP32 unit
  roundoff, because a tensor-core MMA may align its products to the largest
  exponent and truncate inside one instruction;
* the BF16 rounding of a stored result: at most 2^-8 of its magnitude
  (half a unit in the last of BF16's 8 significant bits).

So each output element obeys |y - y64| <= gamma_K S (1 + 2^-8) + 2^-8 |y64|,
where y64 is the oracle's exact FP64 value (after ReLU or the mask, which are
1-Lipschitz) and S is the oracle's convolution of the absolute values.
"""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (1, 16, 64, 64)  # n, z, y, x
U = 2.0 ** -22
H = 2.0 ** -8
TINY = 1e-30


def gamma(k):
    return k * U / (1 - k * U)


def level_of(layer):
    return layer // 2 if layer < 8 else 2 - (layer - 8) // 2


_cache = {}


def case(layer, mode):
    """Seeded inputs and the oracle's exact result and bound for one layer and mode."""
    key = (layer, mode)
    if key in _cache:
        return _cache[key]
    from oracle import unet
    spec = unet.layer_specs()[layer]
    _, ci, co, taps = spec
    theta = unet.init_params(11).astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(100 + 3 * layer + ("forward", "data_grad", "weight_grad").index(mode))
    # non-zero biases so that the bias path is checked too
    P = unet.unpack(theta)
    w = unet.bf16(P[spec[0]][0])
    bias = rng.standard_normal(co).astype(np.float32).astype(np.float64) * 0.1
    q = 0
    for (name, c_i, c_o, t) in unet.layer_specs():
        if name == spec[0]:
            break
        q += c_o * c_i * t + c_o
    theta[q + co * ci * taps:q + co * ci * taps + co] = bias
    l = level_of(layer)
    n, d, h, wd = SHAPE[0], SHAPE[1] >> l, SHAPE[2] >> l, SHAPE[3] >> l
    out = {"theta": theta, "ci": ci, "co": co}
    if mode == "forward":
        x = rng.standard_normal((n, d, h, wd, ci)).astype(np.float32).astype(np.float64)
        xb = unet.bf16(x)
        a64 = unet.conv(xb, w, bias)
        S = unet.conv(np.abs(xb), np.abs(w), np.abs(bias))
        y64 = np.maximum(a64, 0.0)
        out.update(a=x, b=None, y64=y64, E=gamma(27 * ci + 1) * S)
    elif mode == "data_grad":
        gz = rng.standard_normal((n, d, h, wd, co)).astype(np.float32).astype(np.float64)
        mask = rng.standard_normal((n, d, h, wd, ci)).astype(np.float32).astype(np.float64)
        gzb, mb = unet.bf16(gz), unet.bf16(mask)
        zero = np.zeros((n, d, h, wd, ci))
        g64 = unet.conv_backward(zero, w, gzb)[0]
        S = unet.conv_backward(zero, np.abs(w), np.abs(gzb))[0]
        keep = (mb > 0).astype(np.float64)
        out.update(a=gz, b=mask, y64=g64 * keep, E=gamma(27 * co) * S * keep)
    else:
        x = rng.standard_normal((n, d, h, wd, ci)).astype(np.float32).astype(np.float64)
        gz = rng.standard_normal((n, d, h, wd, co)).astype(np.float32).astype(np.float64)
        xb, gzb = unet.bf16(x), unet.bf16(gz)
        _, gw, gb = unet.conv_backward(xb, w, gzb)
        _, sw, _ = unet.conv_backward(np.abs(xb), w, np.abs(gzb))
        sb = np.abs(gzb).sum(axis=(0, 1, 2, 3))
        V = n * d * h * wd
        y64 = np.concatenate([gw.ravel(), gb])
        out.update(a=x, b=gz, y64=y64, E=gamma(V + 1024) * np.concatenate([sw.ravel(), sb]))
    _cache[key] = out
    return out


def run_layer(stp_lib, layer, mode, env, monkeypatch):
    torch = pytest.importorskip("torch")
    for k in ("STP_UNET_TC", "STP_UNET_TC_PLANES", "STP_UNET_MMA_NT"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    c = case(layer, mode)
    net = stp_lib.UNet(*SHAPE)
    try:
        net.set_params(c["theta"].astype(np.float32))
        ta = torch.from_numpy(c["a"].astype(np.float32)).cuda()
        tb = torch.from_numpy(c["b"].astype(np.float32)).cuda() if c["b"] is not None else None
        if mode == "weight_grad":
            shape = c["y64"].shape
        elif mode == "forward":
            shape = c["a"].shape[:4] + (c["co"],)
        else:
            shape = c["a"].shape[:4] + (c["ci"],)
        tout = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda")
        net.layer(layer, mode, ta, tb, tout)
        y = tout.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    return y, c


def check(y, c, what, stored_bf16=True):
    """The rigorous per-element bound, then a norm check that is tight:
    BF16 rounding moves each stored value by at most 2^-8 of itself, and
    FP32 sums of these lengths add about 1e-4 of the result at most, so a
    wrong tap, channel or voxel (an O(1) error) cannot pass it."""
    y64, E = c["y64"], c["E"]
    if y.shape != y64.shape:
        y = y.reshape(y64.shape)
    assert np.all(np.isfinite(y)), what
    bound = E * (1 + H) + H * np.abs(y64) + TINY
    err = np.abs(y - y64)
    bad = err > bound
    assert not bad.any(), "%s: %d of %d elements out of bound; worst err/bound %.3g" % (
        what, int(bad.sum()), bad.size, float((err / bound).max()))
    rel = np.linalg.norm(y - y64) / max(np.linalg.norm(y64), TINY)
    assert rel <= (H if stored_bf16 else 0.0) + 2e-3, (what, rel)


CONFIGS = {
    "default": {},
    "planes2": {"STP_UNET_TC": "1", "STP_UNET_TC_PLANES": "2"},
    "planes4": {"STP_UNET_TC": "1", "STP_UNET_TC_PLANES": "4"},
    "mma_sync": {"STP_UNET_TC": "0"},
}


@pytest.mark.parametrize("layer", list(range(14)))
@pytest.mark.parametrize("mode", ["forward", "data_grad", "weight_grad"])
def test_layer_default_kernels(stp_lib, orc, monkeypatch, layer, mode):
    """Every layer and pass on the kernels the network picks at this shape:
    levels 1-3 (64x64x16, 32x32x8, 16x16x4) on tcgen05, with the 64-channel
    and 192-channel layers of level 3 streaming their weights; level 4
    (8x8x2) on mma.sync; the weight gradients on mma.sync."""
    if mode == "data_grad" and layer == 0:
        pytest.skip("the input layer has no data gradient")
    y, c = run_layer(stp_lib, layer, mode, CONFIGS["default"], monkeypatch)
    check(y, c, "layer %d %s" % (layer, mode), stored_bf16=(mode != "weight_grad"))


@pytest.mark.parametrize("config", ["planes2", "planes4", "mma_sync"])
@pytest.mark.parametrize("layer", [1, 2, 3, 4, 5, 8, 9, 10, 11, 12, 13])
@pytest.mark.parametrize("mode", ["forward", "data_grad"])
def test_layer_forced_kernels(stp_lib, orc, monkeypatch, config, layer, mode):
    """The same layers with the tcgen05 block forced to 2 or 4 z planes
    (where a layer allows it; otherwise the network halves the count) and
    with every convolution on mma.sync."""
    y, c = run_layer(stp_lib, layer, mode, CONFIGS[config], monkeypatch)
    check(y, c, "layer %d %s %s" % (layer, mode, config))


@pytest.mark.parametrize("wiring,s", [((True, True, True), 1), ((False, True, True), 2),
                                      ((False, False, True), 4), ((False, False, False), 8)])
def test_network_wiring_bitwise(stp_lib, orc, wiring, s):
    """The whole network on the GPU with the pass-through parameters of the
    oracle's structure pin (channel 0 carried by each layer's centre tap;
    decoder level l reading the skip or the upsampled half of its
    concatenation) equals the oracle with BF16 storage points bit for bit:
    every sum here is exact in FP32 and both sides round the 2x2x2 means to
    BF16 the same way.  This pins the GPU's pooling, upsampling,
    concatenation layout and voxel indexing at a shape with tcgen05
    levels."""
    torch = pytest.importorskip("torch")
    from oracle import unet
    from .test_unet_oracle import passthrough_theta
    n, D, Hh, W = SHAPE
    k, j, i = np.meshgrid(np.arange(D), np.arange(Hh), np.arange(W), indexing="ij")
    # values in [1, 2): BF16 multiples of 2^-7, so 8 of them sum exactly in FP32
    x = unet.bf16(1.0 + (3 * k + 5 * j + 7 * i) % 128 / 128.0)[None]
    theta = passthrough_theta({1: wiring[0], 2: wiring[1], 3: wiring[2]})
    net = stp_lib.UNet(n, D, Hh, W)
    try:
        net.set_params(theta.astype(np.float32))
        tx = torch.from_numpy(x.astype(np.float32)).cuda()
        ty = torch.zeros_like(tx)
        net.forward(tx, ty)
        y = ty.cpu().numpy().astype(np.float64)
    finally:
        net.close()
    y_o = unet.forward(theta, x[..., None], rnd=unet.bf16)[..., 0]
    assert np.array_equal(y, y_o), np.abs(y - y_o).max()
