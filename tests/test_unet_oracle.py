"""Pins of the FP64 U-Net oracle (learned pressure guess): convolution by
its impulse response and adjointness, pooling/upsampling adjoints, the
full-network gradient against central finite differences, and the first
Adam step against its closed form."""
import numpy as np


def test_param_count(orc):
    from oracle import unet
    # 14 3x3x3 convolutions + the 1x1 output layer of the 16-32-64-128 U-Net
    expect = 0
    for ci, co in [(1, 16), (16, 16), (16, 32), (32, 32), (32, 64), (64, 64), (64, 128), (128, 128),
                   (192, 64), (64, 64), (96, 32), (32, 32), (48, 16), (16, 16)]:
        expect += 27 * ci * co + co
    expect += 16 + 1
    assert unet.n_params() == expect


def test_conv_impulse_response(orc):
    """A unit impulse at v0 returns the weights: y[v0 - off(t)] = W[:, 0, t] + b,
    with the periodic wrap in x and y."""
    from oracle import unet
    rng = np.random.default_rng(1)
    w = rng.standard_normal((3, 1, 27))
    b = rng.standard_normal(3)
    x = np.zeros((1, 6, 5, 4, 1))
    v0 = (3, 0, 3)
    x[0, v0[0], v0[1], v0[2], 0] = 1.0
    y = unet.conv(x, w, b)
    for t in range(27):
        kz, ky, kx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
        v = (v0[0] - kz, (v0[1] - ky) % 5, (v0[2] - kx) % 4)
        assert np.allclose(y[0, v[0], v[1], v[2]], w[:, 0, t] + b)
    # far from the impulse only the bias remains
    assert np.allclose(y[0, 0, 2, 1], b)


def test_conv_zero_padding_in_z(orc):
    """A constant field: interior voxels see all 27 taps, wall voxels 18."""
    from oracle import unet
    rng = np.random.default_rng(2)
    w = rng.standard_normal((2, 1, 27))
    x = np.ones((1, 4, 4, 4, 1))
    y = unet.conv(x, w, np.zeros(2))
    assert np.allclose(y[0, 1:3], w[:, 0, :].sum(axis=1))
    assert np.allclose(y[0, 0], w[:, 0, 9:].sum(axis=1))
    assert np.allclose(y[0, 3], w[:, 0, :18].sum(axis=1))


def test_adjoints(orc):
    from oracle import unet
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 4, 6, 8, 3))
    w = rng.standard_normal((5, 3, 27))
    g = rng.standard_normal((2, 4, 6, 8, 5))
    gx, gw, gb = unet.conv_backward(x, w, g)
    y = unet.conv(x, w, np.zeros(5))
    assert np.isclose(np.sum(y * g), np.sum(x * gx))
    assert np.isclose(np.sum(y * g), np.sum(w * gw))
    assert np.allclose(gb, g.sum(axis=(0, 1, 2, 3)))
    p = rng.standard_normal((2, 2, 3, 4, 3))
    assert np.isclose(np.sum(unet.pool(x) * p), np.sum(x * unet.pool_backward(p)))
    assert np.isclose(np.sum(unet.upsample(p) * x), np.sum(p * unet.upsample_backward(x)))


def test_network_gradient_finite_differences(orc):
    """Directional derivatives of the MSE loss agree with the backward pass."""
    from oracle import unet
    rng = np.random.default_rng(4)
    theta = unet.init_params(5)
    x = rng.standard_normal((1, 8, 8, 8, 1))
    t = rng.standard_normal((1, 8, 8, 8, 1))
    L, g = unet.loss_and_grad(theta, x, t)
    for k in range(4):
        d = rng.standard_normal(theta.size)
        d /= np.linalg.norm(d)
        eps = 1e-5
        lp = unet.mse(unet.forward(theta + eps * d, x), t)[0]
        lm = unet.mse(unet.forward(theta - eps * d, x), t)[0]
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g @ d) < 1e-6 * max(1.0, abs(fd)), (k, fd, g @ d)


def test_adam_first_step_closed_form(orc):
    """First Adam step: m_hat = g, v_hat = g^2, so theta -= lr g / (|g| + eps)."""
    from oracle import unet
    rng = np.random.default_rng(6)
    th = rng.standard_normal(50)
    g = rng.standard_normal(50)
    t1, m, v = unet.adam_step(th, g, np.zeros(50), np.zeros(50), 1, 1e-3)
    assert np.allclose(t1, th - 1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
