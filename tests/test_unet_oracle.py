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


def test_pool_closed_forms(orc):
    """2x2x2 mean pooling: a field constant on each aligned 2x2x2 block pools
    to that constant; a one-hot fine voxel (z, y, x) pools to 1/8 at
    (z//2, y//2, x//2) and nothing else; a linear ramp pools to its value at
    each block's centre (the mean of a linear function over a symmetric
    block)."""
    from oracle import unet
    rng = np.random.default_rng(7)
    D, H, W, C = 4, 6, 8, 2
    blocks = rng.standard_normal((1, D // 2, H // 2, W // 2, C))
    x = np.zeros((1, D, H, W, C))
    for z in range(D):
        for y in range(H):
            for xx in range(W):
                x[0, z, y, xx] = blocks[0, z // 2, y // 2, xx // 2]
    assert np.allclose(unet.pool(x), blocks, rtol=0, atol=1e-15)
    for (z, y, xx) in [(0, 0, 0), (3, 5, 7), (1, 4, 2), (2, 1, 5)]:
        one = np.zeros((1, D, H, W, 1))
        one[0, z, y, xx, 0] = 1.0
        p = unet.pool(one)
        expect = np.zeros((1, D // 2, H // 2, W // 2, 1))
        expect[0, z // 2, y // 2, xx // 2, 0] = 0.125
        assert np.array_equal(p, expect)
    k, j, i = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    ramp = (0.5 + 0.3 * k + 0.2 * j + 0.1 * i)[None, ..., None]
    kc, jc, ic = np.meshgrid(2 * np.arange(D // 2) + 0.5, 2 * np.arange(H // 2) + 0.5, 2 * np.arange(W // 2) + 0.5,
                             indexing="ij")
    centre = (0.5 + 0.3 * kc + 0.2 * jc + 0.1 * ic)[None, ..., None]
    assert np.allclose(unet.pool(ramp), centre, rtol=0, atol=1e-14)


def test_upsample_closed_forms(orc):
    """Nearest x2 upsampling: a one-hot coarse voxel becomes exactly its 8
    fine voxels (2z..2z+1, 2y..2y+1, 2x..2x+1), with value 1 and nothing
    else set."""
    from oracle import unet
    d, h, w = 2, 3, 4
    for (z, y, x) in [(0, 0, 0), (1, 2, 3), (0, 1, 2)]:
        one = np.zeros((1, d, h, w, 1))
        one[0, z, y, x, 0] = 1.0
        up = unet.upsample(one)
        expect = np.zeros((1, 2 * d, 2 * h, 2 * w, 1))
        expect[0, 2 * z:2 * z + 2, 2 * y:2 * y + 2, 2 * x:2 * x + 2, 0] = 1.0
        assert np.array_equal(up, expect)


def passthrough_theta(dec_from_skip):
    """Parameters of a network that carries channel 0 unchanged through every
    layer: each 3x3x3 convolution has the centre tap (t = 13, offset 0) of
    output 0 set to 1 on one input channel, every other weight and bias 0,
    and the output layer copies channel 0.  For decoder level l (1..3)
    dec_from_skip[l] chooses the input channel of its first convolution: the
    skip half of the concatenation (channel C_{l+1}, the first skip
    channel) or the upsampled half (channel 0)."""
    from oracle import unet
    parts = []
    for (name, ci, co, t) in unet.layer_specs():
        w = np.zeros((co, ci, t))
        src = 0
        if name.startswith("dec") and name.endswith("_a"):
            l = int(name[3])
            src = unet.CH[l] if dec_from_skip[l] else 0
        w[0, src, 13 if t == 27 else 0] = 1.0
        parts += [w.ravel(), np.zeros(co)]
    return np.concatenate(parts)


def block_centre_ramp(D, H, W, s):
    """The ramp below averaged over aligned s x s x s blocks and broadcast back:
    for a linear field that is its value at each block's centre."""
    k, j, i = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    c = lambda a: (a // s) * s + 0.5 * (s - 1)
    return 1.0 + 0.03 * c(k) + 0.02 * c(j) + 0.01 * c(i)


def test_network_structure_closed_forms(orc):
    """The U-Net's wiring, through networks with known outputs.  With the
    pass-through parameters and a positive linear input (so every ReLU
    passes), the output is the input averaged over aligned blocks of 2^k
    voxels a side, where k is the number of decoder levels (from the top)
    that read the upsampled half of their concatenation before the first
    that reads the skip: all skips give the input itself, level 1 from the
    upsampled half gives 2-blocks, levels 1 and 2 give 4-blocks, all three
    8-blocks.  A pool that summed, grouped the wrong voxels, an upsample
    that shifted, or a concatenation in the other order (skip first) would
    change these outputs."""
    from oracle import unet
    D, H, W = 8, 16, 8
    k, j, i = np.meshgrid(np.arange(D), np.arange(H), np.arange(W), indexing="ij")
    x = (1.0 + 0.03 * k + 0.02 * j + 0.01 * i)[None, ..., None]
    cases = [({1: True, 2: True, 3: True}, 1), ({1: False, 2: True, 3: True}, 2),
             ({1: False, 2: False, 3: True}, 4), ({1: False, 2: False, 3: False}, 8)]
    for dec_from_skip, s in cases:
        y = unet.forward(passthrough_theta(dec_from_skip), x)
        assert np.allclose(y[0, ..., 0], block_centre_ramp(D, H, W, s), rtol=0, atol=1e-13), s
