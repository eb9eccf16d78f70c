"""3-D U-Net for the learned pressure guess -- TEST INFRASTRUCTURE ONLY.

Plain FP64 numpy definition of the network the CUDA path runs in BF16, used
to check its forward pass, its gradients and one optimiser step.  It shares
no code with the CUDA library.

Network (channels-last tensors [N][D][H][W][C], D = z, H = y, W = x):
  encoder  level l = 1..4 with C_l = 16, 32, 64, 128:
             e_l = relu(conv(relu(conv(in_l))))          in_1 = input (1 channel)
             in_{l+1} = avgpool2(e_l)                    (2x2x2 mean)
  decoder  level l = 3, 2, 1:
             u_l = concat(upsample2(d_{l+1}), e_l)       (d_4 = e_4; nearest x2)
             d_l = relu(conv(relu(conv(u_l))))           C_l output channels
  output   y = conv1x1(d_1) + bias                       (1 channel, linear)
conv = 3x3x3 cross-correlation with bias, periodic in x and y, zero outside
the walls in z: y[v][o] = b[o] + sum_{c,t} W[o][c][t] x[v + off(t)][c],
tap t = (kz*3 + ky)*3 + kx with offset (kz-1, ky-1, kx-1).

Parameters are one flat FP64 vector, layer by layer (weights [o][c][27]
then bias [o]); `layer_specs` gives the order.
"""
import numpy as np

CH = (16, 32, 64, 128)


def layer_specs():
    """(name, c_in, c_out, taps) in parameter order."""
    s = []
    cin = 1
    for l, c in enumerate(CH):
        s.append(("enc%d_a" % (l + 1), cin, c, 27))
        s.append(("enc%d_b" % (l + 1), c, c, 27))
        cin = c
    for l in (2, 1, 0):
        cu = CH[l + 1] + CH[l]
        s.append(("dec%d_a" % (l + 1), cu, CH[l], 27))
        s.append(("dec%d_b" % (l + 1), CH[l], CH[l], 27))
    s.append(("out", CH[0], 1, 1))
    return s


def n_params():
    return sum(co * ci * t + co for (_, ci, co, t) in layer_specs())


def unpack(theta):
    out, q = {}, 0
    for (name, ci, co, t) in layer_specs():
        w = theta[q:q + co * ci * t].reshape(co, ci, t)
        q += co * ci * t
        b = theta[q:q + co]
        q += co
        out[name] = (w, b)
    return out


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.
    Used to state the CUDA path's storage points exactly: its activations,
    weights and activation gradients are stored in bfloat16."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def ident(a):
    return a


def init_params(seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero bias; small output layer."""
    rng = np.random.default_rng(seed)
    parts = []
    for (name, ci, co, t) in layer_specs():
        std = np.sqrt(2.0 / (ci * t)) if name != "out" else 0.1 / np.sqrt(ci)
        parts.append(rng.standard_normal(co * ci * t) * std)
        parts.append(np.zeros(co))
    return np.concatenate(parts)


# ---------------------------------------------------------------- primitives

def shift(x, t):
    """x shifted so that out[v] = x[v + off(t)] (periodic y, x; zero in z)."""
    kz, ky, kx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
    y = np.roll(x, shift=(-ky, -kx), axis=(2, 3))
    out = np.zeros_like(y)
    D = x.shape[1]
    if kz == 0:
        out[:] = y
    elif kz == 1:
        out[:, :D - 1] = y[:, 1:]
    else:
        out[:, 1:] = y[:, :D - 1]
    return out


def shift_adj(g, t):
    """Adjoint of shift: sum_v g[v] * x[v + off] = sum_u shift_adj(g)[u] x[u]."""
    kz, ky, kx = t // 9 - 1, (t // 3) % 3 - 1, t % 3 - 1
    D = g.shape[1]
    out = np.zeros_like(g)
    if kz == 0:
        out[:] = g
    elif kz == 1:
        out[:, 1:] = g[:, :D - 1]
    else:
        out[:, :D - 1] = g[:, 1:]
    return np.roll(out, shift=(ky, kx), axis=(2, 3))


def conv(x, w, b):
    co, ci, taps = w.shape
    y = np.zeros(x.shape[:4] + (co,)) + b
    if taps == 1:
        return y + np.einsum("ndhwc,oc->ndhwo", x, w[:, :, 0])
    for t in range(27):
        y += np.einsum("ndhwc,oc->ndhwo", shift(x, t), w[:, :, t])
    return y


def conv_backward(x, w, gy):
    """(gx, gw, gb) for y = conv(x, w, b)."""
    co, ci, taps = w.shape
    gb = gy.sum(axis=(0, 1, 2, 3))
    gw = np.zeros_like(w)
    if taps == 1:
        gw[:, :, 0] = np.einsum("ndhwo,ndhwc->oc", gy, x)
        return np.einsum("ndhwo,oc->ndhwc", gy, w[:, :, 0]), gw, gb
    gx = np.zeros_like(x)
    for t in range(27):
        gw[:, :, t] = np.einsum("ndhwo,ndhwc->oc", gy, shift(x, t))
        gx += shift_adj(np.einsum("ndhwo,oc->ndhwc", gy, w[:, :, t]), t)
    return gx, gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def pool(x):
    n, d, h, w, c = x.shape
    return x.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4, 6))


def pool_backward(g):
    return np.repeat(np.repeat(np.repeat(g, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def upsample_backward(g):
    n, d, h, w, c = g.shape
    return g.reshape(n, d // 2, 2, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4, 6))


# ---------------------------------------------------------------- network

def forward(theta, x, keep=False, rnd=ident):
    """y = U(x); with keep, also the activations needed for backward.
    rnd is applied where a stored-precision copy is made (identity: exact
    FP64; `bf16`: the CUDA path's storage points)."""
    P = {k: (rnd(w), b) for k, (w, b) in unpack(theta).items()}
    acts = {}
    h = rnd(x)
    skips = []
    for l in range(4):
        a_in = h
        ha = rnd(relu(conv(a_in, *P["enc%d_a" % (l + 1)])))
        e = rnd(relu(conv(ha, *P["enc%d_b" % (l + 1)])))
        acts["enc%d" % (l + 1)] = (a_in, ha, e)
        skips.append(e)
        h = rnd(pool(e)) if l < 3 else e
    d = h
    for l in (2, 1, 0):
        u = np.concatenate([upsample(d), skips[l]], axis=-1)
        ha = rnd(relu(conv(u, *P["dec%d_a" % (l + 1)])))
        d = rnd(relu(conv(ha, *P["dec%d_b" % (l + 1)])))
        acts["dec%d" % (l + 1)] = (u, ha, d)
    y = conv(d, *P["out"])
    acts["out"] = d
    acts["P"] = P
    return (y, acts) if keep else y


def backward(theta, acts, gy, rnd=ident):
    """Gradient of sum(gy * U(x)) with respect to theta (flat vector); rnd
    marks where the CUDA path stores activation gradients."""
    P = acts["P"]
    G = {}
    gd, G["out_w"], G["out_b"] = conv_backward(acts["out"], P["out"][0], gy)
    gd = rnd(gd * (acts["out"] > 0))
    gskip = [None] * 4
    for l in (0, 1, 2):
        u, ha, d = acts["dec%d" % (l + 1)]
        g = gd
        gha, G["dec%d_b_w" % (l + 1)], G["dec%d_b_b" % (l + 1)] = conv_backward(ha, P["dec%d_b" % (l + 1)][0], g)
        g = rnd(gha * (ha > 0))
        gu, G["dec%d_a_w" % (l + 1)], G["dec%d_a_b" % (l + 1)] = conv_backward(u, P["dec%d_a" % (l + 1)][0], g)
        gu = rnd(gu)
        cu = CH[l + 1]
        gskip[l] = gu[..., cu:]
        deeper = acts["dec%d" % (l + 2)][2] if l < 2 else acts["enc4"][2]
        gd = rnd(upsample_backward(gu[..., :cu]) * (deeper > 0))
    gq = None
    for l in (3, 2, 1, 0):
        a_in, ha, e = acts["enc%d" % (l + 1)]
        g = gd if l == 3 else rnd((pool_backward(gq) + gskip[l]) * (e > 0))
        gha, G["enc%d_b_w" % (l + 1)], G["enc%d_b_b" % (l + 1)] = conv_backward(ha, P["enc%d_b" % (l + 1)][0], g)
        g = rnd(gha * (ha > 0))
        gq, G["enc%d_a_w" % (l + 1)], G["enc%d_a_b" % (l + 1)] = conv_backward(a_in, P["enc%d_a" % (l + 1)][0], g)
        gq = rnd(gq)
    parts = []
    for (name, ci, co, t) in layer_specs():
        parts.append(G[name + "_w"].ravel())
        parts.append(G[name + "_b"])
    return np.concatenate(parts)


def mse(y, t):
    """mean((y - t)^2) and its gradient with respect to y."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def loss_and_grad(theta, x, t, rnd=ident):
    y, acts = forward(theta, x, keep=True, rnd=rnd)
    L, gy = mse(y, t)
    return L, backward(theta, acts, gy, rnd=rnd)


def adam_step(theta, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (bias-corrected); step counts from 1."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
