"""FP64 oracle of the learned warm start's network: a 3D convolutional U-Net that maps a
porous geometry and its inlet conditions to steady fields, with the forward pass, the
backward pass (every gradient written out from the layer definitions) and the
mean-squared-error loss.

Test infrastructure only, like the rest of this package: the tests call it to check
the network kernels' outputs and gradients; the product never imports it.

Layers (NCDHW without the batch axis, arrays [channels, z, y, x], FP64):
- conv3: same-size 3x3x3 cross-correlation with zero padding 1 plus a bias,
  y[o] = b[o] + sum_{c, k} w[o, c, k] x[c, . + k - 1];
- conv1: 1x1x1 convolution (the output head), y[o] = b[o] + sum_c w[o, c] x[c];
- relu; avgpool2: mean over 2x2x2 blocks; up2: nearest-neighbour doubling;
- concat along channels (the skip connections).
Network: an encoder of `levels` stages (two conv3 + relu each, avgpool2 between stages)
and a decoder that doubles the resolution, concatenates the encoder stage of the same
size and applies two conv3 + relu, then conv1 to the output channels.
"""
import numpy as np

# --- layers -------------------------------------------------------------------------


def _pad1(x):
    C, D, H, W = x.shape
    xp = np.zeros((C, D + 2, H + 2, W + 2))
    xp[:, 1:-1, 1:-1, 1:-1] = x
    return xp


def conv3(x, w, b):
    """y[o, z, y, x] = b[o] + sum_{c, dz, dy, dx} w[o, c, dz, dy, dx] x[c, z+dz-1, y+dy-1, x+dx-1]
    with x zero outside the volume."""
    C, D, H, W = x.shape
    xp = _pad1(x)
    y = np.empty((w.shape[0], D, H, W))
    y[:] = b[:, None, None, None]
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                y += np.einsum("oc,czyx->ozyx", w[:, :, dz, dy, dx], xp[:, dz:dz + D, dy:dy + H, dx:dx + W])
    return y


def conv3_backward(x, w, gy):
    """Gradients of conv3 for the output gradient gy: the input gradient is the adjoint
    (each output's gradient sent back through the 27 taps it read), the weight gradient
    correlates gy with the shifted inputs, the bias gradient sums gy."""
    C, D, H, W = x.shape
    xp = _pad1(x)
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                xs = xp[:, dz:dz + D, dy:dy + H, dx:dx + W]
                gw[:, :, dz, dy, dx] = np.einsum("ozyx,czyx->oc", gy, xs)
                gxp[:, dz:dz + D, dy:dy + H, dx:dx + W] += np.einsum("oc,ozyx->czyx", w[:, :, dz, dy, dx], gy)
    return gxp[:, 1:-1, 1:-1, 1:-1], gw, gy.sum(axis=(1, 2, 3))


def conv1(x, w, b):
    return np.einsum("oc,czyx->ozyx", w, x) + b[:, None, None, None]


def conv1_backward(x, w, gy):
    return np.einsum("oc,ozyx->czyx", w, gy), np.einsum("ozyx,czyx->oc", gy, x), gy.sum(axis=(1, 2, 3))


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(x, gy):
    return gy * (x > 0.0)


def avgpool2(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def avgpool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(gy):
    C, D, H, W = gy.shape
    return gy.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


# --- network ------------------------------------------------------------------------


def init_params(c_in, c_out, channels, seed):
    """He-normal weights (std sqrt(2 / fan_in)) and zero biases, seeded. Keys: enc{l}a,
    enc{l}b, dec{l}a, dec{l}b for l = 0 .. levels - 1 (decoder stages below the bottom),
    head."""
    rng = np.random.default_rng(seed)
    L = len(channels)
    p = {}

    def conv(name, o, c, k):
        fan = c * k ** 3
        shape = (o, c, 3, 3, 3) if k == 3 else (o, c)
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan), shape)
        p[name + ".b"] = np.zeros(o)

    c = c_in
    for l in range(L):
        conv(f"enc{l}a", channels[l], c, 3)
        conv(f"enc{l}b", channels[l], channels[l], 3)
        c = channels[l]
    for l in range(L - 2, -1, -1):
        conv(f"dec{l}a", channels[l], channels[l + 1] + channels[l], 3)
        conv(f"dec{l}b", channels[l], channels[l], 3)
    conv("head", c_out, channels[0], 1)
    return p


def forward(p, x, channels):
    """Network output and the cache the backward pass needs."""
    L = len(channels)
    cache = {}
    skips = []
    h = x
    for l in range(L):
        if l > 0:
            h = avgpool2(h)
        for s in "ab":
            name = f"enc{l}{s}"
            cache[name] = h
            z = conv3(h, p[name + ".w"], p[name + ".b"])
            cache[name + ".z"] = z
            h = relu(z)
        skips.append(h)
    for l in range(L - 2, -1, -1):
        u = up2(h)
        h = np.concatenate([u, skips[l]], axis=0)
        cache[f"cat{l}"] = u.shape[0]
        for s in "ab":
            name = f"dec{l}{s}"
            cache[name] = h
            z = conv3(h, p[name + ".w"], p[name + ".b"])
            cache[name + ".z"] = z
            h = relu(z)
    cache["head"] = h
    return conv1(h, p["head.w"], p["head.b"]), cache


def mse(y, t, weight=None):
    """Mean over voxels and channels of weight (y - t)^2 (weight broadcast over
    channels, default 1), and its gradient in y."""
    wgt = np.ones(y.shape[1:]) if weight is None else weight
    n = y.shape[0] * wgt.size
    d = y - t
    return float(np.sum(wgt[None] * d * d) / n), 2.0 * wgt[None] * d / n


def backward(p, cache, gy, channels):
    """Gradients of every parameter (dict like p) and of the network input."""
    L = len(channels)
    g = {}
    gh, g["head.w"], g["head.b"] = conv1_backward(cache["head"], p["head.w"], gy)
    gskip = [None] * L
    for l in range(0, L - 1):
        for s in "ba":
            name = f"dec{l}{s}"
            gz = relu_backward(cache[name + ".z"], gh)
            gh, g[name + ".w"], g[name + ".b"] = conv3_backward(cache[name], p[name + ".w"], gz)
        nu = cache[f"cat{l}"]
        gskip[l] = gh[nu:]
        gh = up2_backward(gh[:nu])
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            gh = gh + gskip[l]
        for s in "ba":
            name = f"enc{l}{s}"
            gz = relu_backward(cache[name + ".z"], gh)
            gh, g[name + ".w"], g[name + ".b"] = conv3_backward(cache[name], p[name + ".w"], gz)
        if l > 0:
            gh = avgpool2_backward(gh)
    return g, gh


def inputs(mask, u_in, T_in, X_in):
    """Network input: the solid indicator and the inlet velocity, temperature and mole
    fractions as constant channels, [3 + len(X_in)][z][y][x]."""
    solid = (np.asarray(mask) > 0).astype(np.float64)
    chans = [solid, np.full(solid.shape, float(u_in)), np.full(solid.shape, float(T_in))]
    chans += [np.full(solid.shape, float(x)) for x in X_in]
    return np.stack(chans)


# --- training -----------------------------------------------------------------------


def adam_init(p):
    """Zero first and second moments for every parameter, step count 0."""
    return {"t": 0, "m": {k: np.zeros_like(v) for k, v in p.items()}, "v": {k: np.zeros_like(v) for k, v in p.items()}}


def adam_step(p, g, state, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015) of every parameter in place: moment
    estimates m = beta1 m + (1 - beta1) g and v = beta2 v + (1 - beta2) g^2, bias
    corrected by 1 - beta^t, step -lr m_hat / (sqrt(v_hat) + eps)."""
    state["t"] += 1
    t = state["t"]
    for k in p:
        m = state["m"][k] = beta1 * state["m"][k] + (1.0 - beta1) * g[k]
        v = state["v"][k] = beta2 * state["v"][k] + (1.0 - beta2) * g[k] * g[k]
        mh = m / (1.0 - beta1 ** t)
        vh = v / (1.0 - beta2 ** t)
        p[k] -= lr * mh / (np.sqrt(vh) + eps)
