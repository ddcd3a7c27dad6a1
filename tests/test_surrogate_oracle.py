"""Pins of the FP64 oracle of the learned warm start's network (a 3D U-Net): each layer
against an independent definition (a library correlation, the adjoint identity of the
linear layers) and the whole network's gradients against central finite differences."""
import numpy as np
import pytest

from oracle import surrogate as S

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv3_matches_library_correlation():
    """conv3 is the zero-padded same-size cross-correlation summed over input channels
    plus the bias (scipy.signal.correlate, mode "same")."""
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 5, 6, 7))
    w = rng.normal(size=(4, 3, 3, 3, 3))
    b = rng.normal(size=4)
    y = S.conv3(x, w, b)
    ref = np.stack([b[o] + sum(scipy_signal.correlate(x[c], w[o, c], mode="same") for c in range(3))
                    for o in range(4)])
    np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-12)


def _dot(a, b):
    return float(np.sum(a * b))


def test_linear_layers_adjoint():
    """<L x, y> = <x, L^T y> for the input gradient of conv3 and conv1 and for the
    pooling / upsampling pair (L^T of avgpool2 is up2 / 8); the weight gradient of conv3
    is the derivative of the bilinear form in w."""
    rng = np.random.default_rng(2)
    x = rng.normal(size=(3, 4, 6, 8))
    w = rng.normal(size=(5, 3, 3, 3, 3))
    gy = rng.normal(size=(5, 4, 6, 8))
    zero = np.zeros(5)
    gx, gw, gb = S.conv3_backward(x, w, gy)
    assert abs(_dot(S.conv3(x, w, zero), gy) - _dot(x, gx)) <= 1e-10 * abs(_dot(x, gx))
    w2 = rng.normal(size=w.shape)
    assert abs(_dot(S.conv3(x, w2, zero), gy) - _dot(w2, gw)) <= 1e-10 * abs(_dot(w2, gw))
    assert np.allclose(gb, gy.sum(axis=(1, 2, 3)))
    w1 = rng.normal(size=(5, 3))
    gx1, gw1, _ = S.conv1_backward(x, w1, gy)
    assert abs(_dot(S.conv1(x, w1, zero), gy) - _dot(x, gx1)) <= 1e-10 * abs(_dot(x, gx1))
    yp = rng.normal(size=(3, 2, 3, 4))
    assert abs(_dot(S.avgpool2(x), yp) - _dot(x, S.avgpool2_backward(yp))) <= 1e-12
    assert np.allclose(S.avgpool2_backward(yp), S.up2(yp) / 8.0)
    assert abs(_dot(S.up2(yp), x) - _dot(yp, S.up2_backward(x))) <= 1e-10


def test_unet_gradients_match_finite_differences():
    """A 4-level network on an 8^3 volume: the backward pass's gradients of the MSE loss,
    for a sample of weights, biases and input entries in every stage, equal central
    differences."""
    channels = [3, 4, 5, 5]
    c_in, c_out = 4, 3
    p = S.init_params(c_in, c_out, channels, seed=3)
    rng = np.random.default_rng(4)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.normal(0.0, 0.1, p[k].shape)
    x = rng.normal(size=(c_in, 8, 8, 8))
    t = rng.normal(size=(c_out, 8, 8, 8))
    wgt = (rng.random((8, 8, 8)) > 0.3).astype(float)

    def loss(p_, x_):
        y, _ = S.forward(p_, x_, channels)
        return S.mse(y, t, wgt)[0]

    y, cache = S.forward(p, x, channels)
    _, gy = S.mse(y, t, wgt)
    g, gx = S.backward(p, cache, gy, channels)
    assert set(g) == set(p)
    h = 1e-5  # central differences: truncation ~h^2, rounding ~eps L / h
    checked = 0
    for name in sorted(p):
        arr = p[name]
        for flat in rng.choice(arr.size, size=min(3, arr.size), replace=False):
            idx = np.unravel_index(flat, arr.shape)
            old = arr[idx]
            arr[idx] = old + h
            lp = loss(p, x)
            arr[idx] = old - h
            lm = loss(p, x)
            arr[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(fd - g[name][idx]) <= 1e-6 * abs(fd) + 1e-9, (name, idx, fd, g[name][idx])
            checked += 1
    for flat in rng.choice(x.size, size=8, replace=False):
        idx = np.unravel_index(flat, x.shape)
        old = x[idx]
        x[idx] = old + h
        lp = loss(p, x)
        x[idx] = old - h
        lm = loss(p, x)
        x[idx] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - gx[idx]) <= 1e-6 * abs(fd) + 1e-9, (idx, fd, gx[idx])
    assert checked >= 3 * len(p) - 3


def test_network_shapes_and_inputs():
    channels = [16, 32, 48, 64]
    p = S.init_params(8, 9, channels, seed=0)
    mask = np.zeros((16, 16, 16), np.uint8)
    mask[4:8, 4:8, 4:8] = 2
    x = S.inputs(mask, 0.01, 1.0 / 3.0, [0.1, 0.1, 1e-6, 1e-6, 0.8 - 2e-6])
    assert x.shape == (8, 16, 16, 16)
    assert x[0].sum() == 64 and np.all(x[1] == 0.01)
    y, _ = S.forward(p, x, channels)
    assert y.shape == (9, 16, 16, 16) and np.all(np.isfinite(y))
    # 16 -> 64 channels over four levels, the configuration's network
    n_par = sum(v.size for v in p.values())
    assert 100_000 < n_par < 1_000_000


def test_adam_first_step_closed_form():
    """After one step from zero moments the bias-corrected Adam step is -lr g / (|g| + eps)
    for every element (m_hat = g, v_hat = g^2)."""
    rng = np.random.default_rng(5)
    p = {"a": rng.normal(size=(4, 3))}
    p0 = p["a"].copy()
    g = {"a": rng.normal(size=(4, 3))}
    st = S.adam_init(p)
    S.adam_step(p, g, st, lr=0.01)
    np.testing.assert_allclose(p["a"], p0 - 0.01 * g["a"] / (np.abs(g["a"]) + 1e-8), rtol=1e-12)


def test_training_reduces_the_loss():
    """A small network learns a smooth target of the geometry (the solid indicator
    averaged over its 3x3x3 neighbourhood, a stand-in for a field that follows the
    geometry): 150 Adam steps on 4 seeded 8^3 masks cut the loss at least tenfold."""
    rng = np.random.default_rng(6)
    channels = [4, 6, 8]
    p = S.init_params(1, 1, channels, seed=7)
    data = []
    box = np.ones((1, 1, 3, 3, 3)) / 27.0
    for _ in range(4):
        x = (rng.random((1, 8, 8, 8)) > 0.6).astype(float)
        data.append((x, S.conv3(x, box, np.zeros(1))))
    st = S.adam_init(p)

    def total():
        return sum(S.mse(S.forward(p, x, channels)[0], t)[0] for x, t in data) / len(data)

    first = total()
    for it in range(150):
        x, t = data[it % len(data)]
        y, cache = S.forward(p, x, channels)
        _, gy = S.mse(y, t)
        g, _ = S.backward(p, cache, gy, channels)
        S.adam_step(p, g, st, lr=3e-3)
    assert total() < 0.1 * first
