"""The learned warm start's network kernels (tcgen05 implicit-GEMM 3x3x3 convolution,
its data and weight gradients, pooling, upsampling with concatenation, the 1x1x1 head,
MSE and Adam) against the FP64 network oracle, through the C ABI.

Inputs and weights are drawn, rounded to bf16, and the oracle runs in FP64 on the
rounded values. Tolerances: a bf16 output carries 8 significant bits (relative rounding
2^-9), so bf16 results are held to 1e-2 of the field's maximum; FP32 results (weight and
bias gradients, head, loss) accumulated from bf16 operands to 1e-3. The whole network
(14 convolutions with bf16 activations between them) is compared by relative norm."""
import numpy as np
import pytest

from oracle import surrogate as S

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _net():
    from paper_1804_07588_gb300 import net
    return net


def bf16_round(a):
    """FP64 array rounded to bf16 values (round to nearest even), as FP64."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def to_dev(a_ndhwc, dtype="bf16"):
    torch = _torch()
    t = torch.tensor(np.ascontiguousarray(a_ndhwc), dtype=torch.float32, device="cuda")
    return t.to(torch.bfloat16) if dtype == "bf16" else t


def ora_layout(x_ndhwc):
    """[N, D, H, W, C] -> list of [C, D, H, W]"""
    return [np.ascontiguousarray(x.transpose(3, 0, 1, 2)) for x in x_ndhwc]


def ndhwc(xs):
    return np.stack([x.transpose(1, 2, 3, 0) for x in xs])


def w_dev(w_ora):
    """[o][c][3][3][3] -> bf16 [o][27][c]"""
    torch = _torch()
    a = w_ora.reshape(w_ora.shape[0], w_ora.shape[1], 27).transpose(0, 2, 1)
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda").to(torch.bfloat16)


def rel_max(a, b):
    return float(np.abs(np.asarray(a, np.float64) - b).max() / max(np.abs(b).max(), 1e-30))


SHAPE = (2, 8, 8, 16)  # N, D, H, W


# H = 16: the halo-staged kernel (output tiles 8 x 16 x 1); H = 8: the per-tap kernel
SHAPE_HALO = (1, 4, 16, 16)


@pytest.mark.parametrize("shape", [SHAPE, SHAPE_HALO])
@pytest.mark.parametrize("c0, c1, cout", [(16, 0, 16), (16, 0, 32), (64, 0, 64), (32, 16, 16), (64, 32, 128),
                                          (64, 64, 64), (16, 0, 48), (32, 64, 96)])
def test_conv3_forward(c0, c1, cout, shape):
    net = _net()
    rng = np.random.default_rng(c0 * 7 + c1 + cout)
    N, D, H, W = shape
    x = bf16_round(rng.normal(size=(N, D, H, W, c0 + c1)))
    w = bf16_round(rng.normal(size=(cout, c0 + c1, 3, 3, 3)) / np.sqrt(27 * (c0 + c1)))
    b = rng.normal(size=cout) * 0.1
    torch = _torch()
    xd = to_dev(x)
    x0 = xd[..., :c0].contiguous()
    x1 = xd[..., c0:].contiguous() if c1 else None
    y = net.conv3_fwd(x0, w_dev(w), torch.tensor(b, dtype=torch.float32, device="cuda"), relu=False, x1=x1)
    net.check()
    ref = ndhwc([S.conv3(xs, w, b) for xs in ora_layout(x)])
    err = rel_max(y.float().cpu().numpy(), ref)
    assert err <= 1e-2, err
    # ReLU and a ReLU-backward mask in the epilogue
    mask = to_dev(rng.normal(size=(N, D, H, W, cout)))
    y2 = net.conv3_fwd(x0, w_dev(w), torch.tensor(b, dtype=torch.float32, device="cuda"), relu=True, x1=x1,
                       mask=mask)
    ref2 = np.maximum(ref, 0) * (mask.float().cpu().numpy() > 0)
    assert rel_max(y2.float().cpu().numpy(), ref2) <= 1e-2


@pytest.mark.parametrize("shape", [SHAPE, SHAPE_HALO])
@pytest.mark.parametrize("cin, cout", [(16, 16), (48, 16), (32, 64), (128, 64), (96, 32)])
def test_conv3_data_gradient(cin, cout, shape):
    """The input gradient (the forward kernel with flipped, transposed weights) against
    the oracle's adjoint."""
    net = _net()
    rng = np.random.default_rng(cin + 3 * cout)
    N, D, H, W = shape
    x = rng.normal(size=(N, D, H, W, cin))
    w = bf16_round(rng.normal(size=(cout, cin, 3, 3, 3)) / np.sqrt(27 * cin))
    gy = bf16_round(rng.normal(size=(N, D, H, W, cout)))
    gx = net.conv3_dgrad(to_dev(gy), net.flip_weights(w_dev(w)))
    net.check()
    ref = ndhwc([S.conv3_backward(xs, w, g)[0] for xs, g in zip(ora_layout(x), ora_layout(gy))])
    assert rel_max(gx.float().cpu().numpy(), ref) <= 1e-2


@pytest.mark.parametrize("shape", [SHAPE, SHAPE_HALO])
@pytest.mark.parametrize("c0, c1, cout", [(16, 0, 16), (16, 0, 32), (64, 0, 64), (32, 16, 16), (64, 64, 64),
                                          (32, 0, 128), (48, 0, 8)])
def test_conv3_weight_gradient(c0, c1, cout, shape):
    net = _net()
    rng = np.random.default_rng(100 + c0 + c1 + cout)
    N, D, H, W = shape
    x = bf16_round(rng.normal(size=(N, D, H, W, c0 + c1)))
    gy = bf16_round(rng.normal(size=(N, D, H, W, cout)))
    w = np.zeros((cout, c0 + c1, 3, 3, 3))
    xd = to_dev(x)
    x0 = xd[..., :c0].contiguous()
    x1 = xd[..., c0:].contiguous() if c1 else None
    gw, gb = net.conv3_wgrad(x0, to_dev(gy), x1=x1)
    net.check()
    gw_ref = sum(S.conv3_backward(xs, w, g)[1] for xs, g in zip(ora_layout(x), ora_layout(gy)))
    gb_ref = gy.sum(axis=(0, 1, 2, 3))
    gw_gpu = gw.cpu().numpy().transpose(0, 2, 1).reshape(cout, c0 + c1, 3, 3, 3)
    assert rel_max(gw_gpu, gw_ref) <= 1e-3
    assert rel_max(gb.cpu().numpy(), gb_ref) <= 1e-3


def test_pool_upsample_concat_and_gradients():
    net = _net()
    torch = _torch()
    rng = np.random.default_rng(7)
    N, D, H, W = SHAPE
    x = bf16_round(rng.normal(size=(N, D, H, W, 16)))
    y = net.avgpool2(to_dev(x))
    ref = ndhwc([S.avgpool2(xs) for xs in ora_layout(x)])
    assert rel_max(y.float().cpu().numpy(), ref) <= 1e-2
    gy = bf16_round(rng.normal(size=ref.shape))
    mask = rng.normal(size=x.shape)
    gx = net.avgpool2_bwd(to_dev(gy), x.shape, mask=to_dev(mask))
    ref = ndhwc([S.avgpool2_backward(g) for g in ora_layout(gy)]) * (bf16_round(mask) > 0)
    assert rel_max(gx.float().cpu().numpy(), ref) <= 1e-2
    # decoder input and its gradient
    h = bf16_round(rng.normal(size=(N, D // 2, H // 2, W // 2, 32)))
    skip = bf16_round(rng.normal(size=(N, D, H, W, 16)))
    cat = net.up2cat(to_dev(h), to_dev(skip))
    ref = np.concatenate([ndhwc([S.up2(a) for a in ora_layout(h)]), skip], axis=-1)
    assert rel_max(cat.float().cpu().numpy(), ref) <= 1e-2
    g = bf16_round(rng.normal(size=ref.shape))
    mh = rng.normal(size=h.shape)
    ms = rng.normal(size=skip.shape)
    gskip = torch.zeros((N, D, H, W, 16), dtype=torch.bfloat16, device="cuda")
    gh = net.up2cat_bwd(to_dev(g), 32, to_dev(mh), gskip, to_dev(ms))
    ref_h = ndhwc([S.up2_backward(a) for a in ora_layout(g[..., :32])]) * (bf16_round(mh) > 0)
    ref_s = g[..., 32:] * (bf16_round(ms) > 0)
    assert rel_max(gh.float().cpu().numpy(), ref_h) <= 1e-2
    assert rel_max(gskip.float().cpu().numpy(), ref_s) <= 1e-2


def test_head_mse_and_adam():
    net = _net()
    torch = _torch()
    rng = np.random.default_rng(8)
    N, D, H, W = SHAPE
    h = bf16_round(np.abs(rng.normal(size=(N, D, H, W, 16))) * (rng.random((N, D, H, W, 16)) > 0.3))
    w = rng.normal(size=(9, 16))
    b = rng.normal(size=9)
    wd = torch.tensor(w, dtype=torch.float32, device="cuda")
    bd = torch.tensor(b, dtype=torch.float32, device="cuda")
    y = net.conv1(to_dev(h), wd, bd)
    ref = ndhwc([S.conv1(a, w, b) for a in ora_layout(h)])
    assert rel_max(y.cpu().numpy(), ref) <= 1e-5
    t = rng.normal(size=ref.shape)
    wgt = (rng.random((N, D, H, W)) > 0.4).astype(np.float64)
    loss, gy = net.mse(y, to_dev(t, "f32"), to_dev(wgt, "f32"))
    l_ref, g_ref = zip(*[S.mse(a, b_, c) for a, b_, c in zip(ora_layout(ref), ora_layout(t), wgt)])
    # the oracle's mean is per sample; the kernel's over the whole batch
    assert abs(float(loss) - np.mean(l_ref)) <= 1e-5 * np.mean(l_ref)
    assert rel_max(gy.cpu().numpy(), ndhwc(list(g_ref)) / N) <= 1e-5
    gh, gw, gb = net.conv1_bwd(gy, wd, to_dev(h))
    refs = [S.conv1_backward(a, w, g) for a, g in zip(ora_layout(h), ora_layout(gy.cpu().numpy()))]
    assert rel_max(gh.float().cpu().numpy(), ndhwc([r[0] for r in refs]) * (h > 0)) <= 1e-2
    assert rel_max(gw.cpu().numpy(), sum(r[1] for r in refs)) <= 1e-4
    assert rel_max(gb.cpu().numpy(), sum(r[2] for r in refs)) <= 1e-4
    # Adam: three steps against the oracle's update
    p = {"a": rng.normal(size=(37,))}
    st = S.adam_init(p)
    pd = torch.tensor(p["a"], dtype=torch.float32, device="cuda")
    m = torch.zeros_like(pd)
    v = torch.zeros_like(pd)
    for step in range(1, 4):
        g = {"a": rng.normal(size=37)}
        S.adam_step(p, g, st, lr=1e-2)
        net.adam_(pd, torch.tensor(g["a"], dtype=torch.float32, device="cuda"), m, v, step, lr=1e-2)
    assert rel_max(pd.cpu().numpy(), p["a"]) <= 1e-5


def test_unet_forward_and_gradients_match_the_oracle():
    """A 4-level U-Net (16, 32, 64, 64 channels; the warm start's architecture) on one
    32 x 32 x 64 volume (the coarsest level holds one 4 x 4 x 8 tile): output and every
    parameter gradient of the MSE against the FP64 oracle, by relative norm."""
    net = _net()
    torch = _torch()
    channels = [16, 32, 64, 64]
    c_out = 9
    params = S.init_params(16, c_out, channels, seed=11)
    for k in params:
        if k.endswith(".w") and params[k].ndim == 5:
            params[k] = bf16_round(params[k])
    model = net.UNet(params, channels, c_out)
    rng = np.random.default_rng(12)
    N, D, H, W = 1, 32, 32, 64
    x = bf16_round(rng.normal(size=(N, D, H, W, 16)))
    t = rng.normal(size=(N, D, H, W, c_out))
    y = model.forward(to_dev(x))
    loss, gy = net.mse(y, to_dev(t, "f32"))
    g = model.backward(gy)
    net.check()
    y_ref, grads = [], None
    for n in range(N):
        yo, cache = S.forward(params, ora_layout(x[n:n + 1])[0], channels)
        y_ref.append(yo)
        _, go = S.mse(yo, ora_layout(t[n:n + 1])[0])
        gp, _ = S.backward(params, cache, go / N, channels)
        grads = gp if grads is None else {k: grads[k] + gp[k] for k in gp}
    y_ref = ndhwc(y_ref)
    ry = np.linalg.norm(y.cpu().numpy() - y_ref) / np.linalg.norm(y_ref)
    assert ry <= 3e-2, ry
    gnp = {}
    for k, v in g.items():
        a = v.cpu().numpy()
        if a.ndim == 3:
            a = a.transpose(0, 2, 1).reshape(a.shape[0], a.shape[2], 3, 3, 3)
        gnp[k] = a
    worst = max(np.linalg.norm(gnp[k] - grads[k]) / max(np.linalg.norm(grads[k]), 1e-30) for k in grads)
    assert worst <= 8e-2, {k: float(np.linalg.norm(gnp[k] - grads[k]) / np.linalg.norm(grads[k])) for k in grads}
