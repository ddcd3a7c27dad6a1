"""Python binding of the learned warm start's network kernels (``include/fdlbm_net.h``)
and the U-Net that sequences them.

The layer functions marshal torch CUDA tensors into the C ABI (device pointers, sizes,
the current stream); every arithmetic step runs in the library's kernels. ``UNet``
holds the parameters (FP32 masters with bf16 copies for the tensor cores), runs the
forward pass keeping the activations the backward pass needs, the backward pass and
Adam steps. Architecture (matching the network oracle): an encoder of L stages of two
3x3x3 convolutions + ReLU with 2x2x2 average pooling between stages, a decoder that
upsamples (nearest), concatenates the encoder stage of the same size and applies two
convolutions + ReLU, and a 1x1x1 head. The input has 16 channels (solid indicator, inlet
velocity, temperature and mole fractions, zero-padded); the output the steady fields.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from .fdlbm import FdlbmError, load

_bound = False


def lib():
    global _bound
    L = load()
    if not _bound:
        vp, i, ll, f = C.c_void_p, C.c_int, C.c_longlong, C.c_float
        L.fdlbm_net_last_error.restype = C.c_char_p
        L.fdlbm_net_check.argtypes = [vp]
        L.fdlbm_conv3_fwd.argtypes = [vp, i, vp, i, i, i, i, i, vp, vp, i, i, vp, vp, vp]
        L.fdlbm_conv3_flip_weights.argtypes = [vp, i, i, vp, vp]
        L.fdlbm_conv3_wgrad.argtypes = [vp, i, vp, i, i, i, i, i, vp, i, vp, vp, vp]
        L.fdlbm_net_avgpool2.argtypes = [vp, i, i, i, i, i, vp, vp]
        L.fdlbm_net_avgpool2_bwd.argtypes = [vp, i, i, i, i, i, vp, vp, vp]
        L.fdlbm_net_up2cat.argtypes = [vp, i, vp, i, i, i, i, i, vp, vp]
        L.fdlbm_net_up2cat_bwd.argtypes = [vp, i, i, i, i, i, i, vp, vp, vp, vp, vp]
        L.fdlbm_net_add.argtypes = [vp, vp, ll, vp]
        L.fdlbm_net_conv1.argtypes = [vp, i, vp, vp, i, ll, vp, vp]
        L.fdlbm_net_conv1_bwd.argtypes = [vp, i, vp, i, vp, ll, vp, vp, vp, vp]
        L.fdlbm_net_mse.argtypes = [vp, vp, vp, i, ll, vp, vp, vp]
        L.fdlbm_net_adam.argtypes = [vp, vp, vp, vp, ll, i, f, f, f, f, vp, vp]
        L.fdlbm_net_to_bf16.argtypes = [vp, ll, vp, vp]
        for name in ("fdlbm_net_check", "fdlbm_conv3_fwd", "fdlbm_conv3_flip_weights", "fdlbm_conv3_wgrad",
                     "fdlbm_net_avgpool2", "fdlbm_net_avgpool2_bwd", "fdlbm_net_up2cat", "fdlbm_net_up2cat_bwd",
                     "fdlbm_net_add", "fdlbm_net_conv1", "fdlbm_net_conv1_bwd", "fdlbm_net_mse", "fdlbm_net_adam",
                     "fdlbm_net_to_bf16"):
            getattr(L, name).restype = C.c_int
        _bound = True
    return L


def _chk(status):
    if status != 0:
        raise FdlbmError(status, lib().fdlbm_net_last_error().decode())


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def check():
    """Wait for the stream; raise if a convolution's pipeline timed out."""
    _chk(lib().fdlbm_net_check(_stream()))


# ---- layers (NDHWC bf16 activations: shape [N, D, H, W, C]) -----------------------------

def conv3_fwd(x0, w, bias=None, relu=False, x1=None, mask=None, out=None):
    import torch
    N, D, H, W, c0 = x0.shape
    c1 = 0 if x1 is None else x1.shape[-1]
    cout = w.shape[0]
    if out is None:
        out = torch.empty((N, D, H, W, cout), dtype=torch.bfloat16, device=x0.device)
    _chk(lib().fdlbm_conv3_fwd(_p(x0), c0, _p(x1), c1, N, D, H, W, _p(w), _p(bias), cout, int(relu), _p(mask),
                               _p(out), _stream()))
    return out


def flip_weights(w, out=None):
    import torch
    cout, _, cin = w.shape
    if out is None:
        out = torch.empty((cin, 27, cout), dtype=torch.bfloat16, device=w.device)
    _chk(lib().fdlbm_conv3_flip_weights(_p(w), cout, cin, _p(out), _stream()))
    return out


def conv3_dgrad(gy, wflip, mask=None, out=None):
    """Input gradient of a 3x3x3 convolution, given the flipped weights and the output
    gradient; mask: the input activation (ReLU backward of the layer that produced it)."""
    return conv3_fwd(gy, wflip, None, False, None, mask, out)


def conv3_wgrad(x0, gy, x1=None, gw=None, gb=None):
    import torch
    N, D, H, W, c0 = x0.shape
    c1 = 0 if x1 is None else x1.shape[-1]
    cout = gy.shape[-1]
    if gw is None:
        gw = torch.empty((cout, 27, c0 + c1), dtype=torch.float32, device=x0.device)
    if gb is None:
        gb = torch.empty(cout, dtype=torch.float32, device=x0.device)
    _chk(lib().fdlbm_conv3_wgrad(_p(x0), c0, _p(x1), c1, N, D, H, W, _p(gy), cout, _p(gw), _p(gb), _stream()))
    return gw, gb


def avgpool2(x):
    import torch
    N, D, H, W, c = x.shape
    y = torch.empty((N, D // 2, H // 2, W // 2, c), dtype=torch.bfloat16, device=x.device)
    _chk(lib().fdlbm_net_avgpool2(_p(x), c, N, D, H, W, _p(y), _stream()))
    return y


def avgpool2_bwd(gy, fine_shape, mask=None):
    import torch
    N, D, H, W, c = fine_shape
    gx = torch.empty(fine_shape, dtype=torch.bfloat16, device=gy.device)
    _chk(lib().fdlbm_net_avgpool2_bwd(_p(gy), c, N, D, H, W, _p(mask), _p(gx), _stream()))
    return gx


def up2cat(h, skip):
    import torch
    N, D, H, W, cs = skip.shape
    cu = h.shape[-1]
    out = torch.empty((N, D, H, W, cu + cs), dtype=torch.bfloat16, device=h.device)
    _chk(lib().fdlbm_net_up2cat(_p(h), cu, _p(skip), cs, N, D, H, W, _p(out), _stream()))
    return out


def up2cat_bwd(g, cu, mask_h, gskip, mask_skip=None):
    """(gradient of the coarse input, masked by mask_h); gskip accumulates the skip part."""
    import torch
    N, D, H, W, c = g.shape
    gh = torch.empty((N, D // 2, H // 2, W // 2, cu), dtype=torch.bfloat16, device=g.device)
    _chk(lib().fdlbm_net_up2cat_bwd(_p(g), cu, c - cu, N, D, H, W, _p(mask_h), _p(gh), _p(mask_skip), _p(gskip),
                                    _stream()))
    return gh


def add_(dst, src):
    _chk(lib().fdlbm_net_add(_p(dst), _p(src), dst.numel(), _stream()))
    return dst


def conv1(h, w, b):
    import torch
    N, D, H, W, c = h.shape
    cout = w.shape[0]
    y = torch.empty((N, D, H, W, cout), dtype=torch.float32, device=h.device)
    _chk(lib().fdlbm_net_conv1(_p(h), c, _p(w), _p(b), cout, N * D * H * W, _p(y), _stream()))
    return y


def conv1_bwd(gy, w, h):
    import torch
    N, D, H, W, c = h.shape
    cout = w.shape[0]
    gh = torch.empty_like(h)
    gw = torch.empty_like(w)
    gb = torch.empty(cout, dtype=torch.float32, device=h.device)
    _chk(lib().fdlbm_net_conv1_bwd(_p(gy), cout, _p(w), c, _p(h), N * D * H * W, _p(gh), _p(gw), _p(gb), _stream()))
    return gh, gw, gb


def mse(y, t, wgt=None):
    """(loss as a 0-d FP64 CUDA tensor, gradient in y)."""
    import torch
    cout = y.shape[-1]
    nvox = y.numel() // cout
    loss = torch.empty((), dtype=torch.float64, device=y.device)
    gy = torch.empty_like(y)
    _chk(lib().fdlbm_net_mse(_p(y), _p(t), _p(wgt), cout, nvox, _p(loss), _p(gy), _stream()))
    return loss, gy


def adam_(p, g, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, p_bf16=None):
    _chk(lib().fdlbm_net_adam(_p(p), _p(g), _p(m), _p(v), p.numel(), int(t), lr, b1, b2, eps, _p(p_bf16), _stream()))


def to_bf16(x, out=None):
    import torch
    if out is None:
        out = torch.empty(x.shape, dtype=torch.bfloat16, device=x.device)
    _chk(lib().fdlbm_net_to_bf16(_p(x), x.numel(), _p(out), _stream()))
    return out


# ---- the network ---------------------------------------------------------------------

IN_CHANNELS = 16


class UNet:
    """U-Net with `channels` per level (multiples of 16), IN_CHANNELS inputs and c_out
    outputs; parameters from a dict in the network oracle's layout (w[o][c][dz][dy][dx]
    FP64 numpy arrays) or He-normal from the oracle's initialiser convention."""

    def __init__(self, params: dict, channels, c_out: int, device="cuda"):
        import torch
        self.channels = list(channels)
        self.c_out = c_out
        self.device = device
        self.names = []
        self.p32, self.p16 = {}, {}
        for k, v in params.items():
            a = np.asarray(v, np.float64)
            if k.endswith(".w") and a.ndim == 5:  # [o][c][3][3][3] -> [o][27][c]
                a = a.reshape(a.shape[0], a.shape[1], 27).transpose(0, 2, 1)
            t = torch.tensor(np.ascontiguousarray(a), dtype=torch.float32, device=device)
            self.p32[k] = t
            if k.endswith(".w") and t.dim() == 3:
                self.p16[k] = to_bf16(t)
            self.names.append(k)
        self.m = {k: torch.zeros_like(v) for k, v in self.p32.items()}
        self.v = {k: torch.zeros_like(v) for k, v in self.p32.items()}
        self.t = 0

    def forward(self, x):
        """x: [N, D, H, W, 16] bf16 -> [N, D, H, W, c_out] float32; keeps activations."""
        L = len(self.channels)
        acts = {}
        skips = []
        h = x
        for l in range(L):
            if l > 0:
                h = avgpool2(h)
            for s in "ab":
                name = f"enc{l}{s}"
                acts[name] = h
                h = conv3_fwd(h, self.p16[name + ".w"], self.p32[name + ".b"], relu=True)
                acts[name + ".y"] = h
            skips.append(h)
        for l in range(L - 2, -1, -1):
            name = f"dec{l}a"
            acts[name] = (h, skips[l])
            # the convolution reads the concatenation [up2(h), skip] from its two sources
            h = conv3_fwd(up2_only(h, skips[l].shape), self.p16[name + ".w"], self.p32[name + ".b"], relu=True,
                          x1=skips[l])
            acts[name + ".y"] = h
            name = f"dec{l}b"
            acts[name] = h
            h = conv3_fwd(h, self.p16[name + ".w"], self.p32[name + ".b"], relu=True)
            acts[name + ".y"] = h
        acts["head"] = h
        self.acts = acts
        self.skips = skips
        return conv1(h, self.p32["head.w"], self.p32["head.b"])

    def backward(self, gy):
        """Gradients of every parameter (FP32) for the output gradient gy."""
        import torch
        L = len(self.channels)
        acts = self.acts
        g = {}
        gh, g["head.w"], g["head.b"] = conv1_bwd(gy, self.p32["head.w"], acts["head"])
        gskip = [None] * L
        for l in range(0, L - 1):
            # dec{l}b: input is dec{l}a's ReLU output
            name = f"dec{l}b"
            g[name + ".w"], g[name + ".b"] = conv3_wgrad(acts[name], gh)
            gh = conv3_dgrad(gh, flip_weights(self.p16[name + ".w"]), mask=acts[name])
            # dec{l}a: input is [up2(h_coarse), skip_l]
            name = f"dec{l}a"
            hc, skip = acts[name]
            up = up2_only(hc, skip.shape)
            g[name + ".w"], g[name + ".b"] = conv3_wgrad(up, gh, x1=skip)
            gcat = conv3_dgrad(gh, flip_weights(self.p16[name + ".w"]))
            gskip[l] = torch.zeros_like(skip)
            gh = up2cat_bwd(gcat, hc.shape[-1], hc, gskip[l], skip)
        for l in range(L - 1, -1, -1):
            if l < L - 1:
                add_(gh, gskip[l])
            for s in "ba":
                name = f"enc{l}{s}"
                g[name + ".w"], g[name + ".b"] = conv3_wgrad(acts[name], gh)
                if s == "b":
                    gh = conv3_dgrad(gh, flip_weights(self.p16[name + ".w"]), mask=acts[name])
                elif l > 0:
                    gh = conv3_dgrad(gh, flip_weights(self.p16[name + ".w"]))
            if l > 0:
                # through the pooling into the previous stage's output (a ReLU output)
                gh = avgpool2_bwd(gh, self.skips[l - 1].shape, mask=self.skips[l - 1])
        return g

    def adam_step(self, g, lr=1e-3):
        self.t += 1
        for k in self.names:
            adam_(self.p32[k], g[k], self.m[k], self.v[k], self.t, lr, p_bf16=self.p16.get(k))

    def params_numpy(self) -> dict:
        """Parameters in the network oracle's layout (FP64 numpy)."""
        out = {}
        for k, t in self.p32.items():
            a = t.detach().double().cpu().numpy()
            if a.ndim == 3:  # [o][27][c] -> [o][c][3][3][3]
                a = a.transpose(0, 2, 1).reshape(a.shape[0], a.shape[2], 3, 3, 3)
            out[k] = a
        return out


def up2_only(h, fine_shape):
    """Nearest upsampling of h to the fine grid of fine_shape (up2cat without a skip)."""
    import torch
    N, D, H, W, _ = fine_shape
    cu = h.shape[-1]
    out = torch.empty((N, D, H, W, cu), dtype=torch.bfloat16, device=h.device)
    _chk(lib().fdlbm_net_up2cat(_p(h), cu, None, 0, N, D, H, W, _p(out), _stream()))
    return out


def _profile_main():
    """Training iterations of the warm start's U-Net on a random batch (a fixed workload for
    timing and profiling the network kernels): python -m paper_1804_07588_gb300.net
    [--batch N] [--iters K]; prints the mean time per iteration."""
    import argparse
    import time

    import numpy as np
    import torch

    from . import warmstart as WS
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--iters", type=int, default=5)
    args = ap.parse_args()
    nx, ny, nz = WS.SHAPE
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(size=(args.batch, nz, ny, nx, 16)), dtype=torch.float32, device="cuda")
    x = x.to(torch.bfloat16)
    t = torch.tensor(rng.normal(size=(args.batch, nz, ny, nx, WS.N_OUT)), dtype=torch.float32, device="cuda")
    model = WS.new_model(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.iters):
        y = model.forward(x)
        loss, gy = mse(y, t)
        model.adam_step(model.backward(gy), lr=1e-3)
    check()
    torch.cuda.synchronize()
    print(f"{(time.perf_counter() - t0) / args.iters * 1e3:.2f} ms per training iteration "
          f"(batch {args.batch}, {nx}x{ny}x{nz})")


if __name__ == "__main__":
    _profile_main()
