"""The learned warm start (not in the paper): steady fields of porous sphere packings
generated by the D3Q19 solver, a 3D U-Net trained on them with the library's own
tensor-core kernels (``net.UNet``), and the study of what the network's prediction saves
when it is used as the initial state of the solver.

The network maps the geometry and inlet state of an instance to its steady velocity,
mole fractions and temperature (gas temperature on gas nodes, solid temperature on solid
nodes). Its prediction only initialises a solver run (``Solver.set_fields``); the run
then proceeds to the same steady-state residual as a cold start, so the answer is the
solver's, and a prediction that makes the run diverge, or converge later than a cold
start would, is replaced by a cold start (the fallback is reported).

Encoding, per voxel of the instance's lattice (NDHWC, channels last):
- input (16 channels): solid indicator, u_in / 0.03, (T_in - 525 K) / 75 K, the inlet
  mole fractions, zero padding;
- target (9 channels): u / u_in (3 components), (X_j - X_in,j) * X_SCALE on gas nodes (0
  on solid nodes), (T - T_in) / T_SCALE_K with the solid temperature on solid nodes.
"""
from __future__ import annotations

import time

import numpy as np

from . import workloads as W

SHAPE = (64, 32, 32)        # instance lattice (nx, ny, nz): the reduced data set
CHANNELS = (16, 32, 64, 64)  # U-Net channels per level
N_OUT = 9
X_SCALE = 50.0
T_SCALE_K = 10.0


def instances(n: int, seed: int, shape=SHAPE, porosity=(0.45, 0.6), u_inlet=(0.005, 0.03),
              T_inlet_K=(450.0, 600.0), free_cols: int = 6) -> list:
    """n seeded sphere-packing problems (overlapping spheres r ~ U[5, 10], catalytic FD
    solid, plug inlet, periodic in y and z), drawn like the learning instances of the
    128x64x64 set but on `shape`; draws whose gas does not connect inlet and outlet are
    skipped (the next seed is taken)."""
    rng = np.random.default_rng(seed)
    out = []
    k = 0
    nx, ny, nz = shape
    while len(out) < n:
        por = float(rng.uniform(*porosity))
        u = float(rng.uniform(*u_inlet))
        T = float(rng.uniform(*T_inlet_K))
        try:
            mask, _ = W.sphere_mask(nx, ny, nz, por, 5.0, 10.0, seed + k, free_cols=free_cols)
        except ValueError:
            k += 1
            continue
        k += 1
        out.append(W._base(3, nx, ny, nz, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC],
                           u_inlet=u, inlet_profile=W.PLUG, T0_K=T, T_init_K=T, T_inlet_K=T, T_solid_init_K=T,
                           T_outer_K=T))
    return out


def network_input(p: dict) -> np.ndarray:
    """[D, H, W, 16] float32 input of one instance."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    solid = (np.asarray(p["mask"]).reshape(nz, ny, nx) > 0).astype(np.float32)
    x = np.zeros((nz, ny, nx, 16), np.float32)
    x[..., 0] = solid
    x[..., 1] = p["u_inlet"] / 0.03
    x[..., 2] = (p["T_inlet_K"] - 525.0) / 75.0
    for j, s in enumerate(p["species"]):
        x[..., 3 + j] = s["X_inlet"]
    return x


def target_fields(p: dict, m: np.ndarray) -> np.ndarray:
    """[D, H, W, 9] float32 target from the solver's moments (temperatures as deviations
    from T_in, ``moments_host(t_dev=True)``)."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ns = len(p["species"])
    n = nx * ny * nz
    solid = np.asarray(p["mask"]).reshape(n) > 0
    y = np.zeros((N_OUT, n), np.float32)
    y[0:3] = m[2 * ns:2 * ns + 3] / p["u_inlet"]
    Xin = np.array([s["X_inlet"] for s in p["species"]])
    y[3:3 + ns] = np.where(solid[None], 0.0, (m[ns:2 * ns] - Xin[:, None]) * X_SCALE)
    y[3 + ns] = np.where(solid, m[2 * ns + 4], m[2 * ns + 3]) / T_SCALE_K
    return np.ascontiguousarray(y.reshape(N_OUT, nz, ny, nx).transpose(1, 2, 3, 0))


def fields_from_prediction(p: dict, y: np.ndarray) -> dict:
    """Initial fields for ``Solver.set_fields`` from a [D, H, W, 9] prediction."""
    nx, ny, nz = p["nx"], p["ny"], p["nz"]
    ns = len(p["species"])
    n = nx * ny * nz
    y = np.asarray(y, np.float64).reshape(n, N_OUT).T
    solid = np.asarray(p["mask"]).reshape(n) > 0
    Xin = np.array([s["X_inlet"] for s in p["species"]])
    u = np.where(solid[None], 0.0, y[0:3] * p["u_inlet"])
    X = Xin[:, None] + y[3:3 + ns] / X_SCALE
    X = np.where(solid[None], Xin[:, None], np.maximum(X, 1e-7))
    X /= X.sum(axis=0, keepdims=True)
    T = p["T_inlet_K"] + y[3 + ns] * T_SCALE_K
    return {"X": X, "u": u, "T_K": np.where(solid, p["T_init_K"], T), "Ts_K": np.where(solid, T, p["T_init_K"]),
            "C": np.where(solid, 1.0, p["T_inlet_K"] / T)}


def solve(p: dict, init=None, tol=1e-6, every=250, max_steps=200_000, device=0):
    """Steps and wall time (synchronised host clock) for the solver to reach the
    steady-state residual tol, checked every `every` steps; the solver is returned with
    its final state. A diverged run (FDLBM_EUNSTABLE) returns converged False."""
    import torch

    from . import fdlbm
    s = fdlbm.Solver(p, device=device)
    try:
        if init is not None:
            s.set_fields(init)
        s.residual()
        torch.cuda.synchronize(device)
    except BaseException:
        s.close()                       # the caller never sees this solver
        raise
    t0 = time.perf_counter()
    steps, r, diverged = 0, float("inf"), False
    try:
        while steps < max_steps:
            s.step(every)
            steps += every
            r = s.residual()
            if not np.isfinite(r):
                diverged = True
                break
            if r < tol:
                break
        s.sync()
    except fdlbm.FdlbmError:
        diverged = True
    except BaseException:
        s.close()
        raise
    el = time.perf_counter() - t0
    return s, {"steps": steps, "seconds": el, "residual": r, "converged": (r < tol) and not diverged,
               "diverged": diverged}


def generate(problems, tol=1e-6, every=250, max_steps=200_000, device=0) -> list:
    """Steady fields of every problem from a cold start: (input, target, run stats)."""
    data = []
    for p in problems:
        s, st = solve(p, None, tol, every, max_steps, device)
        try:
            m = s.moments_host(t_dev=True).astype(np.float64)
        finally:
            s.close()
        data.append({"x": network_input(p), "y": target_fields(p, m), "stats": st})
    return data


def init_params(seed: int) -> dict:
    """He-normal 3x3x3 and head weights (std sqrt(2 / fan_in)), zero biases, in the
    layout [o][c][3][3][3] (head [o][c]), FP64."""
    rng = np.random.default_rng(seed)
    p = {}
    L = len(CHANNELS)

    def conv(name, o, c, k):
        fan = c * k ** 3
        shape = (o, c, 3, 3, 3) if k == 3 else (o, c)
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / fan), shape)
        p[name + ".b"] = np.zeros(o)

    c = 16
    for l in range(L):
        conv(f"enc{l}a", CHANNELS[l], c, 3)
        conv(f"enc{l}b", CHANNELS[l], CHANNELS[l], 3)
        c = CHANNELS[l]
    for l in range(L - 2, -1, -1):
        conv(f"dec{l}a", CHANNELS[l], CHANNELS[l + 1] + CHANNELS[l], 3)
        conv(f"dec{l}b", CHANNELS[l], CHANNELS[l], 3)
    conv("head", N_OUT, CHANNELS[0], 1)
    return p


def new_model(seed: int = 0):
    """A U-Net of the warm start's architecture with He-normal weights."""
    from . import net
    return net.UNet(init_params(seed), CHANNELS, N_OUT)


def train(model, data, iters=600, batch=4, lr=2e-3, seed=0):
    """Adam on the mean-squared error over random mini-batches; returns the loss curve
    (one value per iteration)."""
    import torch

    from . import net
    rng = np.random.default_rng(seed)
    xs = torch.tensor(np.stack([d["x"] for d in data]), device="cuda").to(torch.bfloat16)
    ys = torch.tensor(np.stack([d["y"] for d in data]), device="cuda")
    losses = []
    for it in range(iters):
        idx = torch.tensor(rng.choice(len(data), size=min(batch, len(data)), replace=False), device="cuda")
        x = xs.index_select(0, idx).contiguous()
        t = ys.index_select(0, idx).contiguous()
        y = model.forward(x)
        loss, gy = net.mse(y, t)
        g = model.backward(gy)
        model.adam_step(g, lr=lr * (0.5 * (1 + np.cos(np.pi * it / iters)) * 0.9 + 0.1))
        losses.append(loss)
    net.check()
    return [float(l) for l in losses]


def predict(model, p: dict) -> np.ndarray:
    import torch
    x = torch.tensor(network_input(p)[None], device="cuda").to(torch.bfloat16)
    return model.forward(x)[0].cpu().numpy()


def warm_vs_cold(model, p: dict, tol=1e-6, every=250, max_steps=200_000, device=0) -> dict:
    """Steps and wall time to the residual tol from a cold start and from the network's
    prediction (inference time included); a warm run that diverges, needs more steps
    than the cold one, or whose predicted fields the solver rejects is counted as its own
    cost plus the cold run (the fallback)."""
    import torch

    from . import fdlbm
    s, cold = solve(p, None, tol, every, max_steps, device)
    s.close()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    init = fields_from_prediction(p, predict(model, p))
    t_inf = time.perf_counter() - t0
    try:
        s, warm = solve(p, init, tol, every, max(cold["steps"], every), device)
        s.close()
    except fdlbm.FdlbmError as e:  # fields outside the equilibrium's range: not used
        warm = {"steps": 0, "seconds": 0.0, "residual": float("inf"), "converged": False,
                "diverged": False, "rejected": str(e)[:200]}
    warm["seconds"] += t_inf
    warm["inference_seconds"] = t_inf
    warm["fallback"] = not warm["converged"]
    if warm["fallback"]:  # the prediction is discarded: a cold run follows
        warm["steps"] += cold["steps"]
        warm["seconds"] += cold["seconds"]
    return {"cold": cold, "warm": warm}
