"""Seeded synthetic workloads for the coupled FD-LBM solver.

This module only *describes* problems: geometry masks, species and kinetics tables,
solid properties and (optionally) random initial macroscopic fields. It holds none of
the scheme's arithmetic -- no equilibria, no unit conversion, no streaming -- so that
the CUDA library and the FP64 CPU oracle can both be fed from it while sharing no
numerical code.

A problem is a plain ``dict`` (see :func:`channel`, :func:`porous_disks`,
:func:`periodic_box`) with these keys:

``dim, nx, ny, nz, lattice``   lattice shape; ``lattice`` is 9 (D2Q9) or 19 (D3Q19)
``mask``                       uint8 array, flat, x fastest: 0 gas, 1 inert solid,
                               2 catalytic solid
``face_bc``                    six ints for faces x-, x+, y-, y+, z-, z+:
                               0 periodic, 1 inlet, 2 outlet, 3 closed, 4 fixed-T
``species``                    list of dicts ``name, M_gmol, tau1, tau2, X_init, X_inlet``
``Pr, energy_correction``      Prandtl number of the correction term and its switch
``T0_K, T_init_K, T_inlet_K, T_solid_init_K, T_outer_K``  temperatures in kelvin
``u_inlet, inlet_profile``     inlet velocity (lattice units); 0 plug, 1 parabolic
``alpha_s, rhocp_s, kappa_f``  solid diffusivity and volumetric heat capacity, gas
                               conductivity for the paper's wall-temperature coupling
``coupling``                   0 conservative (default), 1 the paper's wall-temperature law
``reactions``                  list of dicts ``nu, k0, Ea_Jmol, Keq, dH_Jmol, rate_form``
``rho_w_tol, rho_w_maxit``     wall-density iteration tolerance and cap
``init``                       ``None`` or dict of float64 arrays ``X [ns, n]``,
                               ``u [dim, n]``, ``T_K [n]``, ``Ts_K [n]``, ``C [n]``
                               (molar concentration, lattice units, default 1)

The workloads follow the paper's test set-ups and the configurations the benchmark is
quoted on: a catalytic channel between FD-solid walls (water-gas shift at the walls,
Sec. 5 and Sec. 6 of the paper), a 2D porous bed of catalytic disks, and small periodic
boxes used for conservation checks.
"""
from __future__ import annotations

import math

import numpy as np

# Faces and mask codes (mirrored by the C header and the oracle header).
PERIODIC, INLET, OUTLET, CLOSED, FIXED_T = 0, 1, 2, 3, 4
GAS, INERT, CATALYTIC = 0, 1, 2
PLUG, PARABOLIC = 0, 1
CONSERVATIVE, PAPER = 0, 1
RATE_CONC_BILINEAR, RATE_XFRAC_REVERSIBLE = 0, 1

# Molar masses (g/mol) built from standard atomic weights so that the water-gas
# shift CO + H2O -> CO2 + H2 balances mass to rounding.
_A = {"C": 12.011, "O": 15.999, "H": 1.008, "N": 14.007}
MOLAR_MASS = {
    "CO": _A["C"] + _A["O"],
    "H2O": 2 * _A["H"] + _A["O"],
    "CO2": _A["C"] + 2 * _A["O"],
    "H2": 2 * _A["H"],
    "N2": 2 * _A["N"],
}
SPECIES_ORDER = ("CO", "H2O", "CO2", "H2", "N2")

# Relaxation times (lattice units) in the 0.6-1.0 range of the benchmark
# configurations; tau1 (viscous/thermal) and tau2 (diffusive) differ so that both
# relaxation stages of the two-step collision are exercised.
TAU1 = {"CO": 0.8, "H2O": 0.7, "CO2": 1.0, "H2": 0.6, "N2": 0.9}
TAU2 = {"CO": 0.7, "H2O": 0.9, "CO2": 0.65, "H2": 1.0, "N2": 0.75}

# Inlet composition CO/H2O/CO2/H2/N2 = 0.1/0.1/0/0/0.8 with the product species held
# at a 1e-6 trace (the paper's own inlet keeps 1e-6 of the products, Sec. 6) and the
# balance taken from N2.
X_INLET = {"CO": 0.1, "H2O": 0.1, "CO2": 1e-6, "H2": 1e-6, "N2": 0.8 - 2e-6}

# Solid: diffusivity 0.03 in lattice units (the paper's showcase value). The volumetric
# heat capacity 20.6 makes the solid conductivity alpha_s * rhocp_s ten times the gas
# conductivity 0.0618 of the inlet mixture (nu / Pr times the 2D molar heat capacity
# C (D + 2) / 2 at C = 1, T = 1/3, Pr = 0.7); 0.0618 is also the gas conductivity used
# by the paper's wall-temperature law.
ALPHA_S = 0.03
RHOCP_S = 20.6
KAPPA_F = 0.0618


def wgs_reaction(k0: float = 167.0, Ea_Jmol: float = 50e3, Keq: float = 10.0,
                 dH_Jmol: float = -41e3, rate_form: int = RATE_XFRAC_REVERSIBLE,
                 order=SPECIES_ORDER) -> dict:
    """Water-gas shift CO + H2O -> CO2 + H2 on the catalytic walls.

    ``k0`` is in lattice moles per wall node per step at unit mole fractions; 167
    gives k(500 K) ~ 1e-3 with Ea = 50 kJ/mol.
    """
    stoich = {"CO": -1, "H2O": -1, "CO2": 1, "H2": 1, "N2": 0}
    return {"nu": [stoich.get(s, 0) for s in order], "k0": k0, "Ea_Jmol": Ea_Jmol,
            "Keq": Keq, "dH_Jmol": dH_Jmol, "rate_form": rate_form}


def species_table(order=SPECIES_ORDER, X_init=None, X_inlet=None, tau1=None, tau2=None):
    X_init = X_init or X_INLET
    X_inlet = X_inlet or X_INLET
    tau1 = tau1 or TAU1
    tau2 = tau2 or TAU2
    return [{"name": s, "M_gmol": MOLAR_MASS[s], "tau1": tau1[s], "tau2": tau2[s],
             "X_init": X_init[s], "X_inlet": X_inlet[s]} for s in order]


def _base(dim, nx, ny, nz, mask, face_bc, **kw) -> dict:
    p = {
        "dim": dim, "nx": nx, "ny": ny, "nz": nz, "lattice": 9 if dim == 2 else 19,
        "mask": np.ascontiguousarray(mask.reshape(-1), dtype=np.uint8),
        "face_bc": list(face_bc) + [PERIODIC] * (6 - len(face_bc)),
        "species": species_table(),
        "Pr": 0.7, "energy_correction": 1,
        "T0_K": 500.0, "T_init_K": 500.0, "T_inlet_K": 500.0,
        "T_solid_init_K": 500.0, "T_outer_K": 500.0,
        "u_inlet": 0.0, "inlet_profile": PLUG,
        "alpha_s": ALPHA_S, "rhocp_s": RHOCP_S, "kappa_f": KAPPA_F,
        "coupling": CONSERVATIVE,
        "reactions": [wgs_reaction()],
        "rho_w_tol": 1e-8, "rho_w_maxit": 50,
        "init": None,
    }
    p.update(kw)
    return p


def channel(nx: int = 128, n_gas: int = 32, wall: int = 8, u_inlet: float = 0.02,
            profile: int = PARABOLIC, **kw) -> dict:
    """Catalytic channel: ``n_gas`` gas rows between two ``wall``-thick FD-solid walls.

    Inlet on x-, outlet on x+, outer solid faces held at ``T_outer_K``. With the
    defaults this is the 128x32 channel with 8-node walls (128 x 48 lattice).
    """
    ny = n_gas + 2 * wall
    mask = np.zeros((ny, nx), np.uint8)
    mask[:wall, :] = CATALYTIC
    mask[wall + n_gas:, :] = CATALYTIC
    return _base(2, nx, ny, 1, mask, [INLET, OUTLET, FIXED_T, FIXED_T],
                 u_inlet=u_inlet, inlet_profile=profile, **kw)


def couette(n_gas: int = 32, U_w: float = 0.03, dT_K: float = 2.0, nx: int = 1, linear_start: bool = True,
            **kw) -> dict:
    """Thermal Couette flow (the paper's viscous-heating test, Sec. 4.4): ``n_gas`` gas rows
    between a plate at rest (y = 0) and a plate moving at ``U_w`` along x (y = ny - 1), the
    moving one ``dT_K`` warmer; periodic in x. The plates are one-node FD-solid rows with
    a huge heat capacity and no conduction, so their temperatures stay fixed. With
    ``linear_start`` the gas starts from the linear velocity and temperature profiles."""
    ny = n_gas + 2
    mask = np.zeros((ny, nx), np.uint8)
    mask[0] = INERT
    mask[-1] = INERT
    kw.setdefault("reactions", [])
    kw.setdefault("alpha_s", 0.0)
    kw.setdefault("rhocp_s", 1e12)
    p = _base(2, nx, ny, 1, mask, [PERIODIC, PERIODIC, CLOSED, CLOSED], **kw)
    n = nx * ny
    wu = np.zeros((2, ny, nx))
    wu[0, -1, :] = U_w
    p["wall_u"] = wu.reshape(2, n)
    Ts = np.full((ny, nx), p["T_solid_init_K"])
    Ts[-1] += dT_K
    init = {"Ts_K": Ts.reshape(n)}
    if linear_start:
        y = np.repeat(np.arange(ny)[:, None], nx, 1) / (ny - 1)
        u = np.zeros((2, ny, nx))
        u[0] = U_w * y
        init["u"] = u.reshape(2, n)
        init["T_K"] = (p["T_init_K"] + dT_K * y).reshape(n)
    p["init"] = init
    return p


def disk_mask(nx: int, ny: int, porosity: float, rmin: float, rmax: float, seed: int,
              free_cols: int = 17, gap: float = 2.0, max_tries: int = 2_000_000):
    """Seeded random sequential addition of non-overlapping disks, periodic in y.

    Disk radii are uniform in [rmin, rmax]; centres keep ``gap`` lattice units of
    clearance between disk surfaces and stay ``free_cols`` columns away from the inlet
    and outlet. Disks are added until the digitised solid fraction of the whole
    lattice reaches ``1 - porosity``. Returns (mask, list of (cx, cy, r)).
    """
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), bool)
    target = (1.0 - porosity) * nx * ny
    n_solid = 0
    disks = []
    # Overlap test against the disks of the neighbouring cells of a grid of cell size
    # >= 2 rmax + gap (any disk closer than r + r' + gap has its centre there).
    cell = 2.0 * rmax + gap
    ncx = max(1, int(nx // cell))
    ncy = max(1, int(ny // cell))
    wx, wy = nx / ncx, ny / ncy
    grid = {}
    tries = 0
    while n_solid < target:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("disk packing did not reach the target porosity")
        r = rng.uniform(rmin, rmax)
        lo = free_cols + r + 1
        hi = nx - 1 - free_cols - r - 1
        cx = rng.uniform(lo, hi)
        cy = rng.uniform(0, ny)
        gx, gy = min(int(cx // wx), ncx - 1), min(int(cy // wy), ncy - 1)
        hit = False
        for ix in range(max(gx - 1, 0), min(gx + 2, ncx)):
            for iy in {(gy + o) % ncy for o in (-1, 0, 1)}:
                for (ox, oy, orr) in grid.get((ix, iy), ()):
                    dy = abs(oy - cy)
                    dy = min(dy, ny - dy)
                    if math.hypot(ox - cx, dy) < orr + r + gap:
                        hit = True
                        break
                if hit:
                    break
            if hit:
                break
        if hit:
            continue
        disks.append((cx, cy, r))
        grid.setdefault((gx, gy), []).append((cx, cy, r))
        xs = np.arange(int(math.floor(cx - r)), int(math.ceil(cx + r)) + 1)
        ys = np.arange(int(math.floor(cy - r)), int(math.ceil(cy + r)) + 1)
        dy = ys[:, None] - cy
        inside = (xs[None, :] - cx) ** 2 + dy ** 2 <= r * r
        yw = np.broadcast_to((ys % ny)[:, None], inside.shape)[inside]
        xw = np.broadcast_to(xs[None, :], inside.shape)[inside]
        n_solid += int((~solid[yw, xw]).sum())
        solid[yw, xw] = True
    mask = np.where(solid, CATALYTIC, GAS).astype(np.uint8)
    return mask, disks


def disk_mask_boolean(nx: int, ny: int, porosity: float, rmin: float, rmax: float, seed: int,
                      free_cols: int = 17, max_disks: int = 1_000_000):
    """Seeded Boolean model of overlapping disks, periodic in y: radii uniform in [rmin,
    rmax], centres uniform in the box but ``free_cols`` columns away from the inlet and
    outlet, disks added until the digitised solid fraction of the lattice reaches
    ``1 - porosity``. Overlap lets the porosity go below the ~0.55 where random sequential
    addition of separated disks jams. The gas phase must connect the inlet columns to the
    outlet columns (4-connected, periodic in y), else a ValueError is raised. Returns
    (mask [ny, nx], list of (cx, cy, r))."""
    rng = np.random.default_rng(seed)
    solid = np.zeros((ny, nx), bool)
    target = (1.0 - porosity) * nx * ny
    disks = []
    n_solid = 0
    while n_solid < target:
        if len(disks) >= max_disks:
            raise RuntimeError("disk packing did not reach the target porosity")
        r = rng.uniform(rmin, rmax)
        cx = rng.uniform(free_cols + r, nx - free_cols - r)
        cy = rng.uniform(0, ny)
        disks.append((cx, cy, r))
        xs = np.arange(max(int(math.floor(cx - r)), 0), min(int(math.ceil(cx + r)), nx - 1) + 1)
        ys = np.arange(int(math.floor(cy - r)), int(math.ceil(cy + r)) + 1)
        inside = ((xs[None, :] - cx) ** 2 + (ys[:, None] - cy) ** 2) <= r * r
        yi, xi = np.nonzero(inside)
        yw, xw = ys[yi] % ny, xs[xi]
        n_solid += int((~solid[yw, xw]).sum())
        solid[yw, xw] = True
    if not _percolates(~solid[None]):
        raise ValueError("disk packing: the gas phase does not connect inlet and outlet")
    return np.where(solid, CATALYTIC, GAS).astype(np.uint8), disks


def porous_disks(nx: int = 1024, ny: int = 512, porosity: float = 0.6, rmin: float = 6.0,
                 rmax: float = 12.0, seed: int = 1000, u_inlet: float = 0.01, **kw) -> dict:
    """2D porous bed of catalytic FD-solid disks, inlet x-, outlet x+, periodic in y.

    Defaults: the 1024x512 bed with radii U[6, 12], porosity 0.6 and plug inlet 0.01.
    """
    mask, _ = disk_mask(nx, ny, porosity, rmin, rmax, seed)
    return _base(2, nx, ny, 1, mask, [INLET, OUTLET, PERIODIC, PERIODIC],
                 u_inlet=u_inlet, inlet_profile=PLUG, **kw)


def periodic_box(nx: int = 16, ny: int = 12, solid_rows: int = 0, solid_cols: int = 0,
                 **kw) -> dict:
    """Fully periodic box. ``solid_rows`` > 0 puts a catalytic solid slab of that many
    rows at the bottom; ``solid_cols`` > 0 a slab of that many columns on the left (the
    quasi-1D 200 x 3 solid/gas enthalpy test of the paper, Sec. 5, is
    ``periodic_box(200, 3, solid_cols=100)``)."""
    mask = np.zeros((ny, nx), np.uint8)
    if solid_rows:
        mask[:solid_rows, :] = CATALYTIC
    if solid_cols:
        mask[:, :solid_cols] = CATALYTIC
    return _base(2, nx, ny, 1, mask, [PERIODIC] * 4, **kw)


def sphere_mask(nx: int, ny: int, nz: int, porosity: float, rmin: float, rmax: float, seed: int,
                free_cols: int = 12, max_spheres: int = 1_000_000):
    """Seeded Boolean model of overlapping spheres, periodic in y and z.

    Radii are uniform in [rmin, rmax]; centres are uniform in the box but keep
    ``free_cols`` columns free of solid at the inlet and outlet ends. Spheres are added
    until the digitised solid fraction of the lattice reaches ``1 - porosity`` (random
    sequential addition of non-overlapping spheres jams near a solid fraction of 0.38,
    below the 0.4-0.6 the 3D packings need, so spheres may overlap). The gas phase must
    connect the inlet columns to the outlet columns (6-connected, periodic in y and z),
    else a ValueError is raised. Returns (mask [nz, ny, nx], list of (cx, cy, cz, r)).
    """
    rng = np.random.default_rng(seed)
    solid = np.zeros((nz, ny, nx), bool)
    target = (1.0 - porosity) * nx * ny * nz
    spheres = []
    n_solid = 0
    while n_solid < target:
        if len(spheres) >= max_spheres:
            raise RuntimeError("sphere packing did not reach the target porosity")
        r = rng.uniform(rmin, rmax)
        cx = rng.uniform(free_cols + r, nx - free_cols - r)
        cy = rng.uniform(0, ny)
        cz = rng.uniform(0, nz)
        spheres.append((cx, cy, cz, r))
        xs = np.arange(max(int(math.floor(cx - r)), 0), min(int(math.ceil(cx + r)), nx - 1) + 1)
        ys = np.arange(int(math.floor(cy - r)), int(math.ceil(cy + r)) + 1)
        zs = np.arange(int(math.floor(cz - r)), int(math.ceil(cz + r)) + 1)
        inside = ((xs[None, None, :] - cx) ** 2 + (ys[None, :, None] - cy) ** 2
                  + (zs[:, None, None] - cz) ** 2) <= r * r
        zi, yi, xi = np.nonzero(inside)
        zw, yw, xw = zs[zi] % nz, ys[yi] % ny, xs[xi]
        n_solid += int((~solid[zw, yw, xw]).sum())
        solid[zw, yw, xw] = True
    if not _percolates(~solid):
        raise ValueError("sphere packing: the gas phase does not connect inlet and outlet")
    mask = np.where(solid, CATALYTIC, GAS).astype(np.uint8)
    return mask, spheres


def _percolates(gas: np.ndarray) -> bool:
    """Breadth-first search over 6-connected gas cells (periodic in y and z) from the
    x = 0 layer; True when it reaches the x = nx - 1 layer."""
    nz, ny, nx = gas.shape
    seen = np.zeros_like(gas)
    front = np.argwhere(gas[:, :, 0])
    front = np.concatenate([front, np.zeros((len(front), 1), np.int64)], axis=1)  # z, y, x
    seen[front[:, 0], front[:, 1], front[:, 2]] = True
    steps = ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))
    while len(front):
        nxt = []
        for dz, dy, dx in steps:
            z = (front[:, 0] + dz) % nz
            y = (front[:, 1] + dy) % ny
            x = front[:, 2] + dx
            ok = (x >= 0) & (x < nx)
            z, y, x = z[ok], y[ok], x[ok]
            new = gas[z, y, x] & ~seen[z, y, x]
            z, y, x = z[new], y[new], x[new]
            seen[z, y, x] = True
            nxt.append(np.stack([z, y, x], axis=1))
        front = np.unique(np.concatenate(nxt), axis=0) if nxt else np.zeros((0, 3), np.int64)
        if seen[:, :, nx - 1].any():
            return True
    return bool(seen[:, :, nx - 1].any())


def porous_spheres(nx: int = 256, ny: int = 128, nz: int = 128, porosity: float = 0.5,
                   rmin: float = 5.0, rmax: float = 10.0, seed: int = 2000, u_inlet: float = 0.01,
                   **kw) -> dict:
    """3D D3Q19 porous bed of catalytic FD-solid spheres (overlapping, Boolean model),
    inlet x-, outlet x+, periodic in y and z. Defaults: the 256x128x128 packing with
    radii U[5, 10], porosity 0.5, plug inlet 0.01."""
    mask, _ = sphere_mask(nx, ny, nz, porosity, rmin, rmax, seed)
    return _base(3, nx, ny, nz, mask, [INLET, OUTLET, PERIODIC, PERIODIC, PERIODIC, PERIODIC],
                 u_inlet=u_inlet, inlet_profile=PLUG, **kw)


def crop3(p: dict, nx: int, ny: int, nz: int, open_outlet: int = 2) -> dict:
    """Corner crop [0, nz) x [0, ny) x [0, nx) of a 3D problem's geometry, with the same
    faces (periodic in y and z) and the last ``open_outlet`` columns cleared of solid so
    that the outlet has upstream gas."""
    mask = np.asarray(p["mask"]).reshape(p["nz"], p["ny"], p["nx"])[:nz, :ny, :nx].copy()
    if open_outlet:
        mask[:, :, nx - open_outlet:] = GAS
    q = {k: v for k, v in p.items() if k not in ("mask", "nx", "ny", "nz", "init")}
    return _base(3, nx, ny, nz, mask, p["face_bc"], **{k: v for k, v in q.items()
                                                        if k not in ("dim", "lattice", "face_bc")})


def periodic_box3(nx: int = 12, ny: int = 10, nz: int = 8, solid_layers: int = 0, **kw) -> dict:
    """Fully periodic 3D box; ``solid_layers`` > 0 puts a catalytic slab of that many
    z-layers at the bottom."""
    mask = np.zeros((nz, ny, nx), np.uint8)
    if solid_layers:
        mask[:solid_layers] = CATALYTIC
    return _base(3, nx, ny, nz, mask, [PERIODIC] * 6, **kw)


def smooth_noise(shape, rng, modes: int = 4) -> np.ndarray:
    """Sum of a few random low-order Fourier modes, scaled to max |value| = 1 (2D shape
    (ny, nx) or 3D shape (nz, ny, nx))."""
    grids = np.meshgrid(*[np.arange(m, dtype=np.float64) for m in shape], indexing="ij")
    out = np.zeros(shape)
    for _ in range(modes):
        ks = [rng.integers(0, 4) for _ in shape]  # drawn x first, then y (then z)
        ph = rng.uniform(0, 2 * np.pi)
        arg = sum(k * g / m for k, g, m in zip(ks, grids[::-1], shape[::-1]))
        out += rng.normal() * np.cos(2 * np.pi * arg + ph)
    m = np.abs(out).max()
    return out / m if m > 0 else out


def random_fields(p: dict, seed: int, dX: float = 0.2, du: float = 0.01,
                  dT_K: float = 5.0, dTs_K: float = 5.0) -> dict:
    """Seeded smooth random initial fields around the problem's initial state.

    Mole fractions are scaled by (1 + dX * noise) and renormalised, velocities are
    +-``du``, gas and solid temperatures deviate by up to ``dT_K`` / ``dTs_K``.
    """
    rng = np.random.default_rng(seed)
    shape = (p["ny"], p["nx"]) if p["dim"] == 2 else (p["nz"], p["ny"], p["nx"])
    dim = p["dim"]
    ns = len(p["species"])
    X0 = np.array([s["X_init"] for s in p["species"]])
    X = np.empty((ns,) + shape)
    for j in range(ns):
        X[j] = X0[j] * (1.0 + dX * smooth_noise(shape, rng))
    X /= X.sum(axis=0, keepdims=True)
    u = np.stack([du * smooth_noise(shape, rng) for _ in range(dim)])
    T = p["T_init_K"] + dT_K * smooth_noise(shape, rng)
    Ts = p["T_solid_init_K"] + dTs_K * smooth_noise(shape, rng)
    n = int(np.prod(shape))
    return {"X": X.reshape(ns, n).copy(), "u": u.reshape(dim, n).copy(),
            "T_K": T.reshape(n).copy(), "Ts_K": Ts.reshape(n).copy()}


def local_transport(p: dict, mu_scale: float = 1.0, D_scale: float = 1.0) -> dict:
    """Switch a problem to locally updated relaxation times: species viscosities mu_j
    and binary diffusivities D_jk (lattice units) chosen so that, in the problem's inlet
    mixture at C = 1, T = 1/3, a species alone would have tau1 = its table value (mu_j =
    tau1_j C T) and every pair diffuses with D_jk = (tau2_j / M_j + tau2_k / M_k) T / 2
    (molar masses relative to the lightest). The Lennard-Jones collision integrals that
    would give these from the species' properties are not printed in the paper."""
    sp = p["species"]
    M = np.array([d["M_gmol"] for d in sp])
    M = M / M.min()
    T = 1.0 / 3.0
    for j, d in enumerate(sp):
        d["mu"] = mu_scale * d["tau1"] * T
        d["D"] = [0.0 if k == j else D_scale * 0.5 * (d["tau2"] / M[j] + e["tau2"] / M[k]) * T
                  for k, e in enumerate(sp)]
    p["local_tau"] = 1
    return p


def config0(**kw) -> dict:
    """2D D2Q9 catalytic channel: 128x32 gas nodes between two 8-node FD-solid walls,
    parabolic inlet peak 0.02, T_in = walls = 500 K (run length 2000 steps)."""
    return channel(**kw)


def config1(**kw) -> dict:
    """2D D2Q9 porous bed 1024x512, catalytic disks r ~ U[6, 12], porosity 0.6, seed
    1000, plug inlet 0.01 (run length 20000 steps)."""
    return porous_disks(**kw)


def config2(**kw) -> dict:
    """3D D3Q19 porous bed 256x128x128 of catalytic spheres r ~ U[5, 10] (overlapping),
    porosity 0.5, seed 2000, plug inlet 0.01."""
    return porous_spheres(**kw)


def config2_crop(nx: int = 64, ny: int = 32, nz: int = 32, **kw) -> dict:
    """The 64x32x32 corner crop of the config-2 packing (same seed), periodic in y and
    z, outlet opened: the oracle-sized case of the 3D bed."""
    return crop3(config2(**kw), nx, ny, nz)


def batch_instances(n: int = 64, seed: int = 3000, nx_range=(256, 1024), ny_range=(128, 256),
                    porosity=(0.4, 0.7), u_inlet=(0.005, 0.03), T_inlet_K=(450.0, 600.0)) -> list:
    """Independent 2D porous beds of uneven size for batched stepping: per instance, nx
    and ny uniform over multiples of 8 in the given ranges, porosity, plug inlet velocity
    and inlet temperature uniform in their ranges (the inlet temperature is also the
    reference T0, the initial gas and solid temperature). Catalytic disks of radius
    U[6, 12] from the Boolean model (overlapping, so that porosities down to 0.4 are
    reachable), seeded by seed + 1 + i; a draw whose gas does not connect inlet and
    outlet takes the next seed."""
    rng = np.random.default_rng(seed)
    out = []
    k = 0
    for i in range(n):
        nx = int(rng.integers(nx_range[0] // 8, nx_range[1] // 8 + 1)) * 8
        ny = int(rng.integers(ny_range[0] // 8, ny_range[1] // 8 + 1)) * 8
        por = float(rng.uniform(*porosity))
        u = float(rng.uniform(*u_inlet))
        T = float(rng.uniform(*T_inlet_K))
        while True:
            k += 1
            try:
                mask, _ = disk_mask_boolean(nx, ny, por, 6.0, 12.0, seed + k)
                break
            except ValueError:
                continue
        out.append(_base(2, nx, ny, 1, mask, [INLET, OUTLET, PERIODIC, PERIODIC], u_inlet=u, inlet_profile=PLUG,
                         T0_K=T, T_init_K=T, T_inlet_K=T, T_solid_init_K=T, T_outer_K=T))
    return out


def learning_instances(n: int = 576, seed: int = 4000, shape=(128, 64, 64), porosity=(0.4, 0.6),
                       u_inlet=(0.005, 0.03), T_inlet_K=(450.0, 600.0)) -> list:
    """Geometries and inlet conditions of the learned warm start's data: D3Q19 sphere
    packings of the given shape (nx, ny, nz), r ~ U[5, 10], porosity uniform in its range
    (overlapping spheres, so 0.4 is reachable), plug inlet velocity and inlet temperature
    uniform in their ranges (the inlet temperature is also T0 and the initial gas and
    solid temperature); instance i uses seed + i (the first 512 train, the last 64 test
    by default)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    out = []
    for i in range(n):
        por = float(rng.uniform(*porosity))
        u = float(rng.uniform(*u_inlet))
        T = float(rng.uniform(*T_inlet_K))
        out.append(porous_spheres(nx=nx, ny=ny, nz=nz, porosity=por, seed=seed + i, u_inlet=u, T0_K=T,
                                  T_init_K=T, T_inlet_K=T, T_solid_init_K=T, T_outer_K=T))
    return out
