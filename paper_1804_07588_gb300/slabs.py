"""Slab decomposition of a D2Q9 or D3Q19 problem along x over ranks of a
torch.distributed group.

Every rank owns a contiguous range of x columns [x0, x1) (its interior; in 3D a column
is a y-z plane) and runs a local solver on a slab lattice: the interior plus HALO ghost
columns on each side that face another rank, and one inert solid padding column beyond
them with a closed face. Once
per time step, before the step, each rank sends the HALO columns at each end of its
interior to the neighbour on that side (point-to-point send/recv; periodic x wraps the
last rank onto the first) and overwrites its ghost columns with what it receives. A
node's update reads only the state of nodes within HALO columns of it, so the interior
of every slab evolves exactly as the same columns of the undecomposed lattice.

HALO = 3, the reach of one step: a gas node pulls with the central stencil of Sec. 4.2
(its own population always exists), 2 nodes upstream, and a wall node's arrival pulls
may take the backward form, 3 nodes upstream; the energy-correction divergence (reading
R8, current time level) reads the moments of the gas axis neighbours only (faces towards
non-gas nodes carry no flux), whose central pulls reach 1 + 2. Wall emissions are pulled
as stored (the wall pass writes the next level), so nothing reaches further; with one
column less the slabs no longer reproduce the undecomposed run. The state that is
exchanged is the state a step reads: the stored populations (post-collision on gas
nodes, emissions on wall nodes), the solid temperature and the gas mixture temperature
of the previous step (read by the paper's coupling law at interface nodes).

The FP64 conserved totals and the steady-state residual (reading R16) are summed over
interiors and all-reduced. The local solver is any object with ``step(n)``,
``get_state() -> (g [ns][Q][n], Ts [n], T [n])``, ``set_state(g, Ts, T)``,
``moments() -> [2 ns + D + 2][n]`` (rho_j, X_j, the D velocity components, T and T_s in
K), ``classes() -> [n]`` and the attribute ``ns``; ``make_solver(problem)`` builds one
for a slab problem dict. Node index x + nx (y + ny z), x fastest: every field is handled
as [lead][rows][columns] with rows = ny nz.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

HALO = 3
# Velocity sets in the population order of the library and of the FP64 oracles.
VELOCITIES = {
    9: ((0, 0, 0), (1, 0, 0), (0, 1, 0), (-1, 0, 0), (0, -1, 0), (1, 1, 0), (-1, 1, 0), (-1, -1, 0),
        (1, -1, 0)),
    19: ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1), (1, 1, 0),
         (-1, -1, 0), (1, -1, 0), (-1, 1, 0), (1, 0, 1), (-1, 0, -1), (1, 0, -1), (-1, 0, 1), (0, 1, 1),
         (0, -1, -1), (0, 1, -1), (0, -1, 1)),
}
GAS_CLASS, WALL_CLASS, SOLID_CLASS = 0, 3, 4


def partition(nx: int, world: int, halo: int = HALO) -> list:
    """Contiguous column ranges [x0, x1), as even as possible; each at least halo wide
    (so that a ghost strip comes from one neighbour's interior)."""
    if world < 1 or nx < world * halo:
        raise ValueError(f"cannot split {nx} columns into {world} slabs of at least {halo}")
    base, extra = divmod(nx, world)
    out, x = [], 0
    for r in range(world):
        w = base + (1 if r < extra else 0)
        out.append((x, x + w))
        x += w
    return out


class SlabLayout:
    """Columns of one rank's slab lattice. ``cols`` are the global columns of the slab
    lattice left to right (-1 marks a padding column); ``lo``/``hi`` the slab-lattice
    column range of the interior."""

    def __init__(self, nx: int, periodic_x: bool, x0: int, x1: int, world: int, rank: int, halo: int = HALO):
        self.x0, self.x1 = x0, x1
        self.halo = halo
        self.left = world > 1 and (periodic_x or rank > 0)          # ghost strip on the left
        self.right = world > 1 and (periodic_x or rank < world - 1)  # ghost strip on the right
        cols = []
        if self.left:
            cols += [-1] + [(x0 - halo + c) % nx for c in range(halo)]
        self.lo = len(cols)
        cols += list(range(x0, x1))
        self.hi = len(cols)
        if self.right:
            cols += [(x1 + c) % nx for c in range(halo)] + [-1]
        self.cols = cols
        self.width = len(cols)


def slab_problem(p: dict, lay: SlabLayout) -> dict:
    """The problem dict of a slab: the global mask's columns (padding columns inert
    solid), the global x faces where the slab reaches them and closed faces at cuts, the
    initial fields of the same columns."""
    nx = p["nx"]
    rows = p["ny"] * (p.get("nz", 1) if p["dim"] == 3 else 1)
    cols = np.array(lay.cols)
    real = cols >= 0
    mask = np.asarray(p["mask"]).reshape(rows, nx)
    sm = np.full((rows, lay.width), W.INERT, np.uint8)
    sm[:, real] = mask[:, cols[real]]
    faces = list(p["face_bc"])
    if lay.left:
        faces[0] = W.CLOSED
    if lay.right:
        faces[1] = W.CLOSED
    q = {k: v for k, v in p.items() if k not in ("mask", "nx", "face_bc", "init", "wall_u")}
    q.update(nx=lay.width, mask=sm.reshape(-1), face_bc=faces)
    if p.get("wall_u") is not None:
        raise NotImplementedError("slab decomposition: moving walls are not supported")
    src = p.get("init") or {}
    if src:
        def cut(a, lead):
            a = np.asarray(a, np.float64).reshape(lead, rows, nx)
            out = np.empty((lead, rows, lay.width))
            out[:, :, real] = a[:, :, cols[real]]
            # padding columns are solid: any admissible state will do
            out[:, :, ~real] = a[:, :, cols[real][:1]]
            return out.reshape(lead, -1)
        init = {}
        for key, lead in (("X", len(p["species"])), ("u", p["dim"]), ("T_K", 1), ("Ts_K", 1), ("C", 1)):
            if src.get(key) is not None:
                v = cut(src[key], lead)
                init[key] = v[0] if key in ("T_K", "Ts_K", "C") else v
        q["init"] = init
    else:
        q["init"] = None
    return q


class SlabRunner:
    """One rank of the decomposition: its layout, its local solver and the exchange.
    ``dist`` is torch.distributed with an initialised process group (world >= 2);
    ``halo`` is the ghost depth (HALO, the reach of one step; less is for tests that show
    the reach is needed)."""

    def __init__(self, p: dict, make_solver, dist, group=None, halo: int = HALO):
        if (p["dim"], p["lattice"]) not in ((2, 9), (3, 19)):
            raise NotImplementedError("slab decomposition covers D2Q9 and D3Q19")
        if p.get("phi_lagged"):
            raise NotImplementedError("slab decomposition reads the current time level only")
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.p = p
        self.dim, self.Q = p["dim"], p["lattice"]
        self.nx, self.ny = p["nx"], p["ny"]
        self.nz = p["nz"] if self.dim == 3 else 1
        self.rows = self.ny * self.nz
        self.periodic_x = p["face_bc"][0] == W.PERIODIC
        self.halo = halo
        self.parts = partition(self.nx, self.world, halo)
        x0, x1 = self.parts[self.rank]
        self.lay = SlabLayout(self.nx, self.periodic_x, x0, x1, self.world, self.rank, halo)
        self.solver = make_solver(slab_problem(p, self.lay))
        self.ns = self.solver.ns
        self._snap = None
        self.steps = 0

    # -- neighbours -------------------------------------------------------------------
    def _nbr(self, side: int):
        if side < 0:
            if not self.lay.left:
                return None
            return (self.rank - 1) % self.world
        if not self.lay.right:
            return None
        return (self.rank + 1) % self.world

    def exchange(self):
        """Send the halo interior columns at each end to the neighbour on that side and
        receive its columns into this slab's ghost strips."""
        import torch
        g, Ts, T = self.solver.get_state()
        ny, w, ns, Q = self.rows, self.lay.width, self.ns, self.Q
        g = g.reshape(ns, Q, ny, w)
        Ts = Ts.reshape(ny, w)
        T = T.reshape(ny, w)
        lo, hi, H = self.lay.lo, self.lay.hi, self.halo

        def pack(c0):
            return torch.from_numpy(np.concatenate([g[:, :, :, c0:c0 + H].reshape(-1),
                                                    Ts[:, c0:c0 + H].reshape(-1),
                                                    T[:, c0:c0 + H].reshape(-1)]))

        count = (ns * Q + 2) * ny * H
        sends, recvs = [], {}
        # to the left neighbour: my first H interior columns fill its right strip
        for side, c0 in ((-1, lo), (1, hi - H)):
            nb = self._nbr(side)
            if nb is None:
                continue
            buf = torch.empty(count, dtype=torch.float64)
            recvs[side] = buf
            sends.append(self.dist.isend(pack(c0), nb, group=self.group, tag=0 if side < 0 else 1))
            sends.append(self.dist.irecv(buf, nb, group=self.group, tag=1 if side < 0 else 0))
        for r in sends:
            r.wait()
        for side, buf in recvs.items():
            a = buf.numpy()
            ng = ns * Q * ny * H
            c0 = lo - H if side < 0 else hi
            g[:, :, :, c0:c0 + H] = a[:ng].reshape(ns, Q, ny, H)
            Ts[:, c0:c0 + H] = a[ng:ng + ny * H].reshape(ny, H)
            T[:, c0:c0 + H] = a[ng + ny * H:].reshape(ny, H)
        self.solver.set_state(g.reshape(ns, Q, -1), Ts.reshape(-1), T.reshape(-1))

    def step(self, n: int = 1):
        for _ in range(n):
            self.exchange()
            self.solver.step(1)
            self.steps += 1

    # -- outputs ----------------------------------------------------------------------
    def interior_moments(self) -> np.ndarray:
        m = self.solver.moments().reshape(-1, self.rows, self.lay.width)
        return np.ascontiguousarray(m[:, :, self.lay.lo:self.lay.hi])

    def interior_classes(self) -> np.ndarray:
        c = self.solver.classes().reshape(self.rows, self.lay.width)
        return np.ascontiguousarray(c[:, self.lay.lo:self.lay.hi])

    def gather_moments(self):
        """The global moment fields [2 ns + D + 2][n] on rank 0 (None elsewhere)."""
        import torch
        mine = torch.from_numpy(self.interior_moments().reshape(-1))
        nf = 2 * self.ns + self.dim + 2
        sizes = [nf * self.rows * (b - a) for a, b in self.parts]
        if self.rank == 0:
            bufs = [mine] + [torch.empty(s, dtype=torch.float64) for s in sizes[1:]]
            for r in range(1, self.world):
                self.dist.recv(bufs[r], r, group=self.group, tag=7)
            out = np.empty((nf, self.rows, self.nx))
            for r, (a, b) in enumerate(self.parts):
                out[:, :, a:b] = bufs[r].numpy().reshape(nf, self.rows, b - a)
            return out.reshape(nf, -1)
        self.dist.send(mine, 0, group=self.group, tag=7)
        return None

    def _allreduce(self, v: np.ndarray) -> np.ndarray:
        import torch
        t = torch.from_numpy(np.ascontiguousarray(v, np.float64))
        self.dist.all_reduce(t, group=self.group)
        return t.numpy()

    def totals(self) -> dict:
        """FP64 conserved totals summed over every rank's interior: gas energy D/2 C T +
        rho u^2 / 2 plus the energy of wall emissions in transit, solid enthalpy
        (rho c_p)_s T_s, species mass and moles on the same basis (lattice units)."""
        ns, D, Q, w = self.ns, self.dim, self.Q, self.lay.width
        ny, nz, rows = self.ny, self.nz, self.rows
        lo, hi = self.lay.lo, self.lay.hi
        T0 = self.p["T0_K"]
        m = self.solver.moments().reshape(2 * ns + D + 2, rows, w)
        cls = self.solver.classes().reshape(rows, w)
        g, _, _ = self.solver.get_state()
        g = g.reshape(ns, Q, rows, w)
        M = np.array([d["M_gmol"] for d in self.p["species"]], np.float64)
        M = M / M.min()
        c = 1.0 / np.sqrt(M)
        gas = cls[:, lo:hi] == GAS_CLASS
        rho = m[:ns, :, lo:hi]
        u2 = m[2 * ns, :, lo:hi] ** 2
        for a in range(1, D):
            u2 = u2 + m[2 * ns + a, :, lo:hi] ** 2
        T = m[2 * ns + D, :, lo:hi] / (3.0 * T0)
        C = (rho / M[:, None, None]).sum(0)
        E = float(np.where(gas, 0.5 * D * C * T + 0.5 * rho.sum(0) * u2, 0.0).sum())
        mass = np.where(gas[None], rho, 0.0).sum((1, 2))
        moles = mass / M
        # wall emissions in transit: population i of a wall node whose neighbour along
        # e_i is gas (y and z wrap where those faces are periodic)
        zz, yy, xx = (a.reshape(rows, hi - lo) for a in
                      np.meshgrid(np.arange(nz), np.arange(ny), np.arange(lo, hi), indexing="ij"))
        per_y = self.p["face_bc"][2] == W.PERIODIC
        per_z = D == 3 and self.p["face_bc"][4] == W.PERIODIC
        wall = cls[:, lo:hi] == WALL_CLASS
        for i, (ex, ey, ez) in enumerate(VELOCITIES[Q]):
            if i == 0:
                continue
            xn, yn, zn = xx + ex, yy + ey, zz + ez
            if per_y:
                yn = yn % ny
            if per_z:
                zn = zn % nz
            inside = (xn >= 0) & (xn < w) & (yn >= 0) & (yn < ny) & (zn >= 0) & (zn < nz)
            to_gas = np.zeros_like(wall)
            to_gas[inside] = cls[(yn + ny * zn)[inside], xn[inside]] == GAS_CLASS
            sel = wall & to_gas
            for j in range(ns):
                v = np.where(sel, g[j, i, :, lo:hi], 0.0).sum()
                mass[j] += v
                moles[j] += v / M[j]
                E += 0.5 * c[j] ** 2 * (ex * ex + ey * ey + ez * ez) * v
        solid = (cls[:, lo:hi] == WALL_CLASS) | (cls[:, lo:hi] == SOLID_CLASS)
        H = float(np.where(solid, self.p["rhocp_s"] * m[2 * ns + D + 1, :, lo:hi] / (3.0 * T0), 0.0).sum())
        v = self._allreduce(np.concatenate([[E, H], mass, moles]))
        return {"E_gas": v[0], "H_solid": v[1], "mass": v[2:2 + ns], "moles": v[2 + ns:]}

    def residual(self, K: int) -> float:
        """Steady-state residual (reading R16) over the interiors, all-reduced:
        max over fields F of ||F(t) - F(t - K)|| / (K max(||F(t) - F_ref||, 1e-30)), F
        in the velocity components, X_j, T on gas nodes and T_s on solid nodes (F_ref 0,
        X_inlet, T_inlet); inf on the first call (no snapshot)."""
        ns, D = self.ns, self.dim
        m = self.interior_moments().reshape(2 * ns + D + 2, -1)
        cls = self.interior_classes().reshape(-1)
        gas = cls == GAS_CLASS
        solid = (cls == WALL_CLASS) | (cls == SOLID_CLASS)
        Xin = [d["X_inlet"] for d in self.p["species"]]
        tK = 3.0 * self.p["T0_K"]
        Tin = self.p["T_inlet_K"] / tK
        fields = [(m[2 * ns + a], 0.0, gas) for a in range(D)]
        fields += [(m[ns + j], Xin[j], gas) for j in range(ns)]
        fields += [(m[2 * ns + D] / tK, Tin, gas), (m[2 * ns + D + 1] / tK, Tin, solid)]
        cur = np.stack([f for f, _, _ in fields])
        sums = np.zeros(2 * len(fields))
        if self._snap is not None:
            for q, (f, ref, sel) in enumerate(fields):
                sums[2 * q] = ((f - self._snap[q]) ** 2)[sel].sum()
                sums[2 * q + 1] = ((f - ref) ** 2)[sel].sum()
        first = self._snap is None
        self._snap = cur
        tot = self._allreduce(sums)
        if first:
            return float("inf")
        r = 0.0
        for q in range(len(fields)):
            r = max(r, np.sqrt(tot[2 * q]) / (K * max(np.sqrt(tot[2 * q + 1]), 1e-30)))
        return r
