"""Slab decomposition of a D2Q9 problem along x over ranks of a torch.distributed group.

Every rank owns a contiguous range of columns [x0, x1) (its interior) and runs a local
solver on a slab lattice: the interior plus HALO ghost columns on each side that face
another rank, and one inert solid padding column beyond them with a closed face. Once
per time step, before the step, each rank sends the HALO columns at each end of its
interior to the neighbour on that side (point-to-point send/recv; periodic x wraps the
last rank onto the first) and overwrites its ghost columns with what it receives. A
node's update reads only the state of nodes within HALO columns of it, so the interior
of every slab evolves exactly as the same columns of the undecomposed lattice.

HALO = 4: the deepest streaming stencil reaches 3 nodes upstream (the backward form of
Sec. 4.2), and the energy-correction divergence (reading R8, current time level) uses
the moments of the axis neighbours, whose own pulls reach 3 further. The state that is
exchanged is the state a step reads: the stored populations (post-collision on gas
nodes, emissions on wall nodes), the solid temperature and the gas mixture temperature
of the previous step (read by the paper's coupling law at interface nodes).

The FP64 conserved totals and the steady-state residual (reading R16) are summed over
interiors and all-reduced. The local solver is any object with ``step(n)``,
``get_state() -> (g [ns][9][n], Ts [n], T [n])``, ``set_state(g, Ts, T)``,
``moments() -> [2 ns + 4][n]`` (T and T_s in K), ``classes() -> [n]`` and the attributes
``ns``, ``nx``, ``ny``; ``make_solver(problem)`` builds one for a slab problem dict.
"""
from __future__ import annotations

import numpy as np

from . import workloads as W

HALO = 4
Q = 9
_EX = (0, 1, 0, -1, 0, 1, -1, -1, 1)
_EY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
GAS_CLASS, WALL_CLASS, SOLID_CLASS = 0, 3, 4


def partition(nx: int, world: int) -> list:
    """Contiguous column ranges [x0, x1), as even as possible; each at least HALO wide
    (so that a ghost strip comes from one neighbour's interior)."""
    if world < 1 or nx < world * HALO:
        raise ValueError(f"cannot split {nx} columns into {world} slabs of at least {HALO}")
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

    def __init__(self, nx: int, periodic_x: bool, x0: int, x1: int, world: int, rank: int):
        self.x0, self.x1 = x0, x1
        self.left = world > 1 and (periodic_x or rank > 0)          # ghost strip on the left
        self.right = world > 1 and (periodic_x or rank < world - 1)  # ghost strip on the right
        cols = []
        if self.left:
            cols += [-1] + [(x0 - HALO + c) % nx for c in range(HALO)]
        self.lo = len(cols)
        cols += list(range(x0, x1))
        self.hi = len(cols)
        if self.right:
            cols += [(x1 + c) % nx for c in range(HALO)] + [-1]
        self.cols = cols
        self.width = len(cols)


def slab_problem(p: dict, lay: SlabLayout) -> dict:
    """The problem dict of a slab: the global mask's columns (padding columns inert
    solid), the global x faces where the slab reaches them and closed faces at cuts, the
    initial fields of the same columns."""
    nx, ny = p["nx"], p["ny"]
    cols = np.array(lay.cols)
    real = cols >= 0
    mask = np.asarray(p["mask"]).reshape(ny, nx)
    sm = np.full((ny, lay.width), W.INERT, np.uint8)
    sm[:, real] = mask[:, cols[real]]
    faces = list(p["face_bc"])
    if lay.left:
        faces[0] = W.CLOSED
    if lay.right:
        faces[1] = W.CLOSED
    q = {k: v for k, v in p.items() if k not in ("mask", "nx", "ny", "face_bc", "init", "wall_u")}
    q.update(nx=lay.width, ny=ny, mask=sm.reshape(-1), face_bc=faces)
    if p.get("wall_u") is not None:
        raise NotImplementedError("slab decomposition: moving walls are not supported")
    src = p.get("init") or {}
    if src:
        def cut(a, lead):
            a = np.asarray(a, np.float64).reshape(lead, ny, nx)
            out = np.empty((lead, ny, lay.width))
            out[:, :, real] = a[:, :, cols[real]]
            # padding columns are solid: any admissible state will do
            out[:, :, ~real] = a[:, :, cols[real][:1]]
            return out.reshape(lead, -1)
        init = {}
        for key, lead in (("X", len(p["species"])), ("u", 2), ("T_K", 1), ("Ts_K", 1), ("C", 1)):
            if src.get(key) is not None:
                v = cut(src[key], lead)
                init[key] = v[0] if key in ("T_K", "Ts_K", "C") else v
        q["init"] = init
    else:
        q["init"] = None
    return q


class SlabRunner:
    """One rank of the decomposition: its layout, its local solver and the exchange.
    ``dist`` is torch.distributed with an initialised process group (world >= 2)."""

    def __init__(self, p: dict, make_solver, dist, group=None):
        if p["dim"] != 2 or p["lattice"] != 9:
            raise NotImplementedError("slab decomposition covers D2Q9")
        if p.get("phi_lagged"):
            raise NotImplementedError("slab decomposition reads the current time level only")
        self.dist, self.group = dist, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.p = p
        self.nx, self.ny = p["nx"], p["ny"]
        self.periodic_x = p["face_bc"][0] == W.PERIODIC
        self.parts = partition(self.nx, self.world)
        x0, x1 = self.parts[self.rank]
        self.lay = SlabLayout(self.nx, self.periodic_x, x0, x1, self.world, self.rank)
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
        """Send the HALO interior columns at each end to the neighbour on that side and
        receive its columns into this slab's ghost strips."""
        import torch
        g, Ts, T = self.solver.get_state()
        ny, w, ns = self.ny, self.lay.width, self.ns
        g = g.reshape(ns, Q, ny, w)
        Ts = Ts.reshape(ny, w)
        T = T.reshape(ny, w)
        lo, hi = self.lay.lo, self.lay.hi

        def pack(c0):
            return torch.from_numpy(np.concatenate([g[:, :, :, c0:c0 + HALO].reshape(-1),
                                                    Ts[:, c0:c0 + HALO].reshape(-1),
                                                    T[:, c0:c0 + HALO].reshape(-1)]))

        count = (ns * Q + 2) * ny * HALO
        sends, recvs = [], {}
        # to the left neighbour: my first HALO interior columns fill its right strip
        for side, c0 in ((-1, lo), (1, hi - HALO)):
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
            ng = ns * Q * ny * HALO
            c0 = lo - HALO if side < 0 else hi
            g[:, :, :, c0:c0 + HALO] = a[:ng].reshape(ns, Q, ny, HALO)
            Ts[:, c0:c0 + HALO] = a[ng:ng + ny * HALO].reshape(ny, HALO)
            T[:, c0:c0 + HALO] = a[ng + ny * HALO:].reshape(ny, HALO)
        self.solver.set_state(g.reshape(ns, Q, -1), Ts.reshape(-1), T.reshape(-1))

    def step(self, n: int = 1):
        for _ in range(n):
            self.exchange()
            self.solver.step(1)
            self.steps += 1

    # -- outputs ----------------------------------------------------------------------
    def interior_moments(self) -> np.ndarray:
        m = self.solver.moments().reshape(-1, self.ny, self.lay.width)
        return np.ascontiguousarray(m[:, :, self.lay.lo:self.lay.hi])

    def interior_classes(self) -> np.ndarray:
        c = self.solver.classes().reshape(self.ny, self.lay.width)
        return np.ascontiguousarray(c[:, self.lay.lo:self.lay.hi])

    def gather_moments(self):
        """The global moment fields [2 ns + 4][n] on rank 0 (None elsewhere)."""
        import torch
        mine = torch.from_numpy(self.interior_moments().reshape(-1))
        sizes = [(2 * self.ns + 4) * self.ny * (b - a) for a, b in self.parts]
        if self.rank == 0:
            bufs = [mine] + [torch.empty(s, dtype=torch.float64) for s in sizes[1:]]
            for r in range(1, self.world):
                self.dist.recv(bufs[r], r, group=self.group, tag=7)
            nf = 2 * self.ns + 4
            out = np.empty((nf, self.ny, self.nx))
            for r, (a, b) in enumerate(self.parts):
                out[:, :, a:b] = bufs[r].numpy().reshape(nf, self.ny, b - a)
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
        ns, ny, w = self.ns, self.ny, self.lay.width
        lo, hi = self.lay.lo, self.lay.hi
        T0 = self.p["T0_K"]
        m = self.solver.moments().reshape(2 * ns + 4, ny, w)
        cls = self.solver.classes().reshape(ny, w)
        g, _, _ = self.solver.get_state()
        g = g.reshape(ns, Q, ny, w)
        M = np.array([d["M_gmol"] for d in self.p["species"]], np.float64)
        M = M / M.min()
        c = 1.0 / np.sqrt(M)
        gas = cls[:, lo:hi] == GAS_CLASS
        rho = m[:ns, :, lo:hi]
        u2 = m[2 * ns, :, lo:hi] ** 2 + m[2 * ns + 1, :, lo:hi] ** 2
        T = m[2 * ns + 2, :, lo:hi] / (3.0 * T0)
        C = (rho / M[:, None, None]).sum(0)
        E = float(np.where(gas, C * T + 0.5 * rho.sum(0) * u2, 0.0).sum())
        mass = np.where(gas[None], rho, 0.0).sum((1, 2))
        moles = mass / M
        # wall emissions in transit: population i of a wall node whose neighbour along
        # e_i is gas
        yy, xx = np.meshgrid(np.arange(ny), np.arange(lo, hi), indexing="ij")
        wall = cls[:, lo:hi] == WALL_CLASS
        for i in range(1, Q):
            xn, yn = xx + _EX[i], (yy + _EY[i]) % ny
            inside = (xn >= 0) & (xn < w)
            to_gas = np.zeros_like(wall)
            to_gas[inside] = cls[yn[inside], xn[inside]] == GAS_CLASS
            sel = wall & to_gas
            for j in range(ns):
                v = np.where(sel, g[j, i, :, lo:hi], 0.0).sum()
                mass[j] += v
                moles[j] += v / M[j]
                E += 0.5 * c[j] ** 2 * (_EX[i] ** 2 + _EY[i] ** 2) * v
        solid = (cls[:, lo:hi] == WALL_CLASS) | (cls[:, lo:hi] == SOLID_CLASS)
        H = float(np.where(solid, self.p["rhocp_s"] * m[2 * ns + 3, :, lo:hi] / (3.0 * T0), 0.0).sum())
        v = self._allreduce(np.concatenate([[E, H], mass, moles]))
        return {"E_gas": v[0], "H_solid": v[1], "mass": v[2:2 + ns], "moles": v[2 + ns:]}

    def residual(self, K: int) -> float:
        """Steady-state residual (reading R16) over the interiors, all-reduced:
        max over fields F of ||F(t) - F(t - K)|| / (K max(||F(t) - F_ref||, 1e-30)), F
        in u_x, u_y, X_j, T on gas nodes and T_s on solid nodes (F_ref 0, X_inlet,
        T_inlet); inf on the first call (no snapshot)."""
        ns = self.ns
        m = self.interior_moments().reshape(2 * ns + 4, -1)
        cls = self.interior_classes().reshape(-1)
        gas = cls == GAS_CLASS
        solid = (cls == WALL_CLASS) | (cls == SOLID_CLASS)
        Xin = [d["X_inlet"] for d in self.p["species"]]
        tK = 3.0 * self.p["T0_K"]
        Tin = self.p["T_inlet_K"] / tK
        fields = [(m[2 * ns], 0.0, gas), (m[2 * ns + 1], 0.0, gas)]
        fields += [(m[ns + j], Xin[j], gas) for j in range(ns)]
        fields += [(m[2 * ns + 2] / tK, Tin, gas), (m[2 * ns + 3] / tK, Tin, solid)]
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
