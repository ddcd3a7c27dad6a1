"""Python binding of the C-ABI solver library ``libfdlbm.so`` (include/fdlbm.h).

Argument marshalling only: every step of the scheme runs in the library's CUDA kernels.
PyTorch provides the device memory (its caching allocator is handed to the library as
the allocation callback) and the stream. There is no CPU fallback: constructing a
:class:`Solver` without a CUDA device, or without the built library, raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

MAX_NS = 6
MAX_NR = 4
Q = 9
STATUS = {0: "FDLBM_OK", -1: "FDLBM_EINVAL", -2: "FDLBM_EGEOM", -3: "FDLBM_ECUDA",
          -4: "FDLBM_EUNSTABLE", -5: "FDLBM_ENOCONV", -6: "FDLBM_ETIMEOUT", -7: "FDLBM_ENOMEM",
          -8: "FDLBM_EIO"}


class FdlbmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Geometry(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("lattice", C.c_int),
                ("mask", C.POINTER(C.c_uint8)), ("face_bc", C.c_int * 6), ("nz", C.c_int),
                ("wall_u", C.POINTER(C.c_double))]


class Species(C.Structure):
    _fields_ = [("M_gmol", C.c_double), ("tau1", C.c_double), ("tau2", C.c_double),
                ("X_init", C.c_double), ("X_inlet", C.c_double), ("mu", C.c_double),
                ("D", C.c_double * MAX_NS)]


class Transport(C.Structure):
    _fields_ = [("Pr", C.c_double), ("energy_correction", C.c_int),
                ("T0_K", C.c_double), ("T_init_K", C.c_double), ("T_inlet_K", C.c_double),
                ("T_solid_init_K", C.c_double), ("T_outer_K", C.c_double),
                ("u_inlet", C.c_double), ("inlet_profile", C.c_int),
                ("alpha_s", C.c_double), ("rhocp_s", C.c_double), ("kappa_f", C.c_double),
                ("coupling", C.c_int), ("local_tau", C.c_int)]


class Kinetics(C.Structure):
    _fields_ = [("n_react", C.c_int), ("nu", (C.c_int * MAX_NS) * MAX_NR),
                ("k0", C.c_double * MAX_NR), ("Ea_Jmol", C.c_double * MAX_NR),
                ("Keq", C.c_double * MAX_NR), ("dH_Jmol", C.c_double * MAX_NR),
                ("rate_form", C.c_int * MAX_NR), ("rho_w_tol", C.c_double),
                ("rho_w_maxit", C.c_int)]


class Fields(C.Structure):
    _fields_ = [("X", C.POINTER(C.c_double)), ("u", C.POINTER(C.c_double)),
                ("T_K", C.POINTER(C.c_double)), ("Ts_K", C.POINTER(C.c_double)),
                ("C", C.POINTER(C.c_double))]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class Options(C.Structure):
    _fields_ = [("storage", C.c_int), ("device", C.c_int), ("stream", C.c_void_p),
                ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_ctx", C.c_void_p), ("band_rows", C.c_int),
                ("ledger_detail", C.c_int), ("strict_geometry", C.c_int), ("tile_entries", C.c_int),
                ("wall_order", C.c_int)]


class Info(C.Structure):
    _fields_ = [("n_nodes", C.c_int64), ("n_gas", C.c_int64), ("n_inlet", C.c_int64),
                ("n_outlet", C.c_int64), ("n_wall", C.c_int64), ("n_solid", C.c_int64),
                ("stencil_counts", C.c_int64 * 6), ("ns", C.c_int), ("T_ref_lat", C.c_double),
                ("steps", C.c_int64), ("device_bytes", C.c_size_t)]


class Balance(C.Structure):
    _fields_ = [("steps", C.c_int64), ("E_gas", C.c_double), ("E_gas0", C.c_double),
                ("H_solid", C.c_double), ("H_solid0", C.c_double), ("Q_reaction", C.c_double),
                ("Q_wall", C.c_double), ("Q_couple", C.c_double), ("Q_fixedT", C.c_double),
                ("residual", C.c_double), ("solid_residual", C.c_double),
                ("eps_paper", C.c_double), ("noconv", C.c_double),
                ("mass", C.c_double * MAX_NS), ("mass0", C.c_double * MAX_NS),
                ("moles", C.c_double * MAX_NS), ("moles0", C.c_double * MAX_NS),
                ("E_pop", C.c_double), ("E_pop0", C.c_double), ("Q_inlet", C.c_double),
                ("Q_outlet", C.c_double), ("D_interp", C.c_double), ("D_collision", C.c_double),
                ("D_coupling", C.c_double), ("D_solid", C.c_double), ("closure", C.c_double),
                ("ledger_detail", C.c_int)]


_lib = None
# fdlbm_moments_ex flag: T and T_s as deviations from the inlet temperature (K).
MOMENTS_T_DEVIATION = 1

EXPORTS = ("fdlbm_create", "fdlbm_step", "fdlbm_sync", "fdlbm_moments", "fdlbm_moments_ex", "fdlbm_populations",
           "fdlbm_enthalpy_balance", "fdlbm_residual", "fdlbm_set_fields", "fdlbm_info",
           "fdlbm_profile", "fdlbm_kernel_times", "fdlbm_totals_static", "fdlbm_save",
           "fdlbm_load", "fdlbm_batch_create", "fdlbm_batch_step", "fdlbm_batch_remove",
           "fdlbm_batch_size", "fdlbm_batch_destroy", "fdlbm_destroy", "fdlbm_last_error")


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfdlbm.so (building it with nvcc if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"solver library not built: {path}")
    L = C.CDLL(path)
    P = C.POINTER
    L.fdlbm_create.argtypes = [P(Geometry), P(Species), C.c_int, P(Transport), P(Kinetics),
                               P(Fields), P(Options), P(C.c_void_p)]
    L.fdlbm_step.argtypes = [C.c_void_p, C.c_int64]
    L.fdlbm_sync.argtypes = [C.c_void_p]
    L.fdlbm_moments.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.fdlbm_moments_ex.argtypes = [C.c_void_p, C.c_uint, C.c_void_p, C.c_int]
    L.fdlbm_populations.argtypes = [C.c_void_p, C.c_void_p, C.c_int]
    L.fdlbm_enthalpy_balance.argtypes = [C.c_void_p, P(Balance)]
    L.fdlbm_residual.argtypes = [C.c_void_p, P(C.c_double)]
    L.fdlbm_set_fields.argtypes = [C.c_void_p, P(Fields)]
    L.fdlbm_info.argtypes = [C.c_void_p, P(Info)]
    L.fdlbm_profile.argtypes = [C.c_void_p, C.c_int]
    L.fdlbm_kernel_times.argtypes = [C.c_void_p, P(C.c_double), P(C.c_int64)]
    L.fdlbm_totals_static.argtypes = [C.c_void_p, P(C.c_double), C.c_int]
    L.fdlbm_save.argtypes = [C.c_void_p, C.c_char_p]
    L.fdlbm_load.argtypes = [C.c_void_p, C.c_char_p]
    L.fdlbm_batch_create.argtypes = [P(C.c_void_p), C.c_int, P(C.c_void_p)]
    L.fdlbm_batch_step.argtypes = [C.c_void_p, C.c_int64]
    L.fdlbm_batch_remove.argtypes = [C.c_void_p, C.c_void_p]
    L.fdlbm_batch_size.argtypes = [C.c_void_p]
    L.fdlbm_batch_destroy.argtypes = [C.c_void_p]
    L.fdlbm_destroy.argtypes = [C.c_void_p]
    L.fdlbm_destroy.restype = None
    L.fdlbm_last_error.restype = C.c_char_p
    for name in EXPORTS[:-2]:
        getattr(L, name).restype = C.c_int
    L.fdlbm_batch_destroy.restype = None
    _lib = L
    return L


def _check(status: int):
    if status != 0:
        raise FdlbmError(status, load().fdlbm_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _fields(init, keep):
    f = Fields()
    if not init:
        return f
    for key, name in (("X", "X"), ("u", "u"), ("T_K", "T_K"), ("Ts_K", "Ts_K"), ("C", "C")):
        if init.get(key) is not None:
            a = np.ascontiguousarray(init[key], dtype=np.float64)
            keep.append(a)
            setattr(f, name, _dptr(a))
    return f


def create_args(p: dict, keep: list):
    """The C structs of fdlbm_create for a problem dict: geometry, species array, species
    count, transport, kinetics and initial fields (argument marshalling only; arrays the
    structs point into are appended to ``keep``)."""
    g = Geometry()
    g.nx, g.ny, g.lattice = p["nx"], p["ny"], p["lattice"]
    g.nz = p["nz"] if p["dim"] == 3 else 1
    mask = np.ascontiguousarray(p["mask"], dtype=np.uint8)
    keep.append(mask)
    g.mask = mask.ctypes.data_as(C.POINTER(C.c_uint8))
    for f in range(6):
        g.face_bc[f] = p["face_bc"][f] if f < len(p["face_bc"]) else 0
    if p.get("wall_u") is not None:
        wu = np.ascontiguousarray(p["wall_u"], dtype=np.float64)
        keep.append(wu)
        g.wall_u = _dptr(wu)
    sp = p["species"]
    ns = len(sp)
    spec = (Species * ns)()
    for j, d in enumerate(sp):
        Drow = (C.c_double * MAX_NS)(*[float(v) for v in d.get("D", [])][:MAX_NS])
        spec[j] = Species(d["M_gmol"], d["tau1"], d["tau2"], d["X_init"], d["X_inlet"],
                          float(d.get("mu", 0.0)), Drow)
    tr = Transport(p["Pr"], int(p["energy_correction"]), p["T0_K"], p["T_init_K"],
                   p["T_inlet_K"], p["T_solid_init_K"], p["T_outer_K"], p["u_inlet"],
                   int(p["inlet_profile"]), p["alpha_s"], p["rhocp_s"], p["kappa_f"],
                   int(p["coupling"]), int(p.get("local_tau", 0)))
    kin = Kinetics()
    kin.n_react = len(p["reactions"])
    for r, d in enumerate(p["reactions"]):
        for j, v in enumerate(d["nu"]):
            kin.nu[r][j] = int(v)
        kin.k0[r], kin.Ea_Jmol[r], kin.Keq[r], kin.dH_Jmol[r] = (
            d["k0"], d["Ea_Jmol"], d["Keq"], d["dH_Jmol"])
        kin.rate_form[r] = int(d["rate_form"])
    kin.rho_w_tol = p["rho_w_tol"]
    kin.rho_w_maxit = int(p["rho_w_maxit"])
    fields = _fields(p.get("init"), keep)
    return g, spec, ns, tr, kin, fields


class Solver:
    """One coupled FD-LBM problem on one GPU, built from a problem dict (see
    ``paper_1804_07588_gb300.workloads``). storage: "fp32", "bf16" or "fp16" population
    storage (FP32 arithmetic in every case). The D2Q9 step kernel's block order:
    band_rows, rows per band and height of the gas tiles (0: 16); tile_entries, gas
    nodes per tile and block size (0: 256; a multiple of 32 in [64, 256]); wall_order, 0
    wall blocks after each band's gas tiles, 1 after all of them. band_rows="auto" takes
    all three from the autotuner's table. ledger_detail: every step also keeps the exact
    energy accounts of ``balance()`` (FP32 storage, constant relaxation times).
    strict_geometry: reject geometries whose pulls need the linear or no-interpolation
    fallbacks (concave corners, narrow gaps) with FDLBM_EGEOM."""

    STORAGE = {"fp32": 0, "bf16": 1, "fp16": 2}

    def __init__(self, p: dict, device: int = 0, stream=None, storage: str = "fp32", band_rows: int = 0,
                 ledger_detail: bool = False, strict_geometry: bool = False, tile_entries: int = 0,
                 wall_order: int = 0):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("fdlbm.Solver needs a CUDA device (no CPU fallback)")
        if (p["dim"], p["lattice"]) not in ((2, 9), (3, 19)):
            raise FdlbmError(-1, "problems are D2Q9 (dim 2) or D3Q19 (dim 3)")
        L = load()
        self._torch = torch
        self.device = device
        torch.cuda.set_device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        keep = []
        g, spec, ns, tr, kin, fields = create_args(p, keep)

        # torch's caching allocator on the solver's stream
        self._blocks = {}

        def _alloc(nbytes, ctx):
            try:
                ptr = torch.cuda.caching_allocator_alloc(int(nbytes), device, self.stream)
            except Exception:
                return None
            self._blocks[ptr] = nbytes
            return ptr

        def _free(ptr, nbytes, ctx):
            if ptr in self._blocks:
                del self._blocks[ptr]
                torch.cuda.caching_allocator_delete(ptr)

        self._alloc_cb = ALLOC_FN(_alloc)
        self._free_cb = FREE_FN(_free)
        if storage not in self.STORAGE:
            raise FdlbmError(-1, f"storage must be one of {sorted(self.STORAGE)}")
        self.storage = storage
        if band_rows == "auto":
            from . import autotune
            band_rows, tile_entries, wall_order = autotune.lookup(p, storage)
        self.band_rows = int(band_rows)
        self.tile_entries = int(tile_entries)
        self.wall_order = int(wall_order)
        opts = Options(self.STORAGE[storage], device, C.c_void_p(self.stream.cuda_stream), self._alloc_cb,
                       self._free_cb, None, self.band_rows, int(bool(ledger_detail)), int(bool(strict_geometry)),
                       self.tile_entries, self.wall_order)
        h = C.c_void_p()
        _check(L.fdlbm_create(C.byref(g), spec, ns, C.byref(tr), C.byref(kin), C.byref(fields),
                              C.byref(opts), C.byref(h)))
        self._h = h
        self.ns = ns
        self.dim = p["dim"]
        self.Q = 9 if self.dim == 2 else 19
        self.nx, self.ny = p["nx"], p["ny"]
        self.nz = p["nz"] if self.dim == 3 else 1
        self.n = self.nx * self.ny * self.nz
        sp = p["species"]
        m = np.array([d["M_gmol"] for d in sp], np.float64)
        self._M_lat = m / m.min()
        self._X_init = np.array([d["X_init"] for d in sp], np.float64)
        self._T_init = float(p["T_init_K"])
        self._T_in = float(p["T_inlet_K"])
        self._solid = np.asarray(p["mask"]).reshape(-1) > 0

    # -- life cycle ---------------------------------------------------------------
    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().fdlbm_destroy(h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- calls ----------------------------------------------------------------------
    def step(self, n: int = 1):
        _check(load().fdlbm_step(self._h, int(n)))

    def sync(self):
        _check(load().fdlbm_sync(self._h))

    @property
    def nfields(self) -> int:
        return 2 * self.ns + 2 + self.dim

    def moments(self, out=None, t_dev: bool = False):
        """[2 ns + 2 + D, n] float32: rho_j, X_j, ux, uy (, uz), T (K), T_s (K); with
        ``t_dev`` T and T_s are deviations from the inlet temperature (K). Returns a CUDA
        tensor (``out`` may be a preallocated CUDA tensor or a numpy float32 array)."""
        torch = self._torch
        nf = self.nfields
        flags = MOMENTS_T_DEVIATION if t_dev else 0
        if out is None:
            out = torch.empty((nf, self.n), dtype=torch.float32, device=f"cuda:{self.device}")
        if isinstance(out, np.ndarray):
            assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == nf * self.n
            _check(load().fdlbm_moments_ex(self._h, flags, out.ctypes.data_as(C.c_void_p), 0))
            return out
        assert out.is_cuda and out.dtype == torch.float32 and out.is_contiguous() and out.numel() == nf * self.n
        _check(load().fdlbm_moments_ex(self._h, flags, C.c_void_p(out.data_ptr()), 1))
        return out

    def moments_host(self, t_dev: bool = False) -> np.ndarray:
        out = np.empty((self.nfields, self.n), np.float32)
        return self.moments(out, t_dev)

    def populations(self) -> np.ndarray:
        out = np.empty((self.ns, self.Q, self.n), np.float32)
        _check(load().fdlbm_populations(self._h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def balance(self) -> dict:
        b = Balance()
        _check(load().fdlbm_enthalpy_balance(self._h, C.byref(b)))
        ns = self.ns
        d = {k: getattr(b, k) for k, _ in Balance._fields_ if k not in ("mass", "mass0", "moles", "moles0")}
        for k in ("mass", "mass0", "moles", "moles0"):
            d[k] = np.array(list(getattr(b, k))[:ns])
        return d

    def residual(self) -> float:
        r = C.c_double()
        _check(load().fdlbm_residual(self._h, C.byref(r)))
        return r.value

    def totals_static(self) -> dict:
        """E_gas, H_solid, mass[ns], moles[ns] of the current time through the
        allocation-free reduction (fixed-order sums in the library's static device
        scratch); same quantities as balance(). Calls must not overlap in time."""
        ns = self.ns
        out = np.empty(2 + 2 * ns, np.float64)
        _check(load().fdlbm_totals_static(self._h, out.ctypes.data_as(C.POINTER(C.c_double)), out.size))
        return {"E_gas": float(out[0]), "H_solid": float(out[1]),
                "mass": out[2:2 + ns].copy(), "moles": out[2 + ns:].copy()}

    def save(self, path: str):
        """Checkpoint the state the next step reads to the file at path."""
        _check(load().fdlbm_save(self._h, os.fsencode(path)))

    def load_state(self, path: str):
        """Restore a checkpoint written by a solver of the same problem."""
        _check(load().fdlbm_load(self._h, os.fsencode(path)))

    def restart_fields(self) -> dict:
        """The current state as initial fields for set_fields (or for another solver of
        the same geometry): mole fractions, velocity, gas and solid temperature (K) and
        molar concentration, with the create-time defaults where a field is undefined
        (gas fields on solid nodes and the reverse)."""
        ns, D = self.ns, self.dim
        m = self.moments_host(t_dev=True).astype(np.float64)  # temperatures as deviations
        rho, X = m[:ns], m[ns:2 * ns]
        T, Ts = m[2 * ns + D] + self._T_in, m[2 * ns + D + 1] + self._T_in
        gas = X.sum(axis=0) > 0
        solid = self._solid
        C_lat = (rho / self._M_lat[:, None]).sum(axis=0)
        X = np.where(gas[None, :], X, self._X_init[:, None])
        return {"X": X, "u": np.where(gas[None, :], m[2 * ns:2 * ns + D], 0.0),
                "T_K": np.where(gas, T, self._T_init), "Ts_K": np.where(solid, Ts, self._T_init),
                "C": np.where(gas, C_lat, 1.0)}

    def set_fields(self, init: dict):
        keep = []
        f = _fields(init, keep)
        _check(load().fdlbm_set_fields(self._h, C.byref(f)))

    def profile(self, enable: bool = True):
        _check(load().fdlbm_profile(self._h, int(bool(enable))))

    def kernel_times(self):
        """(ms of the step kernel summed since profile(), timed steps)."""
        ms = (C.c_double * 2)()
        n = C.c_int64()
        _check(load().fdlbm_kernel_times(self._h, ms, C.byref(n)))
        return ms[0], n.value

    def info(self) -> dict:
        i = Info()
        _check(load().fdlbm_info(self._h, C.byref(i)))
        d = {k: getattr(i, k) for k, _ in Info._fields_}
        d["stencil_counts"] = list(i.stencil_counts)
        return d


class Batch:
    """Several Solvers (same device, species count, storage and energy-correction switch)
    advanced together: one kernel launch per time step for all of them, replayed from a
    captured CUDA graph. Destroy (close) the batch before its solvers."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s._h.value for s in self.solvers])
        b = C.c_void_p()
        _check(load().fdlbm_batch_create(arr, len(self.solvers), C.byref(b)))
        self._b = b

    def step(self, n: int = 1):
        _check(load().fdlbm_batch_step(self._b, int(n)))

    def remove(self, solver):
        _check(load().fdlbm_batch_remove(self._b, solver._h))
        self.solvers = [s for s in self.solvers if s is not solver]

    def __len__(self):
        return load().fdlbm_batch_size(self._b)

    def run_to_steady(self, tol: float = 1e-6, every: int = 500, max_steps: int = 200_000) -> list:
        """Advance the batch until every member's steady-state residual (``Solver.residual``,
        the largest field change per step relative to the field) is below tol: every
        `every` steps the residual of each member still in the batch is read, and members
        below tol, or unstable, are removed so that the remaining launches cover only the
        others. Stops after max_steps. Returns, per member in the original order, {steps,
        residual, converged, unstable}."""
        members = list(self.solvers)
        out = {id(s): {"steps": 0, "residual": float("inf"), "converged": False, "unstable": False}
               for s in members}
        for s in members:
            s.residual()  # snapshot the moments the first change is measured against
        steps = 0
        active = list(members)
        while active and steps < max_steps:
            n = min(every, max_steps - steps)
            self.step(n)
            steps += n
            for s in list(active):
                rec = out[id(s)]
                rec["steps"] = steps
                try:
                    r = s.residual()
                except FdlbmError:
                    r = float("nan")
                rec["residual"] = r
                if not np.isfinite(r):
                    rec["unstable"] = True
                elif r < tol:
                    rec["converged"] = True
                else:
                    continue
                self.remove(s)
                active.remove(s)
        return [out[id(s)] for s in members]

    def close(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            load().fdlbm_batch_destroy(b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
