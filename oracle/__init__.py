"""ctypes wrapper of the plain FP64 CPU oracles of the scheme (``fdlbm_oracle.c``,
D2Q9, and ``fdlbm_oracle3d.c``, D3Q19); ``oracle.surrogate`` holds the FP64 oracle of
the learned warm start's network.

TEST INFRASTRUCTURE ONLY. Imported by the test-suite, the package smoke check and the
benchmark's CPU-baseline / reference leg; the solver library never loads it. It builds
with plain ``gcc`` into ``oracle/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "fdlbm_oracle.c"), os.path.join(_HERE, "fdlbm_oracle3d.c")]
_HDRS = [os.path.join(_HERE, "fdlbm_oracle.h"), os.path.join(_HERE, "fdlbm_oracle3d.h")]
_LIB = os.path.join(_HERE, "liboracle.so")

MAX_NS = 8
MAX_NR = 4
Q = 9

# Ledger indices (mirror the enum in fdlbm_oracle.h)
B_STEPS, B_E_GAS, B_E_GAS0, B_H_SOLID, B_H_SOLID0, B_Q_RXN, B_Q_WALL, B_Q_COUPLE, \
    B_Q_FIXEDT, B_RESIDUAL, B_SOLID_RESIDUAL, B_EPS_PAPER, B_NOCONV, B_MASS = range(14)
A_E_POP, A_E_POP0, A_Q_INLET, A_Q_OUTLET, A_D_INTERP, A_D_COLLISION, A_D_COUPLING, A_CLOSURE, \
    A_MASS = range(9)


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle into a shared library (plain C99, -O2, FP-contract off so the
    FP64 arithmetic follows the source order)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(f) for f in _SRCS + _HDRS):
        cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", _LIB + ".tmp", *_SRCS, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("mask", C.POINTER(C.c_ubyte)),
        ("face_bc", C.c_int * 4),
        ("ns", C.c_int),
        ("M_gmol", C.c_double * MAX_NS), ("tau1", C.c_double * MAX_NS),
        ("tau2", C.c_double * MAX_NS), ("X_init", C.c_double * MAX_NS),
        ("X_inlet", C.c_double * MAX_NS),
        ("Pr", C.c_double), ("energy_correction", C.c_int),
        ("T0_K", C.c_double), ("T_init_K", C.c_double), ("T_inlet_K", C.c_double),
        ("T_solid_init_K", C.c_double), ("T_outer_K", C.c_double),
        ("u_inlet", C.c_double), ("inlet_profile", C.c_int),
        ("alpha_s", C.c_double), ("rhocp_s", C.c_double), ("kappa_f", C.c_double),
        ("coupling", C.c_int),
        ("nr", C.c_int),
        ("nu", (C.c_int * MAX_NS) * MAX_NR),
        ("k0", C.c_double * MAX_NR), ("Ea_Jmol", C.c_double * MAX_NR),
        ("Keq", C.c_double * MAX_NR), ("dH_Jmol", C.c_double * MAX_NR),
        ("rate_form", C.c_int * MAX_NR),
        ("rho_w_tol", C.c_double), ("rho_w_maxit", C.c_int),
        ("init_X", C.POINTER(C.c_double)), ("init_u", C.POINTER(C.c_double)),
        ("init_T", C.POINTER(C.c_double)), ("init_Ts", C.POINTER(C.c_double)),
        ("init_C", C.POINTER(C.c_double)),
        ("local_tau", C.c_int), ("mu", C.c_double * MAX_NS), ("Djk", (C.c_double * MAX_NS) * MAX_NS),
        ("wall_u", C.POINTER(C.c_double)),
        ("phi_lagged", C.c_int),
    ]


class _Problem3(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
        ("mask", C.POINTER(C.c_ubyte)),
        ("face_bc", C.c_int * 6),
        ("ns", C.c_int),
        ("M_gmol", C.c_double * MAX_NS), ("tau1", C.c_double * MAX_NS),
        ("tau2", C.c_double * MAX_NS), ("X_init", C.c_double * MAX_NS),
        ("X_inlet", C.c_double * MAX_NS),
        ("Pr", C.c_double), ("energy_correction", C.c_int),
        ("T0_K", C.c_double), ("T_init_K", C.c_double), ("T_inlet_K", C.c_double),
        ("T_solid_init_K", C.c_double), ("T_outer_K", C.c_double),
        ("u_inlet", C.c_double),
        ("alpha_s", C.c_double), ("rhocp_s", C.c_double), ("kappa_f", C.c_double),
        ("coupling", C.c_int),
        ("nr", C.c_int),
        ("nu", (C.c_int * MAX_NS) * MAX_NR),
        ("k0", C.c_double * MAX_NR), ("Ea_Jmol", C.c_double * MAX_NR),
        ("Keq", C.c_double * MAX_NR), ("dH_Jmol", C.c_double * MAX_NR),
        ("rate_form", C.c_int * MAX_NR),
        ("rho_w_tol", C.c_double), ("rho_w_maxit", C.c_int),
        ("init_X", C.POINTER(C.c_double)), ("init_u", C.POINTER(C.c_double)),
        ("init_T", C.POINTER(C.c_double)), ("init_Ts", C.POINTER(C.c_double)),
        ("init_C", C.POINTER(C.c_double)),
        ("phi_lagged", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        L.ora_create.restype = C.c_void_p
        L.ora_create.argtypes = [C.POINTER(_Problem), C.c_char_p, C.c_int]
        L.ora_destroy.argtypes = [C.c_void_p]
        L.ora_step.argtypes = [C.c_void_p, C.c_int]
        L.ora_nfields.argtypes = [C.c_void_p]
        L.ora_moments.argtypes = [C.c_void_p, dp]
        L.ora_populations.argtypes = [C.c_void_p, dp]
        L.ora_balance.argtypes = [C.c_void_p, dp]
        L.ora_accounts.argtypes = [C.c_void_p, dp]
        L.ora_residual.argtypes = [C.c_void_p, C.c_int]
        L.ora_residual.restype = C.c_double
        L.ora_counts.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
        L.ora_get_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.ora_set_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.ora_classes.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        L.ora_equilibrium.argtypes = [C.c_double] * 5 + [dp]
        L.ora_interp.argtypes = [C.c_int] + [C.c_double] * 6
        L.ora_interp.restype = C.c_double
        L.ora_psi.argtypes = [C.c_double, dp, dp]
        L.ora_phi.argtypes = [C.c_double, dp]
        L.ora_uc.argtypes = [C.c_int, dp, dp, dp, C.c_double]
        L.ora_uc.restype = C.c_double
        L.ora_collide.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp, dp]
        L.ora_units.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.ora_wilke_phi.argtypes = [C.c_double] * 4
        L.ora_wilke_phi.restype = C.c_double
        L.ora_local_tau.argtypes = [C.c_int, dp, dp, dp, dp, C.c_double, dp, dp]
        L.ora3_create.restype = C.c_void_p
        L.ora3_create.argtypes = [C.POINTER(_Problem3), C.c_char_p, C.c_int]
        L.ora3_destroy.argtypes = [C.c_void_p]
        L.ora3_step.argtypes = [C.c_void_p, C.c_int]
        L.ora3_nfields.argtypes = [C.c_void_p]
        L.ora3_moments.argtypes = [C.c_void_p, dp]
        L.ora3_populations.argtypes = [C.c_void_p, dp]
        L.ora3_get_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.ora3_set_state.argtypes = [C.c_void_p, dp, dp, dp]
        L.ora3_balance.argtypes = [C.c_void_p, dp]
        L.ora3_accounts.argtypes = [C.c_void_p, dp]
        L.ora3_residual.argtypes = [C.c_void_p, C.c_int]
        L.ora3_residual.restype = C.c_double
        L.ora3_counts.argtypes = [C.c_void_p, C.POINTER(C.c_long)]
        L.ora3_classes.argtypes = [C.c_void_p, C.POINTER(C.c_int)]
        L.ora3_velocity.argtypes = [C.c_int, C.POINTER(C.c_int)]
        L.ora3_interp.argtypes = [C.c_int] + [C.c_double] * 6
        L.ora3_interp.restype = C.c_double
        L.ora3_equilibrium.argtypes = [C.c_double] * 6 + [dp]
        L.ora3_psi.argtypes = [C.c_double, dp, dp, dp]
        L.ora3_phi.argtypes = [C.c_double, dp]
        L.ora3_collide.argtypes = [C.c_int, dp, dp, dp, dp, dp, dp, dp]
        _lib = L
    return _lib


def _accounts_dict(out, ns):
    m = out[A_MASS:].reshape(8, ns)
    d = {"E_pop": out[A_E_POP], "E_pop0": out[A_E_POP0], "Q_inlet": out[A_Q_INLET],
         "Q_outlet": out[A_Q_OUTLET], "D_interp": out[A_D_INTERP],
         "D_collision": out[A_D_COLLISION], "D_coupling": out[A_D_COUPLING],
         "closure": out[A_CLOSURE]}
    for r, name in enumerate(("M_pop", "M_pop0", "M_inlet", "M_outlet", "Dm_interp",
                              "Dm_collision", "M_rxn", "mass_closure")):
        d[name] = m[r].copy()
    return d


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class Oracle:
    """FP64 CPU solver for one problem dict (see ``paper_1804_07588_gb300.workloads``)."""

    def __init__(self, p: dict):
        if p["dim"] != 2 or p["lattice"] != 9:
            raise NotImplementedError("the oracle covers D2Q9")
        L = lib()
        s = _Problem()
        s.nx, s.ny = p["nx"], p["ny"]
        self._mask = np.ascontiguousarray(p["mask"], dtype=np.uint8)
        s.mask = self._mask.ctypes.data_as(C.POINTER(C.c_ubyte))
        for f in range(4):
            s.face_bc[f] = p["face_bc"][f]
        sp = p["species"]
        s.ns = len(sp)
        for j, d in enumerate(sp):
            s.M_gmol[j] = d["M_gmol"]
            s.tau1[j] = d["tau1"]
            s.tau2[j] = d["tau2"]
            s.X_init[j] = d["X_init"]
            s.X_inlet[j] = d["X_inlet"]
        for k in ("Pr", "T0_K", "T_init_K", "T_inlet_K", "T_solid_init_K", "T_outer_K",
                  "u_inlet", "alpha_s", "rhocp_s", "kappa_f", "rho_w_tol"):
            setattr(s, k, float(p[k]))
        for k in ("energy_correction", "inlet_profile", "coupling", "rho_w_maxit"):
            setattr(s, k, int(p[k]))
        s.phi_lagged = int(p.get("phi_lagged", 0))
        rx = p["reactions"]
        s.nr = len(rx)
        for r, d in enumerate(rx):
            for j, v in enumerate(d["nu"]):
                s.nu[r][j] = int(v)
            s.k0[r], s.Ea_Jmol[r], s.Keq[r], s.dH_Jmol[r] = d["k0"], d["Ea_Jmol"], d["Keq"], d["dH_Jmol"]
            s.rate_form[r] = d["rate_form"]
        self._keep = []
        init = p.get("init") or {}
        for key, field in (("X", "init_X"), ("u", "init_u"), ("T_K", "init_T"), ("Ts_K", "init_Ts"),
                           ("C", "init_C")):
            if init.get(key) is not None:
                a = np.ascontiguousarray(init[key], dtype=np.float64)
                self._keep.append(a)
                setattr(s, field, _dptr(a))
        if p.get("wall_u") is not None:
            wu = np.ascontiguousarray(p["wall_u"], dtype=np.float64)
            self._keep.append(wu)
            s.wall_u = _dptr(wu)
        if p.get("local_tau"):
            s.local_tau = 1
            for j, d in enumerate(sp):
                s.mu[j] = d["mu"]
                for k, v in enumerate(d["D"]):
                    s.Djk[j][k] = v
        err = C.create_string_buffer(256)
        h = L.ora_create(C.byref(s), err, 256)
        if not h:
            raise ValueError("oracle: " + err.value.decode())
        self._h = C.c_void_p(h)
        self.ns = s.ns
        self.n = s.nx * s.ny
        self.nx, self.ny = s.nx, s.ny
        self.T_inlet_K = float(p["T_inlet_K"])

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ora_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        lib().ora_step(self._h, int(n))

    def moments(self) -> np.ndarray:
        """[2*ns + 4, n]: rho_j, X_j, ux, uy, T (K) on gas nodes, T_s (K) on solid nodes."""
        nf = lib().ora_nfields(self._h)
        out = np.zeros((nf, self.n))
        lib().ora_moments(self._h, _dptr(out))
        return out

    def populations(self) -> np.ndarray:
        out = np.zeros((self.ns, Q, self.n))
        lib().ora_populations(self._h, _dptr(out))
        return out

    def get_state(self):
        """(g [ns][9][n], Ts [n], T [n]) of the current time level (lattice units)."""
        g = np.empty((self.ns, Q, self.n))
        Ts = np.empty(self.n)
        T = np.empty(self.n)
        lib().ora_get_state(self._h, _dptr(g), _dptr(Ts), _dptr(T))
        return g, Ts, T

    def set_state(self, g, Ts, T):
        g = np.ascontiguousarray(g, np.float64)
        Ts = np.ascontiguousarray(Ts, np.float64)
        T = np.ascontiguousarray(T, np.float64)
        assert g.size == self.ns * Q * self.n and Ts.size == self.n and T.size == self.n
        lib().ora_set_state(self._h, _dptr(g), _dptr(Ts), _dptr(T))

    def balance(self) -> dict:
        out = np.zeros(B_MASS + 4 * self.ns)
        lib().ora_balance(self._h, _dptr(out))
        ns = self.ns
        return {
            "steps": out[B_STEPS], "E_gas": out[B_E_GAS], "E_gas0": out[B_E_GAS0],
            "H_solid": out[B_H_SOLID], "H_solid0": out[B_H_SOLID0], "Q_reaction": out[B_Q_RXN],
            "Q_wall": out[B_Q_WALL], "Q_couple": out[B_Q_COUPLE], "Q_fixedT": out[B_Q_FIXEDT],
            "residual": out[B_RESIDUAL], "solid_residual": out[B_SOLID_RESIDUAL],
            "eps_paper": out[B_EPS_PAPER], "noconv": out[B_NOCONV],
            "mass": out[B_MASS:B_MASS + ns].copy(), "mass0": out[B_MASS + ns:B_MASS + 2 * ns].copy(),
            "moles": out[B_MASS + 2 * ns:B_MASS + 3 * ns].copy(),
            "moles0": out[B_MASS + 3 * ns:B_MASS + 4 * ns].copy(),
        }

    def accounts(self) -> dict:
        """Exact accounts of the scheme: inventory of the stored populations, shift-sense
        inlet/outlet fluxes, interpolation/collision/coupling defects and the energy
        closure; per-species mass arrays of the same form (the header's ORA_A_* layout)."""
        ns = self.ns
        out = np.zeros(A_MASS + 8 * ns)
        lib().ora_accounts(self._h, _dptr(out))
        return _accounts_dict(out, ns)

    def residual(self, K: int) -> float:
        return lib().ora_residual(self._h, int(K))

    def counts(self) -> dict:
        out = (C.c_long * 11)()
        lib().ora_counts(self._h, out)
        v = list(out)
        return {"gas": v[0], "inlet": v[1], "outlet": v[2], "wall": v[3], "solid": v[4],
                "stencil": v[5:11]}

    def classes(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        lib().ora_classes(self._h, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out


# ---- point functions (pins) --------------------------------------------------------

def equilibrium(rho, ux, uy, M, T) -> np.ndarray:
    out = np.zeros(Q)
    lib().ora_equilibrium(rho, ux, uy, M, T, _dptr(out))
    return out


def interp(code, c, s3, s2, s1, s0, sp) -> float:
    return lib().ora_interp(code, c, s3, s2, s1, s0, sp)


def psi(c):
    px, py = np.zeros(Q), np.zeros(Q)
    lib().ora_psi(c, _dptr(px), _dptr(py))
    return px, py


def phi(c):
    out = np.zeros(Q)
    lib().ora_phi(c, _dptr(out))
    return out


def wilke_phi(mu_j, mu_k, M_j, M_k) -> float:
    return lib().ora_wilke_phi(mu_j, mu_k, M_j, M_k)


def local_tau(M, mu, Djk, rho, T):
    """(tau1[ns], tau2[ns]) of one node (Eqs. tau1s, tau2_approx_text, D_j_text)."""
    M = np.ascontiguousarray(M, np.float64)
    ns = len(M)
    mu = np.ascontiguousarray(mu, np.float64)
    D = np.zeros((ns, MAX_NS))
    D[:, :ns] = np.asarray(Djk, np.float64)
    rho = np.ascontiguousarray(rho, np.float64)
    t1, t2 = np.zeros(ns), np.zeros(ns)
    lib().ora_local_tau(ns, _dptr(M), _dptr(mu), _dptr(D), _dptr(rho), T, _dptr(t1), _dptr(t2))
    return t1, t2


def units(T0_K, M0_gmol, dx_m):
    """(U' m/s, dt s, kelvin per lattice temperature unit)."""
    out = np.zeros(3)
    lib().ora_units(T0_K, M0_gmol, dx_m, _dptr(out))
    return tuple(out)


def collide(M, tau1, tau2, g, divq):
    """One-node collision: returns (g_out [ns, 9], moments rho_j.., ux, uy, T, Tg)."""
    M = np.ascontiguousarray(M, np.float64)
    ns = len(M)
    t1 = np.ascontiguousarray(tau1, np.float64)
    t2 = np.ascontiguousarray(tau2, np.float64)
    g = np.ascontiguousarray(g, np.float64).reshape(ns, Q)
    dq = np.ascontiguousarray(divq, np.float64)
    go = np.zeros((ns, Q))
    mom = np.zeros(ns + 4)
    lib().ora_collide(ns, _dptr(M), _dptr(t1), _dptr(t2), _dptr(g), _dptr(dq), _dptr(go), _dptr(mom))
    return go, mom


# ---- D3Q19 oracle ------------------------------------------------------------------

Q3 = 19


def _fill_common(s, p, keep):
    sp = p["species"]
    s.ns = len(sp)
    for j, d in enumerate(sp):
        s.M_gmol[j] = d["M_gmol"]
        s.tau1[j] = d["tau1"]
        s.tau2[j] = d["tau2"]
        s.X_init[j] = d["X_init"]
        s.X_inlet[j] = d["X_inlet"]
    for k in ("Pr", "T0_K", "T_init_K", "T_inlet_K", "T_solid_init_K", "T_outer_K",
              "u_inlet", "alpha_s", "rhocp_s", "kappa_f", "rho_w_tol"):
        setattr(s, k, float(p[k]))
    for k in ("energy_correction", "coupling", "rho_w_maxit"):
        setattr(s, k, int(p[k]))
    s.phi_lagged = int(p.get("phi_lagged", 0))
    rx = p["reactions"]
    s.nr = len(rx)
    for r, d in enumerate(rx):
        for j, v in enumerate(d["nu"]):
            s.nu[r][j] = int(v)
        s.k0[r], s.Ea_Jmol[r], s.Keq[r], s.dH_Jmol[r] = d["k0"], d["Ea_Jmol"], d["Keq"], d["dH_Jmol"]
        s.rate_form[r] = d["rate_form"]
    init = p.get("init") or {}
    for key, field in (("X", "init_X"), ("u", "init_u"), ("T_K", "init_T"), ("Ts_K", "init_Ts"),
                       ("C", "init_C")):
        if init.get(key) is not None:
            a = np.ascontiguousarray(init[key], dtype=np.float64)
            keep.append(a)
            setattr(s, field, _dptr(a))


class Oracle3:
    """FP64 CPU solver of the D3Q19 form of the scheme for one 3D problem dict."""

    def __init__(self, p: dict):
        if p["dim"] != 3 or p["lattice"] != 19:
            raise NotImplementedError("Oracle3 covers D3Q19")
        if p.get("inlet_profile", 0) != 0:
            raise NotImplementedError("Oracle3: plug inlet only")
        L = lib()
        s = _Problem3()
        s.nx, s.ny, s.nz = p["nx"], p["ny"], p["nz"]
        self._mask = np.ascontiguousarray(p["mask"], dtype=np.uint8)
        s.mask = self._mask.ctypes.data_as(C.POINTER(C.c_ubyte))
        for f in range(6):
            s.face_bc[f] = p["face_bc"][f]
        self._keep = []
        _fill_common(s, p, self._keep)
        err = C.create_string_buffer(256)
        h = L.ora3_create(C.byref(s), err, 256)
        if not h:
            raise ValueError("oracle3: " + err.value.decode())
        self._h = C.c_void_p(h)
        self.ns = s.ns
        self.nx, self.ny, self.nz = s.nx, s.ny, s.nz
        self.T_inlet_K = float(p["T_inlet_K"])
        self.n = s.nx * s.ny * s.nz

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.ora3_destroy(h)
            self._h = None

    def step(self, n: int = 1):
        lib().ora3_step(self._h, int(n))

    def moments(self) -> np.ndarray:
        """[2*ns + 5, n]: rho_j, X_j, ux, uy, uz, T (K) on gas nodes, T_s (K) on solid nodes."""
        nf = lib().ora3_nfields(self._h)
        out = np.zeros((nf, self.n))
        lib().ora3_moments(self._h, _dptr(out))
        return out

    def populations(self) -> np.ndarray:
        out = np.zeros((self.ns, Q3, self.n))
        lib().ora3_populations(self._h, _dptr(out))
        return out

    def get_state(self):
        """(g [ns][19][n], Ts [n], T [n]) of the current time level (lattice units)."""
        g = np.empty((self.ns, Q3, self.n))
        Ts = np.empty(self.n)
        T = np.empty(self.n)
        lib().ora3_get_state(self._h, _dptr(g), _dptr(Ts), _dptr(T))
        return g, Ts, T

    def set_state(self, g, Ts, T):
        g = np.ascontiguousarray(g, np.float64)
        Ts = np.ascontiguousarray(Ts, np.float64)
        T = np.ascontiguousarray(T, np.float64)
        assert g.size == self.ns * Q3 * self.n and Ts.size == self.n and T.size == self.n
        lib().ora3_set_state(self._h, _dptr(g), _dptr(Ts), _dptr(T))

    def accounts(self) -> dict:
        """Exact accounts of the D3Q19 scheme (the layout of Oracle.accounts)."""
        ns = self.ns
        out = np.zeros(A_MASS + 8 * ns)
        lib().ora3_accounts(self._h, _dptr(out))
        return _accounts_dict(out, ns)

    def balance(self) -> dict:
        out = np.zeros(B_MASS + 4 * self.ns)
        lib().ora3_balance(self._h, _dptr(out))
        ns = self.ns
        return {
            "steps": out[B_STEPS], "E_gas": out[B_E_GAS], "E_gas0": out[B_E_GAS0],
            "H_solid": out[B_H_SOLID], "H_solid0": out[B_H_SOLID0], "Q_reaction": out[B_Q_RXN],
            "Q_wall": out[B_Q_WALL], "Q_couple": out[B_Q_COUPLE], "Q_fixedT": out[B_Q_FIXEDT],
            "residual": out[B_RESIDUAL], "solid_residual": out[B_SOLID_RESIDUAL],
            "eps_paper": out[B_EPS_PAPER], "noconv": out[B_NOCONV],
            "mass": out[B_MASS:B_MASS + ns].copy(), "mass0": out[B_MASS + ns:B_MASS + 2 * ns].copy(),
            "moles": out[B_MASS + 2 * ns:B_MASS + 3 * ns].copy(),
            "moles0": out[B_MASS + 3 * ns:B_MASS + 4 * ns].copy(),
        }

    def residual(self, K: int) -> float:
        return lib().ora3_residual(self._h, int(K))

    def counts(self) -> dict:
        out = (C.c_long * 11)()
        lib().ora3_counts(self._h, out)
        v = list(out)
        return {"gas": v[0], "inlet": v[1], "outlet": v[2], "wall": v[3], "solid": v[4],
                "stencil": v[5:11]}

    def classes(self) -> np.ndarray:
        out = np.zeros(self.n, np.int32)
        lib().ora3_classes(self._h, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out


def interp3(code, c, s3, s2, s1, s0, sp) -> float:
    return lib().ora3_interp(code, c, s3, s2, s1, s0, sp)


def velocities3() -> np.ndarray:
    """[19, 3] lattice velocities of the D3Q19 oracle, in its direction order."""
    out = np.zeros((Q3, 3), np.int64)
    v = (C.c_int * 3)()
    for i in range(Q3):
        lib().ora3_velocity(i, v)
        out[i] = list(v)
    return out


def equilibrium3(rho, ux, uy, uz, M, T) -> np.ndarray:
    out = np.zeros(Q3)
    lib().ora3_equilibrium(rho, ux, uy, uz, M, T, _dptr(out))
    return out


def psi3(c):
    px, py, pz = np.zeros(Q3), np.zeros(Q3), np.zeros(Q3)
    lib().ora3_psi(c, _dptr(px), _dptr(py), _dptr(pz))
    return px, py, pz


def phi3(c):
    out = np.zeros(Q3)
    lib().ora3_phi(c, _dptr(out))
    return out


def collide3(M, tau1, tau2, g, divq):
    """One-node D3Q19 collision: (g_out [ns, 19], moments rho_j.., ux, uy, uz, T, Tg)."""
    M = np.ascontiguousarray(M, np.float64)
    ns = len(M)
    t1 = np.ascontiguousarray(tau1, np.float64)
    t2 = np.ascontiguousarray(tau2, np.float64)
    g = np.ascontiguousarray(g, np.float64).reshape(ns, Q3)
    dq = np.ascontiguousarray(divq, np.float64)
    go = np.zeros((ns, Q3))
    mom = np.zeros(ns + 5)
    lib().ora3_collide(ns, _dptr(M), _dptr(t1), _dptr(t2), _dptr(g), _dptr(dq), _dptr(go), _dptr(mom))
    return go, mom
