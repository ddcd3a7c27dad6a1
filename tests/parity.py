"""Helpers shared by the GPU parity tests: run the CUDA solver and the FP64 oracle on the
same seeded problem and compare their moment fields."""
import numpy as np

import oracle

# Field-normalised tolerance on every moment field: max |gpu - oracle| / max |oracle|.
TOL = 1e-5
# FP32 resolution floor of the temperatures, relative to the inlet temperature: the
# solver carries T in FP32 populations whose velocity-carrying parts (|h| up to ~0.4 in
# a channel at u = 0.02) are rounded at ~1e-8 every step, a noise that accumulates like
# a random walk to ~4e-4 K after 1000 steps (30 ulps of T at 500 K). A temperature
# passes when its deviation-normalised error is within TOL or its absolute error within
# T_FLOOR_REL * T_in (1 mK at 500 K).
T_FLOOR_REL = 2e-6

FIELD_NAMES = None


def field_names(ns):
    return ([f"rho_{j}" for j in range(ns)] + [f"X_{j}" for j in range(ns)] +
            ["ux", "uy", "T", "Ts"])


def temperature_scale(dev):
    """Scale of a temperature field given as its deviation from the inlet temperature:
    max |T - T_in| (the scheme's temperature signal is its departure from the inlet
    state, a few kelvin against 500 K), or 1 K where the field does not depart from T_in
    at all (an isothermal problem)."""
    s = float(np.abs(dev).max()) if dev.size else 0.0
    return s if s > 1e-9 else 1.0


def field_errors(m_gpu, m_ora, classes, ns, vector_u=False, T_in=None):
    """Per-field max |gpu - oracle| / max |oracle| over gas nodes (T_s: solid nodes). With
    T_in, the GPU's T and T_s are deviations from T_in (``moments_host(t_dev=True)``) and
    are compared with the oracle's T - T_in, normalised by max |T_oracle - T_in|. With
    vector_u the velocity is one vector field: both components are normalised by the
    maximum speed (for flows where one component is zero up to rounding)."""
    gas = classes == 0
    solid = classes >= 3
    u_scale = np.sqrt((np.asarray(m_ora[2 * ns:2 * ns + 2][:, gas], np.float64) ** 2).sum(0)).max()
    errs = {}
    for f, name in enumerate(field_names(ns)):
        sel = solid if name == "Ts" else gas
        if not sel.any():
            continue
        a = np.asarray(m_ora[f][sel], np.float64)
        b = np.asarray(m_gpu[f][sel], np.float64)
        if T_in is not None and name in ("T", "Ts"):
            a = a - T_in
            scale = temperature_scale(a)
        else:
            scale = u_scale if (vector_u and name in ("ux", "uy")) else np.abs(a).max()
        errs[name] = float(np.abs(a - b).max() / scale) if scale > 0 else float(np.abs(b).max())
    return errs


def run_both(p, steps, chunks=1):
    from paper_1804_07588_gb300 import fdlbm
    s = fdlbm.Solver(p)
    o = oracle.Oracle(p)
    per = steps // chunks
    for _ in range(chunks):
        s.step(per)
        o.step(per)
    s.sync()
    return s, o


def temperature_abs_errors(m_gpu, m_ora, classes, ns, T_in):
    """max |T_gpu - T_oracle| in kelvin over gas nodes (T) and solid nodes (T_s), the GPU's
    temperatures given as deviations from T_in."""
    out = {}
    for f, name, sel in ((2 * ns + 2, "T", classes == 0), (2 * ns + 3, "Ts", classes >= 3)):
        if sel.any():
            out[name] = float(np.abs(np.asarray(m_gpu[f][sel], np.float64) - (m_ora[f][sel] - T_in)).max())
    return out


def check_fields(errs, abs_T, T_in, tol, what):
    """Every field within tol; a temperature also passes within the FP32 floor."""
    floor = T_FLOOR_REL * T_in
    bad = {k: v for k, v in errs.items() if v > tol and not (k in abs_T and abs_T[k] <= floor)}
    assert not bad, f"{what} over {tol:.1e}: " + ", ".join(f"{k}={v:.2e}" for k, v in errs.items()) + \
        "; |dT| K: " + ", ".join(f"{k}={v:.2e}" for k, v in abs_T.items()) + f" (floor {floor:.1e} K)"


def assert_parity(s, o, tol=TOL, what="", vector_u=False):
    m_gpu = s.moments_host(t_dev=True)
    m_ora = o.moments()
    errs = field_errors(m_gpu, m_ora, o.classes(), o.ns, vector_u, T_in=o.T_inlet_K)
    abs_T = temperature_abs_errors(m_gpu, m_ora, o.classes(), o.ns, o.T_inlet_K)
    check_fields(errs, abs_T, o.T_inlet_K, tol, what)
    return errs
