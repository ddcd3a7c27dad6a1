"""Helpers shared by the GPU parity tests: run the CUDA solver and the FP64 oracle on the
same seeded problem and compare their moment fields."""
import numpy as np

import oracle

# Field-normalised tolerance on every moment field: max |gpu - oracle| / max |oracle|.
TOL = 1e-5

FIELD_NAMES = None


def field_names(ns):
    return ([f"rho_{j}" for j in range(ns)] + [f"X_{j}" for j in range(ns)] +
            ["ux", "uy", "T", "Ts"])


def field_errors(m_gpu, m_ora, classes, ns, vector_u=False):
    """Per-field max |gpu - oracle| / max |oracle| over gas nodes (T_s: solid nodes). With
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


def assert_parity(s, o, tol=TOL, what="", vector_u=False):
    m_gpu = s.moments_host()
    m_ora = o.moments()
    errs = field_errors(m_gpu, m_ora, o.classes(), o.ns, vector_u)
    worst = max(errs.values())
    assert worst <= tol, f"{what} worst {worst:.3e} > {tol:.1e}: " + \
        ", ".join(f"{k}={v:.2e}" for k, v in errs.items())
    return errs
