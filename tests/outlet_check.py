"""Outlet condition (reading R13) measured on an oracle run: shared by the D2Q9 and
D3Q19 oracle pins."""
import numpy as np


def outlet_condition_errors(p, o, E):
    """Per outlet node: relative error of its pressure C T against the inlet pressure
    (C from the node's stored populations, T of the upstream gas node), and the largest
    differences of its mole fractions and velocity (moments of its populations) from the
    upstream node's; plus the upstream temperatures in K."""
    ns = len(p["species"])
    nd = E.shape[1]
    M = np.array([s["M_gmol"] for s in p["species"]])
    M = M / M.min()
    c = np.sqrt(1.0 / M)
    g, cls, m = o.populations(), o.classes(), o.moments()

    def conc(k):
        return sum(g[j, :, k].sum() / M[j] for j in range(ns))

    inlet = np.where(cls == 1)[0]
    p_in = conc(inlet[len(inlet) // 2]) * p["T_inlet_K"]
    rows = []
    for k in np.where(cls == 2)[0]:
        ku = k - 1                                   # the outlet is the x+ face
        T_up = m[2 * ns + nd][ku]
        rho = np.array([g[j, :, k].sum() for j in range(ns)])
        X = rho / M / (rho / M).sum()
        u = sum(c[j] * (E.T.astype(float) @ g[j, :, k]) for j in range(ns)) / rho.sum()
        rows.append((abs(conc(k) * T_up / p_in - 1.0), np.abs(X - m[ns:2 * ns, ku]).max(),
                     np.abs(u - m[2 * ns:2 * ns + nd, ku]).max(), T_up))
    return np.array(rows)
