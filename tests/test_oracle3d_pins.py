"""Pins of the D3Q19 FP64 oracle against what the mathematics and the paper fix.

The 3D lattice is the paper's announced extension (reading R1b). Each test checks the
oracle against something other than itself: the textbook D3Q19 rest weights, moment
identities of the folded product-form equilibrium and of the correction coefficients,
conservation laws, fixed points, and decay rates of diffusion, entropy and shear modes
against their transport coefficients (including the Prandtl number 5/2 of the
uncorrected 3D model, which pins the 3D reading of the lattice heat-flux correction).
"""
import math

import numpy as np
import pytest

import oracle
from outlet_check import outlet_condition_errors
from paper_1804_07588_gb300 import workloads as W

E = None


def _vel():
    global E
    if E is None:
        E = oracle.velocities3()
    return E


def test_velocity_set_d3q19():
    """Rest, the 6 axis links and the 12 face diagonals, each with its opposite."""
    e = _vel()
    assert e.shape == (19, 3)
    n2 = (e * e).sum(1)
    assert (n2 == 0).sum() == 1 and (n2 == 1).sum() == 6 and (n2 == 2).sum() == 12
    rows = {tuple(v) for v in e}
    assert len(rows) == 19 and all(tuple(-v) in rows for v in e)


def test_equilibrium3_rest_weights():
    """At u = 0 and T = 1/3 the folded equilibrium is the standard D3Q19 lattice
    (weights 1/3, 1/18, 1/36)."""
    e = _vel()
    f = oracle.equilibrium3(1.0, 0.0, 0.0, 0.0, 1.0, 1.0 / 3.0)
    n2 = (e * e).sum(1)
    ref = np.where(n2 == 0, 1 / 3, np.where(n2 == 1, 1 / 18, 1 / 36))
    np.testing.assert_allclose(f, ref, rtol=1e-14)


@pytest.mark.parametrize("M", [1.0, 8.936, 13.894, 21.83])
def test_equilibrium3_moments(M):
    """The folded equilibrium carries the species density, momentum rho u and pressure
    tensor rho (u u + T/M I) (Eq. eq_state_pop moments, reading R1b)."""
    rng = np.random.default_rng(21)
    c = 1.0 / math.sqrt(M)
    cv = c * _vel().astype(float)
    for _ in range(20):
        rho = rng.uniform(0.01, 5.0)
        u = rng.uniform(-0.05, 0.05, 3)
        T = rng.uniform(0.25, 0.4)
        f = oracle.equilibrium3(rho, *u, M, T)
        assert np.isclose(f.sum(), rho, rtol=1e-14)
        np.testing.assert_allclose(cv.T @ f, rho * u, atol=1e-15, rtol=1e-12)
        P = (cv[:, :, None] * cv[:, None, :] * f[:, None, None]).sum(0)
        np.testing.assert_allclose(P, rho * (np.outer(u, u) + np.eye(3) * T / M), atol=1e-15, rtol=1e-12)
        assert (f > 0).all()


def test_equilibrium3_closed_form():
    """Summing the fold by hand: a face diagonal (a, b) keeps rho w(a) w(b) (its two
    corners add rho w(a) w(b) (w(+) + w(-)) and w(0) + w(+) + w(-) = 1); an axis link a
    gets rho w(a) (w0_b w0_c - S_b S_c), the rest rho (w0_x w0_y w0_z + S_x S_y S_z), with
    w0 = 1 - M u^2 - T and S = w(+) + w(-) = M u^2 + T per axis."""
    rng = np.random.default_rng(22)
    e = _vel()
    for _ in range(10):
        M = rng.uniform(1, 22)
        rho = rng.uniform(0.1, 3)
        u = rng.uniform(-0.04, 0.04, 3)
        T = rng.uniform(0.28, 0.38)

        def w(a, v):
            return 1 - M * v * v - T if a == 0 else 0.5 * (a * math.sqrt(M) * v + M * v * v + T)

        S = [M * v * v + T for v in u]
        w0 = [w(0, v) for v in u]
        f = oracle.equilibrium3(rho, *u, M, T)
        for i, v in enumerate(e):
            nz = [ax for ax in range(3) if v[ax] != 0]
            if not nz:
                ref = rho * (w0[0] * w0[1] * w0[2] + S[0] * S[1] * S[2])
            elif len(nz) == 1:
                a = nz[0]
                b, cc = [ax for ax in range(3) if ax != a]
                ref = rho * w(v[a], u[a]) * (w0[b] * w0[cc] - S[b] * S[cc])
            else:
                ref = rho * w(v[nz[0]], u[nz[0]]) * w(v[nz[1]], u[nz[1]])
            assert np.isclose(f[i], ref, rtol=1e-12, atol=1e-16)


@pytest.mark.parametrize("M", [1.0, 13.894, 21.83])
def test_psi3_phi3_moments(M):
    """psi (reading R4 on D3Q19) has zero mass, unit momentum along its axis, zero
    energy and zero energy flux c_alpha c^2; phi has zero mass and momentum, unit energy
    and an isotropic second moment."""
    c = 1.0 / math.sqrt(M)
    cv = c * _vel().astype(float)
    c2 = (cv * cv).sum(1)
    ps = oracle.psi3(c)
    ph = oracle.phi3(c)
    for al, p in enumerate(ps):
        assert abs(p.sum()) < 1e-14
        for be in range(3):
            assert np.isclose((cv[:, be] * p).sum(), 1.0 if be == al else 0.0, atol=1e-14)
        assert abs((c2 * p).sum()) < 1e-13
        assert abs((cv[:, al] * c2 * p).sum()) < 1e-13
    assert abs(ph.sum()) < 1e-13
    assert np.abs(cv.T @ ph).max() < 1e-14
    assert np.isclose((c2 * ph).sum(), 1.0, rtol=1e-13)
    P = (cv[:, :, None] * cv[:, None, :] * ph[:, None, None]).sum(0)
    np.testing.assert_allclose(P, np.eye(3) / 3.0, atol=1e-13)


def _random_node3(ns, rng):
    M = np.array([W.MOLAR_MASS[s] for s in W.SPECIES_ORDER])[:ns]
    M = M / M.min()
    g = np.zeros((ns, 19))
    for j in range(ns):
        g[j] = oracle.equilibrium3(rng.uniform(0.1, 3.0), *rng.uniform(-0.04, 0.04, 3), M[j],
                                   rng.uniform(0.3, 0.36))
        g[j] *= 1.0 + 0.05 * rng.normal(size=19)
    return M, g


TAU1 = np.array([0.8, 0.7, 1.0, 0.6, 0.9])
TAU2 = np.array([0.7, 0.9, 0.65, 1.0, 0.75])


def test_collision3_conserves_species_mass_and_mixture_momentum():
    """Eq. final_kinetic_equation with U^c (reading R3) keeps every species mass and
    the mixture momentum exactly on D3Q19."""
    rng = np.random.default_rng(23)
    e = _vel().astype(float)
    for _ in range(20):
        M, g = _random_node3(5, rng)
        c = 1.0 / np.sqrt(M)
        go, mom = oracle.collide3(M, TAU1, TAU2, g, rng.normal(size=5) * 1e-3)
        np.testing.assert_allclose(go.sum(1), g.sum(1), rtol=1e-13)
        J0 = ((c[:, None, None] * e[None]) * g[:, :, None]).sum((0, 1))
        J1 = ((c[:, None, None] * e[None]) * go[:, :, None]).sum((0, 1))
        assert np.abs(J1 - J0).max() < 1e-13


def test_collision3_energy_equal_relaxation():
    """Equal relaxation times: the collision changes the energy sum c^2 g by exactly
    the Phi divergence sum_j divq_j (T(f) of Eq. moments_of_g with D = 3)."""
    rng = np.random.default_rng(24)
    tau = np.full(5, 0.8)
    e2 = (_vel() ** 2).sum(1)
    for _ in range(10):
        M, g = _random_node3(5, rng)
        c2 = (1.0 / M)[:, None] * e2[None]
        dq = rng.normal(size=5) * 1e-3
        go, _ = oracle.collide3(M, tau, tau, g, dq)
        assert np.isclose((c2 * go).sum() - (c2 * g).sum(), dq.sum(), rtol=1e-9, atol=1e-14)


def test_rest_state3_fixed_point_periodic():
    p = W.periodic_box3(8, 6, 5, reactions=[])
    o = oracle.Oracle3(p)
    g0 = o.populations()
    o.step(10)
    np.testing.assert_allclose(o.populations(), g0, rtol=1e-13, atol=1e-15)


def test_rest_state3_fixed_point_with_walls():
    """Gas at rest at the wall temperature above an FD-solid slab stays at rest: the
    diffusive wall re-emits the gas equilibrium, near-wall stencils reproduce uniform
    fields, the solid is at equilibrium."""
    p = W.periodic_box3(8, 6, 9, solid_layers=3, reactions=[])
    o = oracle.Oracle3(p)
    m0 = o.moments()
    o.step(15)
    np.testing.assert_allclose(o.moments(), m0, rtol=1e-12, atol=1e-14)


def test_uniform_flow3_inlet_outlet_fixed_point():
    nx, ny, nz = 16, 3, 3
    mask = np.zeros((nz, ny, nx), np.uint8)
    p = W._base(3, nx, ny, nz, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC],
                u_inlet=0.02, inlet_profile=W.PLUG, reactions=[])
    n = nx * ny * nz
    X = np.array([s["X_inlet"] for s in p["species"]])
    p["init"] = {"X": np.repeat(X[:, None], n, 1), "u": np.vstack([np.full(n, 0.02), np.zeros(n), np.zeros(n)]),
                 "T_K": np.full(n, p["T_inlet_K"]), "Ts_K": np.full(n, p["T_inlet_K"])}
    o = oracle.Oracle3(p)
    m0 = o.moments()
    o.step(15)
    np.testing.assert_allclose(o.moments(), m0, rtol=1e-12, atol=1e-14)


def test_periodic3_conservation():
    """Periodic 3D box from random smooth fields: species masses and the mixture
    momentum are conserved to rounding."""
    p = W.periodic_box3(10, 8, 6, reactions=[], Pr=0.7)
    p["init"] = W.random_fields(p, seed=31)
    o = oracle.Oracle3(p)
    b0 = o.balance()
    gas = o.classes() == 0

    def momentum():
        m = o.moments()
        rho = m[:5].sum(0)
        return np.array([(rho * m[10 + a])[gas].sum() for a in range(3)])

    P0 = momentum()
    o.step(20)
    b = o.balance()
    np.testing.assert_allclose(b["mass"], b0["mass"], rtol=1e-13)
    assert np.abs(momentum() - P0).max() < 1e-12 * b0["mass"].sum() * 0.01


def test_periodic3_energy_equal_relaxation():
    p = W.periodic_box3(10, 8, 6, reactions=[], Pr=0.7)
    for s in p["species"]:
        s["tau1"] = s["tau2"] = 0.8
    p["init"] = W.random_fields(p, seed=32)
    o = oracle.Oracle3(p)
    o.step(20)
    b = o.balance()
    assert abs(b["E_gas"] - b["E_gas0"]) < 1e-12 * b["E_gas0"]


def _unit_mass(p, tau=0.25):
    for s in p["species"]:
        s["M_gmol"] = 2.016
        s["tau1"] = s["tau2"] = tau
    return p


def test_reactive_closed_box3_exact_balance_unit_mass():
    """Equal species masses (every species on-lattice): the reactive diffusive wall on
    D3Q19 keeps exact mole bookkeeping and, with the conservative coupling, the gas
    energy gain plus the solid enthalpy gain equal the reaction heat to rounding."""
    p = _unit_mass(W.periodic_box3(10, 6, 8, solid_layers=3, reactions=[W.wgs_reaction(k0=2000.0)]))
    o = oracle.Oracle3(p)
    o.step(60)
    b = o.balance()
    dH = p["reactions"][0]["dH_Jmol"] / (3 * 8.314462618 * p["T0_K"])
    extent = b["Q_reaction"] / (-dH)
    assert extent > 1e-3
    nu = np.array(p["reactions"][0]["nu"], float)
    np.testing.assert_allclose(b["moles"] - b["moles0"], nu * extent, atol=1e-11 * b["moles0"].sum())
    assert abs(b["solid_residual"]) < 1e-12 * b["H_solid0"]
    assert abs(b["residual"]) < 1e-10 * b["Q_reaction"]


def test_fixed_t_solid_eigenmode3():
    """Eq. heat_equation_fd with the 7-point difference in a solid column between two
    fixed-T faces (z): the discrete eigenmode sin(pi (z + 1) / (N + 1)) decays by
    1 - 4 alpha sin^2(pi / (2 (N + 1))) per step."""
    nx, ny, nz = 2, 2, 13
    mask = np.full((nz, ny, nx), W.INERT, np.uint8)
    p = W._base(3, nx, ny, nz, mask, [W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.FIXED_T, W.FIXED_T],
                reactions=[])
    z = np.arange(nz)
    A = 6.0
    Ts = p["T_outer_K"] + A * np.sin(np.pi * (z + 1) / (nz + 1))
    p["init"] = {"Ts_K": np.repeat(Ts, nx * ny).astype(np.float64)}
    o = oracle.Oracle3(p)
    o.step(30)
    lam = 1.0 - 4.0 * p["alpha_s"] * math.sin(math.pi / (2 * (nz + 1))) ** 2
    got = o.moments()[-1].reshape(nz, ny, nx)[:, 0, 0] - p["T_outer_K"]
    np.testing.assert_allclose(got, A * lam ** 30 * np.sin(np.pi * (z + 1) / (nz + 1)), rtol=1e-11)


def test_fixed_t_solid_product_eigenmode3():
    """All three axes of the 7-point difference: in a solid block with fixed-T faces all
    round (three different side lengths) the product of the axis eigenmodes decays by
    1 - 4 alpha sum_a sin^2(pi / (2 (n_a + 1))) per step; a wrong weight or neighbour on
    any axis changes the rate."""
    nx, ny, nz = 9, 11, 13
    mask = np.full((nz, ny, nx), W.INERT, np.uint8)
    p = W._base(3, nx, ny, nz, mask, [W.FIXED_T] * 6, reactions=[])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.sin(np.pi * (x + 1) / (nx + 1)) * np.sin(np.pi * (y + 1) / (ny + 1))
            * np.sin(np.pi * (z + 1) / (nz + 1)))
    A = 6.0
    p["init"] = {"Ts_K": (p["T_outer_K"] + A * mode).ravel()}
    o = oracle.Oracle3(p)
    o.step(30)
    lam = 1.0 - 4.0 * p["alpha_s"] * sum(math.sin(math.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    got = o.moments()[-1].reshape(nz, ny, nx) - p["T_outer_K"]
    np.testing.assert_allclose(got, A * lam ** 30 * mode, rtol=1e-11, atol=1e-13)


# ---------------------------------------------------------------------------------------
# Transport against analytic decay rates
# ---------------------------------------------------------------------------------------

def _amp(f, nx):
    x = np.arange(nx)
    return 2.0 * (f * np.cos(2 * np.pi * x / nx)).mean()


def _trace_rate3(species, nx, t0, t1):
    p = W.periodic_box3(nx, 1, 1, reactions=[], energy_correction=0)
    j = W.SPECIES_ORDER.index(species)
    X0 = np.array([s["X_init"] for s in p["species"]])
    X0[j] = 1e-3
    x = np.arange(nx)
    X = np.repeat(X0[:, None], nx, 1)
    X[j] *= 1.0 + 0.01 * np.cos(2 * np.pi * x / nx)
    X[4] = 1.0 - X[:4].sum(0)
    p["init"] = {"X": X}
    o = oracle.Oracle3(p)
    o.step(t0)
    a0 = _amp(o.moments()[5 + j], nx)
    o.step(t1 - t0)
    a1 = _amp(o.moments()[5 + j], nx)
    k = 2 * np.pi / nx
    return -math.log(a1 / a0) / (k * k * (t1 - t0)), p, j


@pytest.mark.parametrize("species", ["CO2", "H2O"])
def test_trace_species_diffusion3(species):
    """Heavy trace species on D3Q19: D = tau2 T / M_j (extrapolated to k -> 0 from two
    wavelengths; 1% tolerance)."""
    D1, p, j = _trace_rate3(species, 48, 100, 900)
    D2, _, _ = _trace_rate3(species, 96, 400, 3600)
    D0 = (4.0 * D2 - D1) / 3.0
    M = np.array([s["M_gmol"] for s in p["species"]])
    M = M / M.min()
    D_th = p["species"][j]["tau2"] * (1.0 / 3.0) / M[j]
    assert abs(D0 / D_th - 1.0) < 0.01, (D1, D2, D0, D_th)


_PLANES = {"xy": (0, 1), "xz": (0, 2), "yz": (1, 2)}


def _diagonal_mode3(plane, sgn, n, steps, u0=0.0, species="CO2"):
    """A trace-species mode cos(2 pi (a + sgn b) / n) on an n x n periodic plane of the
    box (a, b the plane's two axes, the third axis one node deep), optionally carried by
    a uniform flow u0 (1, sgn) along its wave vector. Returns the projections of the
    species' mole-fraction deviation on cos and sin of the phase after each entry of
    `steps` (cumulative), the wave number |k| and the problem."""
    shape = [1, 1, 1]
    a, b = _PLANES[plane]
    shape[a] = shape[b] = n
    nx, ny, nz = shape
    p = W.periodic_box3(nx, ny, nz, reactions=[], energy_correction=0)
    j = W.SPECIES_ORDER.index(species)
    xyz = [g.ravel() for g in np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")[::-1]]
    ph = 2 * np.pi * (xyz[a] + sgn * xyz[b]) / n
    N = nx * ny * nz
    X0 = np.array([s["X_init"] for s in p["species"]])
    X0[j] = 1e-3
    X = np.repeat(X0[:, None], N, 1)
    X[j] *= 1.0 + 0.01 * np.cos(ph)
    X[4] = 1.0 - X[:4].sum(0)
    u = np.zeros((3, N))
    u[a], u[b] = u0, sgn * u0
    p["init"] = {"X": X, "u": u}
    o = oracle.Oracle3(p)
    out, done = [], 0
    for t in steps:
        o.step(t - done)
        done = t
        f = o.moments()[5 + j] - X0[j]
        out.append((2.0 * (f * np.cos(ph)).mean(), 2.0 * (f * np.sin(ph)).mean()))
    return out, 2 * np.pi * math.sqrt(2.0) / n, p


def _diagonal_D3(plane, sgn, n, t0, t1):
    (a0, _), (a1, _) = _diagonal_mode3(plane, sgn, n, (t0, t1))[0]
    k = 2 * np.pi * math.sqrt(2.0) / n
    return -math.log(a1 / a0) / (k * k * (t1 - t0))


def test_trace_species_diffusion3_along_face_diagonals():
    """The interpolated pulls of the 12 face-diagonal links: a heavy trace species' mode
    along a face diagonal diffuses with D = tau2 T / M_j like an axis mode (D3Q19 is
    isotropic to second order; k -> 0 from two wavelengths, 1%), and the modes along
    (1, 1) and (1, -1) of all three planes decay at the same rate (the lattice's
    reflection and axis-permutation symmetries; a (1, -1) mode is the one that sees a
    wrong pull position of the links perpendicular to a (1, 1) mode)."""
    D1 = _diagonal_D3("xy", 1, 24, 15, 130)
    D2 = _diagonal_D3("xy", 1, 48, 60, 520)
    D0 = (4.0 * D2 - D1) / 3.0
    p = W.periodic_box3(4, 4, 4, reactions=[])
    M = np.array([s["M_gmol"] for s in p["species"]])
    j = W.SPECIES_ORDER.index("CO2")
    D_th = p["species"][j]["tau2"] * (1.0 / 3.0) / (M[j] / M.min())
    assert abs(D0 / D_th - 1.0) < 0.01, (D1, D2, D0, D_th)
    for plane, sgn in (("xy", -1), ("xz", 1), ("xz", -1), ("yz", 1), ("yz", -1)):
        assert math.isclose(_diagonal_D3(plane, sgn, 24, 15, 130), D1, rel_tol=1e-9), (plane, sgn)


def test_trace_species_advection3_along_face_diagonals():
    """A heavy trace species' mode carried by a uniform flow along a face diagonal moves
    with the flow: its phase advances by |k| |u| per step (k -> 0 from two wavelengths,
    0.5%; the interpolation's dispersion is O(k^2)). The sign of every pull offset enters
    here, and again all six diagonal modes of the three planes agree."""
    u0 = 0.01
    ph = {}
    for n, t in ((24, 100), (48, 400)):
        ((A, B),), k, _ = _diagonal_mode3("xy", 1, n, (t,), u0=u0)
        ph[n] = math.atan2(B, A) / (k * math.sqrt(2.0) * u0 * t)
    r0 = (4.0 * ph[48] - ph[24]) / 3.0
    assert abs(r0 - 1.0) < 0.005, (ph, r0)
    for plane, sgn in (("xy", -1), ("xz", 1), ("xz", -1), ("yz", 1), ("yz", -1)):
        ((A, B),), k, _ = _diagonal_mode3(plane, sgn, 24, (100,), u0=u0)
        assert math.isclose(math.atan2(B, A) / (k * math.sqrt(2.0) * u0 * 100), ph[24], rel_tol=1e-9), (plane, sgn)


@pytest.mark.parametrize("axis", [0, 1, 2])
@pytest.mark.parametrize("ec,pr,pr_eff", [(1, 1.0, 1.0), (1, 0.7, 0.7), (0, 1.0, 2.5)])
def test_entropy_mode3_thermal_diffusivity(ec, pr, pr_eff, axis):
    """Isobaric temperature mode of an equal-mass gas on D3Q19 decays with
    alpha = tau1 T / Pr. Without the energy correction the folded product form carries
    (D - 1) / (D + 2) = 2/5 of the kinetic heat flux, i.e. Pr = 5/2 (the 3D counterpart
    of the paper's Pr = 4 for D2Q9). 2% tolerance. The mode runs along each axis in turn:
    the correction's divergence has a term per axis."""
    nx, tau = 48, 0.25
    shape = [1, 1, 1]
    shape[axis] = nx
    p = _unit_mass(W.periodic_box3(*shape, reactions=[], Pr=pr, energy_correction=ec), tau=tau)
    x = np.arange(nx)
    T = p["T_init_K"] * (1.0 + 0.002 * np.cos(2 * np.pi * x / nx))
    X0 = np.array([s["X_init"] for s in p["species"]])
    p["init"] = {"X": np.repeat(X0[:, None], nx, 1), "T_K": T, "C": p["T_init_K"] / T}
    o = oracle.Oracle3(p)
    k = 2 * np.pi / nx
    ts, amps = [], []
    dt = 10
    nsamp = int(1.2 / (tau / 3.0 / pr_eff * k * k) / dt)
    o.step(100)
    for i in range(nsamp):
        ts.append(100 + i * dt)
        amps.append(_amp(o.moments()[13] - p["T_init_K"], nx))
        o.step(dt)
    rate = -np.polyfit(np.array(ts, float), np.log(np.array(amps)), 1)[0]
    alpha = rate / (k * k)
    alpha_th = tau * (1.0 / 3.0) / pr_eff
    assert abs(alpha / alpha_th - 1.0) < 0.02, (alpha, alpha_th)


def _shear_rate3(nz, tsteps):
    p = W.periodic_box3(1, 1, nz, reactions=[], Pr=0.7)
    z = np.arange(nz)
    u = np.zeros((3, nz))
    u[0] = 0.002 * np.cos(2 * np.pi * z / nz)
    p["init"] = {"u": u}
    o = oracle.Oracle3(p)
    k = 2 * np.pi / nz
    ts, amps = [], []
    dt = 10
    o.step(20)
    for i in range(tsteps // dt):
        ts.append(20 + i * dt)
        amps.append(2.0 * (o.moments()[10] * np.cos(2 * np.pi * z / nz)).mean())
        o.step(dt)
    rate = -np.polyfit(np.array(ts, float), np.log(np.array(amps)), 1)[0]
    return rate / (k * k), p


def test_shear_wave3_mixture_viscosity():
    """A shear wave u_x(z) in the 5-species mixture on D3Q19 decays with nu = mu / rho,
    mu = sum_j tau1_j C_j T (Eq. multicomponent_mu); two wavelengths, 1% tolerance."""
    nu1, p = _shear_rate3(32, 400)
    nu2, _ = _shear_rate3(64, 1600)
    nu0 = (4.0 * nu2 - nu1) / 3.0
    M = np.array([s["M_gmol"] for s in p["species"]])
    M = M / M.min()
    X = np.array([s["X_init"] for s in p["species"]])
    t1 = np.array([s["tau1"] for s in p["species"]])
    mu = (t1 * X / 3.0).sum()
    rho = (X * M).sum()
    assert abs(nu0 / (mu / rho) - 1.0) < 0.01, (nu1, nu2, nu0, mu / rho)


# ---------------------------------------------------------------------------------------
# Exact accounts of the D3Q19 scheme
# ---------------------------------------------------------------------------------------

def test_accounts3_uniform_inlet_flux_closed_form():
    """Uniform inlet state, open channel periodic in y and z, one step: per inlet node the
    net mass the pulls take is sum e_x f = rho_j sqrt(M_j) u and the energy
    sum (1/2) c_j^2 |e|^2 e_x f = (1/2) rho_j u (1 + 2T) / sqrt(M_j): the folded D3Q19
    equilibrium keeps the first moments and the third moments c_a c_b^2 of the D3Q27
    product form (sum e_x e_y^2 f = rho sqrt(M) u T). The outlet carries the negatives;
    uniform data leave no interpolation or collision defect."""
    nx, ny, nz, u = 16, 6, 5, 0.02
    p = W._base(3, nx, ny, nz, np.zeros((nz, ny, nx), np.uint8),
                [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC, W.PERIODIC, W.PERIODIC],
                u_inlet=u, inlet_profile=W.PLUG, reactions=[])
    n = nx * ny * nz
    X = np.array([s["X_inlet"] for s in p["species"]])
    p["init"] = {"X": np.repeat(X[:, None], n, axis=1), "u": np.vstack([np.full(n, u), np.zeros(n), np.zeros(n)]),
                 "T_K": np.full(n, p["T_inlet_K"]), "Ts_K": np.full(n, p["T_inlet_K"])}
    o = oracle.Oracle3(p)
    o.step(1)
    a = o.accounts()
    M = np.array([s["M_gmol"] for s in p["species"]])
    M = M / M.min()
    rho = X * M
    T = p["T_inlet_K"] / (3.0 * p["T0_K"])
    m_in = ny * nz * rho * np.sqrt(M) * u
    q_in = ny * nz * np.sum(0.5 * rho * u * (1.0 + 2.0 * T) / np.sqrt(M))
    np.testing.assert_allclose(a["M_inlet"], m_in, rtol=1e-12)
    np.testing.assert_allclose(a["M_outlet"], -m_in, rtol=1e-12)
    assert abs(a["Q_inlet"] - q_in) <= 1e-12 * q_in
    assert abs(a["Q_outlet"] + q_in) <= 1e-12 * q_in
    scale = abs(a["E_pop"])
    assert abs(a["D_interp"]) <= 1e-14 * scale and abs(a["D_collision"]) <= 1e-14 * scale


@pytest.mark.parametrize("name", ["closed_reactive_box", "closed_box_paper_coupling", "sphere_crop"])
def test_accounts3_close_exactly(name):
    """The D3Q19 inventory of stored populations moves by the face fluxes, the
    interpolation and collision defects and the walls' emission minus arrival; with the
    solid's identity energy closes to rounding, and so does each species' mass with the
    walls' reaction production as its source."""
    if name == "sphere_crop":
        p, steps = W.crop3(W.config2(), 32, 16, 16), 60
    else:
        kw = {"coupling": W.PAPER} if name == "closed_box_paper_coupling" else {}
        p = W.periodic_box3(14, 10, 12, solid_layers=3, **kw)
        p["init"] = W.random_fields(p, seed=3)
        steps = 30
    o = oracle.Oracle3(p)
    o.step(steps)
    a, b = o.accounts(), o.balance()
    scale = abs(a["E_pop"]) + abs(b["H_solid"])
    assert abs(a["closure"]) <= 1e-12 * scale, a
    assert np.abs(a["mass_closure"]).max() <= 1e-12 * a["M_pop"].sum(), a["mass_closure"]
    if name == "closed_box_paper_coupling":
        assert abs(a["D_coupling"]) > 0.0
    else:
        assert abs(a["D_coupling"]) <= 1e-12 * scale
    if name == "sphere_crop":
        assert a["Q_inlet"] > 0.0 and a["Q_outlet"] < 0.0


def test_channel3_develops_poiseuille_profile():
    """D3Q19 laminar flow between two walls (periodic across the flow in z) from a plug
    inlet: downstream the profile is the plane Poiseuille parabola, symmetric about the
    mid-plane, uniform in z, vanishing at the diffusive walls up to a first-order slip."""
    nx, ng, wall, nz = 24, 10, 2, 2
    ny = ng + 2 * wall
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :wall, :] = W.INERT
    mask[:, wall + ng:, :] = W.INERT
    p = W._base(3, nx, ny, nz, mask, [W.INLET, W.OUTLET, W.FIXED_T, W.FIXED_T, W.PERIODIC, W.PERIODIC],
                u_inlet=0.02, inlet_profile=W.PLUG, reactions=[])
    o = oracle.Oracle3(p)
    o.step(900)
    ns = len(p["species"])
    ux = o.moments()[2 * ns].reshape(nz, ny, nx)
    col = ux[0, wall:wall + ng, 16]
    y = np.arange(ng, dtype=float)
    c = np.polyfit(y, col, 2)
    assert c[0] < 0.0
    assert np.abs(col - np.polyval(c, y)).max() <= 1e-3 * col.max()
    assert abs(-c[1] / (2.0 * c[0]) - (ng - 1) / 2.0) <= 1e-6
    assert abs(np.polyval(c, -1.0)) <= 0.06 * col.max()
    assert np.abs(ux[1, wall:wall + ng, 16] - col).max() <= 1e-12 * col.max()


@pytest.mark.parametrize("rate_form", [W.RATE_CONC_BILINEAR, W.RATE_XFRAC_REVERSIBLE])
def test_single_wall_node3_one_step_by_hand(rate_form):
    """Brute force of one reactive-wall application on the D3Q19 lattice (Sec. 4.3, count
    form of reading R11): one catalytic solid node in a periodic 8x8x8 gas box, equal
    species masses (every pull a pure shift). The emission shape at rest comes from the
    folded product form (reading R1b): rest 1 - 3T + 3T^2, axis T/2 - T^2, face diagonal
    T^2/4. From the populations at t = 0 the test forms the arrivals, the wall-density
    fixed point, the emitted populations and the reaction heat by hand."""
    n1 = 8
    c0 = 4
    mask = np.zeros((n1, n1, n1), np.uint8)
    mask[c0, c0, c0] = W.CATALYTIC
    rx = W.wgs_reaction(rate_form=rate_form)
    p = W._base(3, n1, n1, n1, mask, [W.PERIODIC] * 6, reactions=[rx], rho_w_tol=1e-15, rho_w_maxit=500)
    for s in p["species"]:
        s["M_gmol"] = 2.016
    p["init"] = W.random_fields(p, seed=7)
    o = oracle.Oracle3(p)
    g0 = o.populations()
    o.step(1)
    g1 = o.populations()
    b = o.balance()

    E = oracle.velocities3()  # direction order of the stored populations
    ns = len(p["species"])
    idx = lambda x, y, z: (x % n1) + n1 * ((y % n1) + n1 * (z % n1))
    k = idx(c0, c0, c0)
    T0 = p["T0_K"]
    Tw = p["init"]["Ts_K"][k] / (3.0 * T0)
    nnz = np.abs(E).sum(axis=1)
    wr = np.where(nnz == 0, 1 - 3 * Tw + 3 * Tw ** 2, np.where(nnz == 1, Tw / 2 - Tw ** 2, Tw ** 2 / 4))
    B = wr[1:].sum()
    arrived = np.array([[g0[j, i, idx(c0 - E[i, 0], c0 - E[i, 1], c0 - E[i, 2])] for i in range(1, 19)]
                        for j in range(ns)])
    A = arrived.sum(axis=1)
    nu = np.array(rx["nu"], dtype=float)
    R = 8.314462618
    kT = rx["k0"] * math.exp(-rx["Ea_Jmol"] / (R * 3.0 * T0 * Tw))

    def rate(rw):
        if rate_form == W.RATE_CONC_BILINEAR:
            return kT * np.prod([rw[j] ** (-nu[j]) for j in range(ns) if nu[j] < 0])
        x = rw / rw.sum()
        fwd = np.prod([x[j] ** (-nu[j]) for j in range(ns) if nu[j] < 0])
        bwd = np.prod([x[j] ** nu[j] for j in range(ns) if nu[j] > 0])
        return kT * (fwd - bwd / rx["Keq"])

    rw = A / B
    for _ in range(2000):
        new = (A + nu * rate(rw)) / B
        done = np.abs(new - rw).max() <= 1e-17
        rw = new
        if done:
            break
    r = rate(rw)
    emitted = wr[None, 1:] * ((A + nu * r) / B)[:, None]
    np.testing.assert_allclose(g1[:, 1:, k], emitted, rtol=1e-12)
    q = -(rx["dH_Jmol"] / (3.0 * R * T0)) * r
    assert r != 0.0 and abs(b["Q_reaction"] - q) <= 1e-12 * abs(q)
    dE = 0.5 * np.sum(nnz[None, 1:] * (emitted - arrived))
    assert abs(b["Q_wall"] - dE) <= 1e-12 * np.abs(0.5 * nnz[None, 1:] * emitted).sum()


def test_single_species_wall_density_closed_form():
    """Non-reacting single species (reading R7's special case): the converged wall
    density is the arrived mass over the emission normalisation, rho_w = A / B, and the
    wall re-emits exactly what arrived."""
    n1, c0 = 8, 4
    mask = np.zeros((n1, n1, n1), np.uint8)
    mask[c0, c0, c0] = W.INERT
    p = W._base(3, n1, n1, n1, mask, [W.PERIODIC] * 6, reactions=[])
    p["species"] = [dict(p["species"][3], X_init=1.0, X_inlet=1.0)]
    p["init"] = W.random_fields(p, seed=8)
    o = oracle.Oracle3(p)
    g0 = o.populations()
    o.step(1)
    g1 = o.populations()
    E = oracle.velocities3()
    idx = lambda x, y, z: (x % n1) + n1 * ((y % n1) + n1 * (z % n1))
    k = idx(c0, c0, c0)
    A = sum(g0[0, i, idx(c0 - E[i, 0], c0 - E[i, 1], c0 - E[i, 2])] for i in range(1, 19))
    assert abs(g1[0, 1:, k].sum() - A) <= 1e-14 * A


def test_reactive_wall3_delivers_c_squared_of_its_production():
    """The D3Q19 form of the closed-form delivery of a flat reactive wall: a uniform gas at
    rest and in equilibrium over a catalytic slab (periodic box, wall normal +z). The
    walls' step-1 reaction production goes out on the five links with e_z = +1; in step 2
    the first gas node along each such link takes it with the forward stencil's weight
    c (1 + c) / 2, the second with the central stencil's -(1 - c) c / 2, so the gas
    inventory of species j grows by exactly c_j^2 times the production. A wrong stencil
    choice near the wall, a wrong coefficient or a lost share of a diagonal emission link
    breaks the identity."""
    p = W.periodic_box3(8, 6, 12, solid_layers=4)
    o = oracle.Oracle3(p)
    gas = o.classes() == 0
    ns = len(p["species"])
    M = np.array([s["M_gmol"] for s in p["species"]])
    c2 = M.min() / M
    o.step(1)
    g1 = o.moments()[:ns][:, gas].sum(axis=1)
    r1 = o.accounts()["M_rxn"].copy()
    o.step(1)
    g2 = o.moments()[:ns][:, gas].sum(axis=1)
    assert np.all(np.abs(r1[:4]) > 0) and r1[4] == 0  # CO and H2O consumed, CO2 and H2 made, N2 inert
    # the difference of two inventories of ~10^3 carries their FP64 rounding, ~1e-12
    np.testing.assert_allclose(g2 - g1, c2 * r1, rtol=1e-9, atol=1e-14 * g1.max())
    assert abs((g2 - g1)[3] - r1[3]) <= 1e-9 * abs(r1[3])  # H2 (c = 1) in full


def test_outlet3_holds_inlet_pressure_with_upstream_state():
    """Reading R13 on D3Q19: every outlet node holds the equilibrium at the inlet
    pressure p = C_in T_in with the composition, velocity and temperature of its upstream
    gas node. Checked where the channel's hotter walls have warmed the gas (the outlet's
    upstream temperature differs from T_in, so holding C instead of p would fail)."""
    nx, ng, wall, nz = 24, 10, 2, 2
    ny = ng + 2 * wall
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :wall, :] = W.INERT
    mask[:, wall + ng:, :] = W.INERT
    p = W._base(3, nx, ny, nz, mask, [W.INLET, W.OUTLET, W.FIXED_T, W.FIXED_T, W.PERIODIC, W.PERIODIC],
                u_inlet=0.02, inlet_profile=W.PLUG, reactions=[], T_solid_init_K=540.0, T_outer_K=540.0)
    o = oracle.Oracle3(p)
    o.step(200)
    r = outlet_condition_errors(p, o, _vel())
    assert len(r) == ny * nz - 2 * wall * nz and r[:, 3].min() > p["T_inlet_K"] + 2.0
    assert r[:, 0].max() < 1e-12 and r[:, 1].max() < 1e-13 and r[:, 2].max() < 1e-14


def test_paper_coupling3_one_step_by_hand():
    """Eq. wall_temperature on D3Q19: a one-layer FD slab in a periodic box (gas above and
    below every slab node, no gradient along the slab); from a uniform gas at T_g and
    solid at T_s0 the first step moves the solid by exactly
    2 kappa_f (T_g - T_s0) / (rho c_p)_s."""
    p = W.periodic_box3(6, 6, 6, solid_layers=1, reactions=[], coupling=1)
    n = p["nx"] * p["ny"] * p["nz"]
    p["init"] = {"T_K": np.full(n, 520.0), "Ts_K": np.full(n, 500.0)}
    o = oracle.Oracle3(p)
    wall = o.classes() == 3
    assert wall.sum() == p["nx"] * p["ny"]
    o.step(1)
    dT = o.moments()[-1][wall] - 500.0
    np.testing.assert_allclose(dT, 2.0 * p["kappa_f"] * (520.0 - 500.0) / p["rhocp_s"], rtol=1e-9)


def test_residual3_closed_form_on_a_decaying_eigenmode():
    """Reading R16's residual on D3Q19: a solid block with fixed-T faces at T_inlet
    carrying the product eigenmode of the 7-point FD step decays as lam^t, so the
    residual over K steps is (lam^-K - 1) / K; +inf on the first call."""
    nx, ny, nz = 9, 11, 13
    mask = np.full((nz, ny, nx), W.INERT, np.uint8)
    p = W._base(3, nx, ny, nz, mask, [W.FIXED_T] * 6, reactions=[])
    assert p["T_outer_K"] == p["T_inlet_K"]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    mode = (np.sin(np.pi * (x + 1) / (nx + 1)) * np.sin(np.pi * (y + 1) / (ny + 1))
            * np.sin(np.pi * (z + 1) / (nz + 1)))
    p["init"] = {"Ts_K": (p["T_outer_K"] + 6.0 * mode).ravel()}
    o = oracle.Oracle3(p)
    lam = 1.0 - 4.0 * p["alpha_s"] * sum(math.sin(math.pi / (2 * (m + 1))) ** 2 for m in (nx, ny, nz))
    assert o.residual(0) == float("inf")
    for K in (10, 25):
        o.step(K)
        assert math.isclose(o.residual(K), (lam ** -K - 1.0) / K, rel_tol=1e-11)


def test_inlet3_holds_the_inlet_equilibrium():
    """Sec. 6's inlet on D3Q19 (plug profile): every inlet node holds, from its stored
    populations, u = (u_inlet, 0, 0), the inlet composition, C = 1 and T_inlet, here in
    a channel whose gas starts 10 K below the inlet temperature; T from the moments,
    T = (E - |J|^2 / rho) / (D C), D = 3."""
    nx, ng, wall, nz = 12, 6, 2, 4
    ny = ng + 2 * wall
    mask = np.zeros((nz, ny, nx), np.uint8)
    mask[:, :wall, :] = W.INERT
    mask[:, wall + ng:, :] = W.INERT
    p = W._base(3, nx, ny, nz, mask, [W.INLET, W.OUTLET, W.FIXED_T, W.FIXED_T, W.PERIODIC, W.PERIODIC],
                u_inlet=0.02, inlet_profile=W.PLUG, reactions=[], T_init_K=490.0)
    assert p["T_inlet_K"] == 500.0
    o = oracle.Oracle3(p)
    o.step(3)
    ns = len(p["species"])
    M = np.array([s["M_gmol"] for s in p["species"]])
    M = M / M.min()
    c = np.sqrt(1.0 / M)
    e = _vel().astype(float)
    e2 = (e * e).sum(1)
    g = o.populations()
    inlet = np.where(o.classes() == 1)[0]
    assert len(inlet) == ng * nz
    rho = np.array([g[:, :, k].sum(1) for k in inlet])
    J = np.array([sum(c[j] * (e.T @ g[j, :, k]) for j in range(ns)) for k in inlet])
    E = np.array([sum(c[j] ** 2 * (e2 * g[j, :, k]).sum() for j in range(ns)) for k in inlet])
    C = (rho / M).sum(1)
    u = J / rho.sum(1)[:, None]
    T_K = (E - (J ** 2).sum(1) / rho.sum(1)) / (3.0 * C) * 3.0 * p["T0_K"]
    X_in = np.array([s["X_inlet"] for s in p["species"]])
    np.testing.assert_allclose(u, np.repeat([[p["u_inlet"], 0.0, 0.0]], len(inlet), 0), rtol=1e-13, atol=1e-16)
    np.testing.assert_allclose(rho / M / C[:, None], np.repeat(X_in[None], len(inlet), 0), rtol=1e-13, atol=1e-18)
    np.testing.assert_allclose(C, 1.0, rtol=1e-13)
    np.testing.assert_allclose(T_K, p["T_inlet_K"], rtol=1e-12)
