"""GPU parity: the CUDA solver (through the C ABI) against the FP64 oracle on the same
seeded inputs, field by field, at sizes that span several 32x8 tiles with ragged tails,
plus the full-size porous bed of the benchmark for a few steps.

Tolerance: 1e-5 of max |field| on every moment field (field-normalised relative error),
the bar the FP32 path is held to after 1000 steps."""
import numpy as np
import pytest

import oracle
from paper_1804_07588_gb300 import workloads as W
from parity import assert_parity, run_both

pytestmark = pytest.mark.gpu


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


def test_initial_moments_match():
    p = W.periodic_box(40, 28, solid_rows=5)
    p["init"] = W.random_fields(p, seed=21)
    s, o = run_both(p, 0)
    assert_parity(s, o, tol=1e-6, what="t=0")


def test_populations_one_step_periodic_ragged():
    """One step on a 40x28 periodic box (one full and one ragged tile in x, a ragged tile
    in y): every stored population matches."""
    p = W.periodic_box(40, 28, reactions=[])
    p["init"] = W.random_fields(p, seed=22)
    s, o = run_both(p, 1)
    g_gpu = s.populations().astype(np.float64)
    g_ora = o.populations()
    gas = o.classes() == 0
    err = np.abs(g_gpu[:, :, gas] - g_ora[:, :, gas]).max() / np.abs(g_ora[:, :, gas]).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("pr,ec", [(0.7, 1), (1.0, 0)])
def test_parity_periodic_random(pr, ec):
    p = W.periodic_box(40, 28, reactions=[], Pr=pr, energy_correction=ec)
    p["init"] = W.random_fields(p, seed=23)
    s, o = run_both(p, 100)
    assert_parity(s, o, what="periodic")


def test_parity_closed_box_reactive():
    p = W.periodic_box(70, 20, solid_rows=5)
    p["init"] = W.random_fields(p, seed=24)
    s, o = run_both(p, 200)
    assert_parity(s, o, what="reactive box")


@pytest.mark.parametrize("coupling", [W.CONSERVATIVE, W.PAPER])
def test_parity_channel_short(coupling):
    p = W.channel(nx=72, n_gas=20, wall=4, coupling=coupling)
    s, o = run_both(p, 150)
    assert_parity(s, o, what=f"channel coupling={coupling}")


def test_parity_channel_conc_bilinear():
    p = W.channel(nx=48, n_gas=12, wall=3, reactions=[W.wgs_reaction(k0=50.0, rate_form=W.RATE_CONC_BILINEAR)])
    s, o = run_both(p, 120)
    assert_parity(s, o, what="bilinear")


def test_parity_porous_small():
    """Digitised disks (concave staircase corners, one-node fallbacks), periodic in y,
    inlet and outlet, from random fields."""
    p = W.porous_disks(nx=100, ny=60, porosity=0.75, rmin=3.0, rmax=7.0, seed=7, u_inlet=0.01)
    p["init"] = W.random_fields(p, seed=25, du=0.005)
    s, o = run_both(p, 200)
    info = s.info()
    assert info["stencil_counts"][4] + info["stencil_counts"][5] + info["stencil_counts"][0] > 0
    assert_parity(s, o, what="porous")


def test_parity_config0_1000_steps():
    """The catalytic channel (128x32 gas between 8-node FD walls) after 1000 steps:
    every moment field within 1e-5 of the FP64 oracle."""
    p = W.config0()
    s, o = run_both(p, 1000, chunks=4)
    errs = assert_parity(s, o, what="config0 1000 steps")
    print("config0 errors", errs)


def _bed_crop(w, h):
    """The top-left w x h crop of the 1024x512 bed (same disk packing), outlet columns
    opened, periodic in y."""
    full = W.config1()
    mask = full["mask"].reshape(512, 1024)[:h, :w].copy()
    mask[:, w - 2:] = W.GAS
    return W._base(2, w, h, 1, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC], u_inlet=full["u_inlet"],
                   inlet_profile=W.PLUG)


def test_parity_bed_crop_1000_steps():
    """The 128x128 crop of the disk bed (catalytic disks of radius 6-12, digitised
    corners, inlet, outlet) from random fields, 1000 steps: every field within 1e-5."""
    p = _bed_crop(128, 128)
    p["init"] = W.random_fields(p, seed=29, du=0.005)
    s, o = run_both(p, 1000, chunks=4)
    errs = assert_parity(s, o, what="bed crop 1000 steps")
    print("bed crop errors", errs)
    s.close()


def test_parity_config1_full_size_few_steps():
    """The full 1024x512 porous bed, in the launch configuration the benchmark times,
    from random fields: 4 steps, every node of every field."""
    p = W.config1()
    p["init"] = W.random_fields(p, seed=26, du=0.005)
    s, o = run_both(p, 4)
    assert_parity(s, o, what="config1 full size")


def test_ledger_matches_oracle():
    p = W.periodic_box(60, 20, solid_rows=6)
    p["init"] = W.random_fields(p, seed=27)
    s, o = run_both(p, 300)
    bg, bo = s.balance(), o.balance()
    for k in ("E_gas", "H_solid", "E_gas0", "H_solid0"):
        assert abs(bg[k] - bo[k]) <= 1e-6 * abs(bo[k]), (k, bg[k], bo[k])
    for k in ("Q_reaction", "Q_wall", "Q_couple"):
        assert abs(bg[k] - bo[k]) <= 1e-4 * max(abs(bo[k]), 1e-12), (k, bg[k], bo[k])
    # species inventories, normalised by the total (trace products are tiny)
    np.testing.assert_allclose(bg["mass"], bo["mass"], rtol=0, atol=1e-6 * bo["mass"].sum())
    np.testing.assert_allclose(bg["moles"], bo["moles"], rtol=0, atol=1e-6 * bo["moles"].sum())
    assert abs(bg["solid_residual"]) < 1e-6 * bo["H_solid0"]


def test_residual_matches_oracle():
    p = W.channel(nx=64, n_gas=16, wall=4)
    from paper_1804_07588_gb300 import fdlbm
    s = fdlbm.Solver(p)
    o = oracle.Oracle(p)
    assert s.residual() == float("inf") and o.residual(0) == float("inf")
    s.step(50)
    o.step(50)
    rg, ro = s.residual(), o.residual(50)
    assert abs(rg - ro) <= 1e-3 * ro, (rg, ro)


def test_set_fields_restarts():
    p = W.periodic_box(36, 20, solid_rows=4)
    init = W.random_fields(p, seed=28)
    from paper_1804_07588_gb300 import fdlbm
    s = fdlbm.Solver(p)
    s.step(10)
    s.set_fields(init)
    p2 = dict(p)
    p2["init"] = init
    o = oracle.Oracle(p2)
    s.step(30)
    o.step(30)
    assert_parity(s, o, what="after set_fields")


def test_single_species_and_no_solid():
    p = W.periodic_box(33, 17, reactions=[], energy_correction=0)
    p["species"] = p["species"][:1]
    p["species"][0]["X_init"] = p["species"][0]["X_inlet"] = 1.0
    n = 33 * 17
    p["init"] = {"u": np.vstack([0.01 * np.sin(np.arange(n) / 7.0), np.zeros(n)]),
                 "T_K": 500 + 3 * np.cos(np.arange(n) / 5.0)}
    s, o = run_both(p, 60)
    assert_parity(s, o, what="1 species")


def test_unstable_state_is_reported_not_faulted():
    """An explicit energy correction past its stability limit (pure H2 at Pr 0.7: K/C =
    ((D + 2)/Pr - (D - 1)) tau1 T is about 0.94, above 1/2) blows up to NaN; the kernel's
    sticky flag turns that into FDLBM_EUNSTABLE on the host (no device trap)."""
    fdlbm = _fdlbm()
    p = _species_subset(W.periodic_box(32, 16, reactions=[], Pr=0.7), 1)
    p["init"] = W.random_fields(p, seed=81)
    s = fdlbm.Solver(p)
    s.step(400)
    with pytest.raises(fdlbm.FdlbmError) as ei:
        s.sync()
    assert ei.value.status == -4


# ---------------------------------------------------------------------------------------
# Locally updated relaxation times (Sec. 3)
# ---------------------------------------------------------------------------------------

def test_parity_local_tau_periodic():
    """Relaxation times updated at every node and step from the local composition and
    temperature (Wilke viscosity, mixture-averaged diffusion): GPU against the oracle on a
    periodic box from random fields."""
    p = W.local_transport(W.periodic_box(40, 28, reactions=[], Pr=0.7))
    p["init"] = W.random_fields(p, seed=71)
    s, o = run_both(p, 150)
    assert_parity(s, o, what="local tau periodic")
    s.close()


def test_parity_local_tau_channel():
    """Catalytic channel with inlet, outlet, reactive walls and FD solid, local relaxation
    times."""
    p = W.local_transport(W.channel(nx=72, n_gas=20, wall=4))
    s, o = run_both(p, 200)
    assert_parity(s, o, what="local tau channel")
    s.close()


def test_local_tau_rejected_where_not_built():
    fdlbm = _fdlbm()
    p = W.local_transport(W.periodic_box(16, 12, reactions=[]))
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Solver(p, storage="bf16")
    a = fdlbm.Solver(p)
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Batch([a])
    a.close()


# ---------------------------------------------------------------------------------------
# Moving diffusive walls (thermal Couette flow)
# ---------------------------------------------------------------------------------------

@pytest.mark.parametrize("unit_mass", [True, False])
def test_parity_couette_moving_wall(unit_mass):
    """Thermal Couette flow between a plate at rest and a moving, hotter plate: GPU against
    the oracle (equal-mass species, and the 5-species mixture with off-lattice streaming
    next to the moving wall), 3000 steps from the linear profiles, width 8 (several
    wall nodes per plate)."""
    p = W.couette(32, U_w=0.03, dT_K=2.0, nx=8, Pr=0.7)
    for s in p["species"]:
        s["tau1"] = s["tau2"] = 0.25 if unit_mass else s["tau1"]
        if unit_mass:
            s["M_gmol"] = 2.016
    if not unit_mass:
        p["energy_correction"] = 0
    s_, o = run_both(p, 3000)
    assert_parity(s_, o, what="couette", vector_u=True)  # uy is zero up to rounding
    s_.close()


def test_enthalpy_coupling_error_paper_box_gpu():
    """The paper's enthalpy-coupling box on the GPU (FP32 state, FP64 ledger): eps of Eq.
    error_coupling below the paper's order 1e-5. 200 x 8 instead of the paper's 200 x 3:
    the library needs at least 8 nodes across a periodic direction (twice its ghost
    depth), and the paper finds the error independent of the system size."""
    p = W.periodic_box(200, 8, solid_cols=100, energy_correction=0, reactions=[W.wgs_reaction(k0=2000.0)])
    for s in p["species"]:
        s["M_gmol"] = 2.016
        s["tau1"] = s["tau2"] = 0.8
    sv = _fdlbm().Solver(p)
    sv.step(3000)
    b = sv.balance()
    assert b["Q_reaction"] > 0
    assert abs(b["eps_paper"]) < 1e-5, b["eps_paper"]
    sv.close()


def test_short_periodic_axis_rejected():
    """A periodic axis shorter than twice the ghost depth is rejected (a node would have to
    write the periodic copies of both faces)."""
    fdlbm = _fdlbm()
    with pytest.raises(fdlbm.FdlbmError) as ei:
        fdlbm.Solver(W.periodic_box(20, 6, reactions=[]))
    assert ei.value.status == -1
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Solver(W.periodic_box3(12, 12, 5, reactions=[]))


# ---------------------------------------------------------------------------------------
# Species counts other than 5 (each is its own kernel instantiation) and degenerate
# lattices
# ---------------------------------------------------------------------------------------

def _species_subset(p, ns):
    """A subset of the five-species table that keeps H2 (the lightest species, whose
    relaxation time sets the stable range of the energy-correction flux once its molar
    mass is the unit), or the five plus argon for ns = 6, with the mole fractions
    renormalised; reactions only for the full table (their stoichiometry spans all of
    CO, H2O, CO2 and H2)."""
    pick = {1: [3], 2: [0, 3], 3: [0, 1, 3], 5: [0, 1, 2, 3, 4], 6: [0, 1, 2, 3, 4]}[ns]
    sp = [dict(p["species"][k]) for k in pick]
    if ns == 6:
        sp.append({"name": "Ar", "M_gmol": 39.948, "tau1": 0.85, "tau2": 0.8, "X_init": 0.05, "X_inlet": 0.05})
    for key in ("X_init", "X_inlet"):
        tot = sum(s[key] for s in sp)
        for s in sp:
            s[key] = s[key] / tot
    p["species"] = sp
    if ns < 5:
        p["reactions"] = []
    else:
        for r in p["reactions"]:
            r["nu"] = (list(r["nu"]) + [0] * 6)[:ns]
    return p


@pytest.mark.parametrize("ns", [1, 2, 3, 6])
def test_parity_species_counts(ns):
    """2, 3 and 6 species: periodic box over a catalytic FD-solid slab. 1 species (pure
    H2): a channel between FD-solid walls, driven by its inlet (in a closed periodic box
    the single gas's random velocity decays 30-fold in 120 steps, to where the
    field-normalised error measures FP32 rounding of a vanishing field). It takes
    Pr = 2.5: the energy-correction coefficient K/C = ((D + 2)/Pr - (D - 1)) tau1 T of
    unit-mass H2 is about 0.94 at Pr = 0.7 and T = 1/3, past the explicit limit of the
    lagged flux; in the mixtures H2 is a small part of the heat capacity."""
    if ns == 1:
        p = _species_subset(W.channel(96, n_gas=20, wall=6, Pr=2.5), ns)
    else:
        p = _species_subset(W.periodic_box(36, 20, solid_rows=5), ns)
    p["init"] = W.random_fields(p, seed=80 + ns)
    s, o = run_both(p, 120)
    assert_parity(s, o, what=f"{ns} species", vector_u=True)
    s.close()


def test_all_solid_lattice():
    """A lattice without gas nodes: the FD heat step alone (fixed-T faces), against the
    oracle's solid temperature."""
    p = W._base(2, 24, 16, 1, np.full((16, 24), W.INERT, np.uint8),
                [W.PERIODIC, W.PERIODIC, W.FIXED_T, W.FIXED_T], reactions=[], T_outer_K=480.0)
    p["init"] = {"Ts_K": 500.0 + 5.0 * W.smooth_noise((16, 24), np.random.default_rng(9)).reshape(-1)}
    s, o = run_both(p, 200)
    ts_g = s.moments_host()[-1].astype(np.float64)
    ts_o = o.moments()[-1]
    assert np.abs(ts_g - ts_o).max() <= 1e-5 * np.abs(ts_o - 480.0).max()
    s.close()
