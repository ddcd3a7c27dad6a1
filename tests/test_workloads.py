"""The seeded synthetic inputs have the sizes, value distributions and structure of the
benchmark configurations (the recipe the design notes state): porosity, radius ranges,
non-overlap and clearances, free inlet/outlet columns, percolation, determinism, and the
ranges of the batched instances. Host logic only."""
import math

import numpy as np
import pytest

from paper_1804_07588_gb300 import workloads as W


def test_channel_geometry():
    p = W.config0()
    mask = p["mask"].reshape(p["ny"], p["nx"])
    assert (p["nx"], p["ny"]) == (128, 48)
    assert np.all(mask[:8] == W.CATALYTIC) and np.all(mask[40:] == W.CATALYTIC)
    assert np.all(mask[8:40] == W.GAS)
    assert p["face_bc"][:4] == [W.INLET, W.OUTLET, W.FIXED_T, W.FIXED_T]
    assert p["inlet_profile"] == W.PARABOLIC and p["u_inlet"] == 0.02


def test_disk_bed_recipe():
    """1024x512, disks r ~ U[6, 12] by random sequential addition with a 2-node surface
    gap (periodic in y), porosity 0.6, 17 free columns at each end; seeded."""
    mask, disks = W.disk_mask(1024, 512, 0.6, 6.0, 12.0, 1000)
    solid = mask > 0
    assert abs(1.0 - solid.mean() - 0.6) <= 2e-3
    r = np.array([d[2] for d in disks])
    # radii are drawn uniform in [6, 12]; the accepted ones skew small (8.2 on average)
    # because late in the addition large disks no longer fit
    assert r.min() >= 6.0 and r.max() <= 12.0
    assert not solid[:, :17].any() and not solid[:, -17:].any()
    # no two disks closer than the gap (periodic in y): brute force on all pairs
    c = np.array([(d[0], d[1]) for d in disks])
    dx = c[:, None, 0] - c[None, :, 0]
    dy = np.abs(c[:, None, 1] - c[None, :, 1])
    dy = np.minimum(dy, 512 - dy)
    dist = np.hypot(dx, dy) - (r[:, None] + r[None, :])
    np.fill_diagonal(dist, np.inf)
    assert dist.min() >= 2.0 - 1e-9
    mask2, _ = W.disk_mask(1024, 512, 0.6, 6.0, 12.0, 1000)
    assert np.array_equal(mask, mask2)


def test_sphere_bed_recipe():
    """256x128x128, overlapping spheres r ~ U[5, 10] added to porosity 0.5, 12 free
    columns at each end, the gas connected from inlet to outlet (6-connected, periodic in
    y and z); seeded."""
    mask, spheres = W.sphere_mask(256, 128, 128, 0.5, 5.0, 10.0, 2000)
    solid = mask > 0
    assert abs(1.0 - solid.mean() - 0.5) <= 2e-3
    r = np.array([s[3] for s in spheres])
    assert r.min() >= 5.0 and r.max() <= 10.0
    assert not solid[:, :, :12].any() and not solid[:, :, -12:].any()
    assert W._percolates(~solid)
    p = W.config2()
    assert (p["nx"], p["ny"], p["nz"]) == (256, 128, 128)
    assert np.array_equal(p["mask"].reshape(128, 128, 256), mask)
    assert p["face_bc"] == [W.INLET, W.OUTLET] + [W.PERIODIC] * 4


def test_percolation_check_detects_a_blocked_bed():
    gas = np.ones((6, 6, 20), bool)
    assert W._percolates(gas)
    gas[:, :, 10] = False  # a solid wall across the flow
    assert not W._percolates(gas)


def test_batch_instance_ranges():
    """Instances: nx, ny multiples of 8 in [256, 1024] x [128, 256], porosity in [0.4,
    0.7], inlet 0.005-0.03, inlet temperature 450-600 K (also T0 and the initial
    temperatures); every instance its own seed, its gas connecting inlet and outlet."""
    inst = W.batch_instances(n=8)
    assert len(inst) == 8
    pors = []
    for p in inst:
        assert p["nx"] % 8 == 0 and 256 <= p["nx"] <= 1024
        assert p["ny"] % 8 == 0 and 128 <= p["ny"] <= 256
        por = 1.0 - (p["mask"] > 0).mean()
        pors.append(por)
        assert 0.4 - 2e-3 <= por <= 0.7 + 2e-3
        assert W._percolates((np.asarray(p["mask"]).reshape(1, p["ny"], p["nx"]) == 0))
        assert 0.005 <= p["u_inlet"] <= 0.03
        assert 450.0 <= p["T_inlet_K"] <= 600.0
        assert p["T0_K"] == p["T_inlet_K"] == p["T_init_K"] == p["T_solid_init_K"]
    assert len({p["mask"].tobytes() for p in inst}) == len(inst)
    assert min(pors) < 0.55  # below what separated disks reach


def test_boolean_disks_reach_low_porosity():
    """Overlapping disks reach porosity 0.4 (digitised, within one disk's area), keep the
    inlet and outlet columns free, and a packing whose gas is cut is rejected."""
    mask, disks = W.disk_mask_boolean(256, 128, 0.4, 6.0, 12.0, 27)
    por = (mask == W.GAS).mean()
    assert 0.4 - math.pi * 144 / (256 * 128) <= por <= 0.4 + 1e-12
    assert (mask[:, :17] == W.GAS).all() and (mask[:, -17:] == W.GAS).all()
    with pytest.raises((ValueError, RuntimeError)):
        W.disk_mask_boolean(128, 64, 0.05, 6.0, 12.0, 3)


def test_species_and_kinetics_tables():
    """CO/H2O/CO2/H2/N2 with inlet 0.1/0.1/1e-6/1e-6/balance, relaxation times in
    0.6-1.0, and a water-gas shift that conserves mass (sum nu_j M_j = 0)."""
    sp = W.species_table()
    assert [s["name"] for s in sp] == ["CO", "H2O", "CO2", "H2", "N2"]
    assert math.isclose(sum(s["X_inlet"] for s in sp), 1.0, rel_tol=0, abs_tol=1e-15)
    assert all(0.6 <= s["tau1"] <= 1.0 and 0.6 <= s["tau2"] <= 1.0 for s in sp)
    rx = W.wgs_reaction()
    assert abs(sum(n * s["M_gmol"] for n, s in zip(rx["nu"], sp))) <= 1e-9
    assert rx["Ea_Jmol"] == 50e3 and rx["Keq"] == 10.0 and rx["dH_Jmol"] == -41e3


def test_learning_instance_ranges():
    """The warm start's geometries: 128x64x64 sphere packings, porosity in [0.4, 0.6]
    (each percolating from inlet to outlet), inlet 0.005-0.03, 450-600 K; per-instance
    seeds."""
    inst = W.learning_instances(n=3)
    assert len(inst) == 3
    for p in inst:
        assert (p["nx"], p["ny"], p["nz"], p["lattice"]) == (128, 64, 64, 19)
        solid = p["mask"].reshape(64, 64, 128) > 0
        assert 0.4 - 3e-3 <= 1.0 - solid.mean() <= 0.6 + 3e-3
        assert W._percolates(~solid)
        assert 0.005 <= p["u_inlet"] <= 0.03 and 450.0 <= p["T_inlet_K"] <= 600.0
    assert len({p["mask"].tobytes() for p in inst}) == 3
