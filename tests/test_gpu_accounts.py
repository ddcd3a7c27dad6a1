"""Exact energy accounts of the D2Q9 and D3Q19 steps (handles created with ledger_detail): the FP64
ledger terms measured from the FP32 values the kernel stores and pulls close the energy
balance to FP64 rounding, in closed and open systems and both coupling modes; the terms
match the FP64 oracle's accounts; and keeping the accounts changes none of the step's
results."""
import math

import numpy as np
import pytest

import oracle
from paper_1804_07588_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


def _case(name):
    if name == "closed_reactive_box":
        p = W.periodic_box(36, 20, solid_rows=5)
        p["init"] = W.random_fields(p, seed=3)
        return p, 60
    if name == "open_channel":
        return W.channel(nx=64, n_gas=16, wall=4), 200
    if name == "open_channel_paper_coupling":
        return W.channel(nx=64, n_gas=16, wall=4, coupling=W.PAPER), 200
    if name == "couette_moving_wall":
        return W.couette(n_gas=16, U_w=0.03, dT_K=2.0, nx=8), 150
    raise KeyError(name)


CASES = ["closed_reactive_box", "open_channel", "open_channel_paper_coupling", "couette_moving_wall"]


@pytest.mark.parametrize("name", CASES)
def test_exact_accounts_close(name):
    """dE_pop + dH_solid - Q_rxn - Q_fixedT - Q_inlet - Q_outlet - D_interp - D_collision -
    D_coupling - D_solid vanishes to FP64 rounding: every term is a sum of exact
    differences of stored FP32 values."""
    p, steps = _case(name)
    s = _fdlbm().Solver(p, ledger_detail=True)
    s.step(steps)
    b = s.balance()
    s.close()
    assert b["ledger_detail"] == 1
    scale = abs(b["E_pop"]) + abs(b["H_solid"])
    assert abs(b["closure"]) <= 1e-12 * scale, b
    # the FP32 rounding of the FD step and of the wall exchange the solid receives (it
    # accrues on the gross flows through the walls, not on the net exchange Q_wall)
    assert abs(b["D_solid"]) <= 1e-8 * scale
    if name != "open_channel_paper_coupling":
        assert abs(b["D_coupling"]) <= 1e-8 * scale


@pytest.mark.parametrize("name", CASES)
def test_exact_accounts_match_oracle(name):
    """Inventory, face fluxes and defects of the GPU step against the oracle's FP64
    accounts of the same steps (the oracle has no FP32 rounding, so its D_solid is zero
    and its D_coupling is the paper law's imbalance alone)."""
    p, steps = _case(name)
    s = _fdlbm().Solver(p, ledger_detail=True)
    o = oracle.Oracle(p)
    s.step(steps)
    o.step(steps)
    b, a = s.balance(), o.accounts()
    s.close()
    scale = abs(a["E_pop"])
    for k in ("E_pop", "E_pop0"):
        assert abs(b[k] - a[k]) <= 1e-6 * scale, (k, b[k], a[k])
    flux = max(abs(a["Q_inlet"]), abs(a["Q_outlet"]), abs(a["D_interp"]), abs(a["D_collision"]), 1e-30)
    for k in ("Q_inlet", "Q_outlet", "D_interp", "D_collision"):
        assert abs(b[k] - a[k]) <= 1e-4 * flux + 1e-9 * scale, (k, b[k], a[k])
    # the GPU's D_coupling also carries the FP32 rounding of the exchange the solid
    # receives (zero in the FP64 oracle)
    assert abs(b["D_coupling"] - a["D_coupling"]) <= 1e-4 * abs(a["D_coupling"]) + 1e-6 * scale


def test_accounts_change_no_result():
    """The exact-accounts step stores the same populations and moments and keeps the
    same basic ledger, bit for bit."""
    fdlbm = _fdlbm()
    p = W.channel(nx=64, n_gas=16, wall=4)
    s0, s1 = fdlbm.Solver(p), fdlbm.Solver(p, ledger_detail=True)
    s0.step(150)
    s1.step(150)
    assert np.array_equal(s0.moments_host(), s1.moments_host())
    assert np.array_equal(s0.populations(), s1.populations())
    b0, b1 = s0.balance(), s1.balance()
    for k in ("Q_reaction", "Q_wall", "Q_couple", "Q_fixedT"):  # per-block slots, summed in order
        assert b0[k] == b1[k], k
    for k in ("E_gas", "H_solid"):  # block sums added atomically: order-dependent last bits
        assert abs(b0[k] - b1[k]) <= 1e-13 * abs(b0[k]), k
    assert b0["ledger_detail"] == 0 and math.isnan(b0["closure"])
    s0.close()
    s1.close()


def test_accounts_survive_checkpoint(tmp_path):
    """A checkpoint carries the accounts: stepping on after a restore closes as before."""
    fdlbm = _fdlbm()
    p = W.channel(nx=48, n_gas=12, wall=4)
    s = fdlbm.Solver(p, ledger_detail=True)
    s.step(40)
    path = str(tmp_path / "ck.bin")
    s.save(path)
    s.step(40)
    b_ref = s.balance()
    s.close()
    r = fdlbm.Solver(p, ledger_detail=True)
    r.load_state(path)
    r.step(40)
    b = r.balance()
    r.close()
    for k in ("E_pop", "E_pop0", "Q_inlet", "Q_outlet", "D_interp", "D_collision", "closure"):
        assert b[k] == b_ref[k], k


def test_accounts_rejected_where_not_built():
    fdlbm = _fdlbm()

    def chan():
        return W.channel(nx=32, n_gas=8, wall=4)

    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Solver(chan(), storage="bf16", ledger_detail=True)
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Solver(W.local_transport(chan()), ledger_detail=True)
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Solver(W.periodic_box3(8, 8, 8), storage="fp16", ledger_detail=True)
    s = fdlbm.Solver(chan(), ledger_detail=True)
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Batch([s])
    s.close()


# ---------------------------------------------------------------------------------------
# D3Q19
# ---------------------------------------------------------------------------------------

def _case3(name):
    if name == "sphere_crop":
        return W.crop3(W.config2(), 32, 16, 16), 60
    kw = {"coupling": W.PAPER} if name == "closed_box_paper_coupling" else {}
    p = W.periodic_box3(14, 10, 12, solid_layers=3, **kw)
    p["init"] = W.random_fields(p, seed=3)
    return p, 30


CASES3 = ["closed_reactive_box", "closed_box_paper_coupling", "sphere_crop"]


@pytest.mark.parametrize("name", CASES3)
def test_exact_accounts3_close_and_match_oracle(name):
    """The D3Q19 step's accounts close to FP64 rounding and match the D3Q19 oracle's."""
    p, steps = _case3(name)
    s = _fdlbm().Solver(p, ledger_detail=True)
    o = oracle.Oracle3(p)
    s.step(steps)
    o.step(steps)
    b, a = s.balance(), o.accounts()
    s.close()
    scale = abs(b["E_pop"]) + abs(b["H_solid"])
    assert abs(b["closure"]) <= 1e-12 * scale, b
    assert abs(b["D_solid"]) <= 1e-8 * scale
    assert abs(b["E_pop"] - a["E_pop"]) <= 1e-6 * abs(a["E_pop"])
    flux = max(abs(a["Q_inlet"]), abs(a["Q_outlet"]), abs(a["D_interp"]), abs(a["D_collision"]), 1e-30)
    for k in ("Q_inlet", "Q_outlet", "D_interp", "D_collision"):
        assert abs(b[k] - a[k]) <= 1e-4 * flux + 1e-9 * abs(a["E_pop"]), (k, b[k], a[k])
    assert abs(b["D_coupling"] - a["D_coupling"]) <= 1e-4 * abs(a["D_coupling"]) + 1e-6 * scale


def test_accounts3_change_no_result():
    fdlbm = _fdlbm()
    p, _ = _case3("sphere_crop")
    s0, s1 = fdlbm.Solver(p), fdlbm.Solver(p, ledger_detail=True)
    s0.step(40)
    s1.step(40)
    assert np.array_equal(s0.moments_host(), s1.moments_host())
    assert np.array_equal(s0.populations(), s1.populations())
    s0.close()
    s1.close()


def test_exact_accounts_close_on_the_bench_bed():
    """The 1024x512 porous bed of the benchmark (inlet, outlet, 58,795 catalytic wall
    nodes), 1000 steps: the exact accounts close to FP64 rounding at full size."""
    s = _fdlbm().Solver(W.config1(), ledger_detail=True)
    s.step(1000)
    b = s.balance()
    s.close()
    scale = abs(b["E_pop"]) + abs(b["H_solid"])
    assert abs(b["closure"]) <= 1e-12 * scale, b
    assert b["Q_reaction"] > 0.0 and b["Q_inlet"] > 0.0
