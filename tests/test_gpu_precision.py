"""Reduced-precision population storage (BF16 and FP16 deviations from the rest
equilibrium of the inlet state, FP32 arithmetic, stochastic rounding of the stored
values) against the FP64 oracle on the catalytic channel after 1000 steps.

The paper fixes no precision for this: the bounds below are the stated ones, about three
times the errors measured on GB300, per field (field-normalised: max |gpu - oracle| /
max |oracle| over gas nodes, T_s over solid nodes; T and T_s as deviations from the
inlet temperature, normalised by max |T_oracle - T_in|). The trace product species (CO2,
H2) and the transverse velocity, whose maxima are small, carry the largest relative
errors.
BF16 keeps 8 significant bits of a deviation, FP16 11 (after a power-of-two scale per
species), so BF16 bounds are 8 times the FP16 ones."""
import numpy as np
import pytest

import oracle
from paper_1804_07588_gb300 import workloads as W
from parity import field_errors

pytestmark = pytest.mark.gpu

# measured on GB300 (FP16): major 1.2e-4, trace 1.4e-3, ux 7.5e-4, uy 6.0e-3, T 1.2e-3,
# Ts 6.8e-4; BF16 about 8 times these
FP16_BOUND = {"major": 5e-4, "trace": 6e-3, "ux": 3e-3, "uy": 2e-2, "T": 4e-3, "Ts": 2e-3}
BOUNDS = {"fp16": FP16_BOUND, "bf16": {k: 8 * v for k, v in FP16_BOUND.items()}}
TRACE = (2, 3)  # CO2, H2: inlet mole fraction 1e-6


def _bound(name, b):
    if name in ("ux", "uy", "T", "Ts"):
        return b[name]
    j = int(name.split("_")[1])
    return b["trace"] if j in TRACE else b["major"]


@pytest.fixture(scope="module")
def oracle_channel_1000():
    p = W.config0()
    o = oracle.Oracle(p)
    o.step(1000)
    return p, o


@pytest.mark.parametrize("storage", ["fp16", "bf16"])
def test_reduced_storage_field_errors(storage, oracle_channel_1000):
    from paper_1804_07588_gb300 import fdlbm
    p, o = oracle_channel_1000
    s = fdlbm.Solver(p, storage=storage)
    s.step(1000)
    errs = field_errors(s.moments_host(t_dev=True), o.moments(), o.classes(), o.ns, T_in=o.T_inlet_K)
    print(storage, {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if v > _bound(k, BOUNDS[storage])}
    assert not bad, f"{storage}: {bad}"
    # stochastic rounding is unbiased: species inventories follow the oracle's
    b, bo = s.balance(), o.balance()
    drift = (b["mass"].sum() - bo["mass"].sum()) / bo["mass0"].sum()
    assert abs(drift) < (1e-5 if storage == "fp16" else 1e-4), drift
    s.close()


def test_reduced_storage_halves_population_bytes():
    from paper_1804_07588_gb300 import fdlbm
    p = W.channel(nx=64, n_gas=16, wall=4)
    b32 = fdlbm.Solver(p).info()["device_bytes"]
    b16 = fdlbm.Solver(p, storage="fp16").info()["device_bytes"]
    plane = ((64 + 16 + 31) // 32 * 32) * (24 + 8)
    plane = (plane + 63) // 64 * 64
    assert b32 - b16 == 2 * 2 * 5 * 9 * plane  # two copies, 2 bytes saved per value


def test_reduced_storage_restart_is_bitwise(tmp_path):
    """The stochastic rounding is a function of (node, population, step): a run restored
    from a checkpoint continues with the same bits."""
    from paper_1804_07588_gb300 import fdlbm
    p = W.channel(nx=48, n_gas=12, wall=3)
    a = fdlbm.Solver(p, storage="fp16")
    a.step(30)
    path = str(tmp_path / "h.ck")
    a.save(path)
    a.step(17)
    b = fdlbm.Solver(p, storage="fp16")
    b.load_state(path)
    b.step(17)
    assert np.array_equal(a.moments_host(), b.moments_host())
    # a checkpoint of another storage type does not load
    c = fdlbm.Solver(p)
    with pytest.raises(fdlbm.FdlbmError):
        c.load_state(path)
