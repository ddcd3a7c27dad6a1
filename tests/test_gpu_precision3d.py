"""Reduced-precision population storage on the D3Q19 path: FP32, FP16 and BF16
deviations (FP32 arithmetic, stochastic rounding of stored values) against the FP64
D3Q19 oracle on the 64x32x32 crop of the 256x128x128 sphere packing, 200 steps.

The paper fixes no precision: the bounds are the stated ones, about three times the
errors measured on GB300 per field (field-normalised; velocity components share the
maximum speed as their scale). FP32 storage is held to the parity bar 1e-5."""
import pytest

import oracle
from paper_1804_07588_gb300 import workloads as W
from test_gpu_parity3d import errors3

pytestmark = pytest.mark.gpu

STEPS = 200
TRACE = (2, 3)  # CO2, H2: inlet mole fraction 1e-6
# measured on GB300 (FP16; T and T_s as deviations from T_in, normalised by the oracle's
# largest deviation): major rho/X 6.3e-5, trace CO2/H2 4.5e-4, u 4.7e-4, T 6.4e-4, Ts 4.0e-4;
# BF16 about 8 times these
FP16_BOUND = {"major": 2e-4, "trace": 2.5e-3, "u": 1.5e-3, "T": 2e-3, "Ts": 1.2e-3}
BOUNDS = {"fp32": None, "fp16": FP16_BOUND, "bf16": {k: 8 * v for k, v in FP16_BOUND.items()}}


def _bound(name, b):
    if b is None:
        return 1e-5
    if name in ("ux", "uy", "uz"):
        return b["u"]
    if name in ("T", "Ts"):
        return b[name]
    j = int(name.split("_")[1])
    return b["trace"] if j in TRACE else b["major"]


@pytest.fixture(scope="module")
def oracle_crop():
    p = W.config2_crop()
    o = oracle.Oracle3(p)
    o.step(STEPS)
    return p, o


@pytest.mark.parametrize("storage", ["fp32", "fp16", "bf16"])
def test_storage3_field_errors(storage, oracle_crop):
    from paper_1804_07588_gb300 import fdlbm
    p, o = oracle_crop
    s = fdlbm.Solver(p, storage=storage)
    s.step(STEPS)
    errs = errors3(s.moments_host(t_dev=True), o.moments(), o.classes(), o.ns, T_in=o.T_inlet_K)
    print(storage, {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: v for k, v in errs.items() if v > _bound(k, BOUNDS[storage])}
    assert not bad, f"{storage}: {bad}"
    s.close()


def test_storage3_halves_population_bytes():
    from paper_1804_07588_gb300 import fdlbm
    p = W.periodic_box3(16, 8, 8)
    b32 = fdlbm.Solver(p).info()["device_bytes"]
    b16 = fdlbm.Solver(p, storage="bf16").info()["device_bytes"]
    pitch = (16 + 8 + 31) // 32 * 32
    plane = (pitch * (8 + 6) * (8 + 6) + 63) // 64 * 64
    assert b32 - b16 == 2 * 2 * 5 * 19 * plane  # two copies, 2 bytes saved per value
