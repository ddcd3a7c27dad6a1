"""The allocation-free totals entry point (fdlbm_totals_static) against the ledger
entry point (fdlbm_enthalpy_balance), both through the C ABI.

Both reduce the same FP32 device fields in FP64; only the order of the additions
differs (fixed block order here, atomics there), so the totals agree to a few units in
the last place: relative tolerance 1e-12. The file is named so that pytest collects it
last, and it also passes alone in a fresh process (the first call does the per-device
set-up)."""
import ctypes as C

import numpy as np
import pytest

from paper_1804_07588_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-12


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


def _compare(t, b):
    for k in ("E_gas", "H_solid"):
        assert abs(t[k] - b[k]) <= RTOL * abs(b[k]), (k, t[k], b[k])
    for k in ("mass", "moles"):
        np.testing.assert_allclose(t[k], b[k], rtol=RTOL, atol=RTOL * np.abs(b[k]).sum())


@pytest.mark.parametrize("storage", ["fp32", "bf16", "fp16"])
def test_totals_static_two_calls_match_balance(storage):
    """Reactive closed box with interface walls (wall emissions in transit count):
    two consecutive calls, then one more after further steps; FP32, BF16 and FP16
    population storage (the 16-bit forms decode the wall emissions in transit)."""
    fdlbm = _fdlbm()
    p = W.periodic_box(60, 20, solid_rows=6)
    p["init"] = W.random_fields(p, seed=31)
    s = fdlbm.Solver(p, storage=storage)
    s.step(25)
    t1 = s.totals_static()
    t2 = s.totals_static()
    b = s.balance()
    _compare(t1, b)
    _compare(t2, b)
    # fixed reduction order: identical bits on the same state
    assert t1["E_gas"] == t2["E_gas"] and t1["H_solid"] == t2["H_solid"]
    assert np.array_equal(t1["mass"], t2["mass"]) and np.array_equal(t1["moles"], t2["moles"])
    s.step(10)
    _compare(s.totals_static(), s.balance())
    s.close()


def test_totals_static_matches_oracle():
    """The same totals from the FP64 oracle after the same steps: the FP32 state's
    inventories agree with the oracle's to the parity level of the ledger (1e-6 of the
    energy inventories, 1e-6 of the total mass and moles)."""
    import oracle
    fdlbm = _fdlbm()
    p = W.periodic_box(60, 20, solid_rows=6)
    p["init"] = W.random_fields(p, seed=31)
    s = fdlbm.Solver(p)
    o = oracle.Oracle(p)
    s.step(25)
    o.step(25)
    t, b = s.totals_static(), o.balance()
    for k in ("E_gas", "H_solid"):
        assert abs(t[k] - b[k]) <= 1e-6 * abs(b[k]), (k, t[k], b[k])
    for k in ("mass", "moles"):
        np.testing.assert_allclose(t[k], b[k], rtol=0, atol=1e-6 * np.abs(b[k]).sum())
    s.close()


def test_totals_static_channel_with_inlet_outlet():
    fdlbm = _fdlbm()
    p = W.channel(nx=96, n_gas=24, wall=4)
    s = fdlbm.Solver(p)
    s.step(40)
    _compare(s.totals_static(), s.balance())
    s.close()


def test_totals_static_rejects_short_output():
    fdlbm = _fdlbm()
    p = W.periodic_box(32, 16, solid_rows=4)
    s = fdlbm.Solver(p)
    out = (C.c_double * 1)()
    status = fdlbm.load().fdlbm_totals_static(s._h, out, 1)
    assert status == -1
    assert b"out_len" in fdlbm.load().fdlbm_last_error()
    s.close()


def test_totals_static_rejects_lattice_over_the_limit():
    """1024 x 700 nodes with 5 species need (2800 + 1) x 12 doubles = 268,896 bytes of
    scratch, above the 262,144-byte limit: EINVAL with both sizes in the message."""
    fdlbm = _fdlbm()
    p = W.periodic_box(1024, 700, solid_rows=8)
    assert len(p["species"]) == 5
    s = fdlbm.Solver(p)
    with pytest.raises(fdlbm.FdlbmError) as ei:
        s.totals_static()
    assert ei.value.status == -1
    msg = str(ei.value)
    assert "268896" in msg and "262144" in msg
    s.close()
