"""Checkpoint and restore through the C ABI (fdlbm_save / fdlbm_load): a run restored
from a checkpoint continues with the same bits as the run that wrote it."""
import numpy as np
import pytest

from paper_1804_07588_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


@pytest.mark.parametrize("coupling", [W.CONSERVATIVE, W.PAPER])
def test_restart_is_bitwise(tmp_path, coupling):
    fdlbm = _fdlbm()
    p = W.channel(nx=72, n_gas=20, wall=4, coupling=coupling)
    p_init = dict(p)
    p_init["init"] = W.random_fields(p, seed=41, du=0.005)
    a = fdlbm.Solver(p_init)
    a.step(37)
    a.residual()          # take a residual snapshot before the checkpoint
    a.step(5)
    path = str(tmp_path / "state.ck")
    a.save(path)
    a.step(23)
    ma, pa, ba, ra = a.moments_host(), a.populations(), a.balance(), a.residual()
    # a handle of the same problem without the initial fields: everything the next
    # step reads comes from the file
    b = fdlbm.Solver(p)
    b.load_state(path)
    b.step(23)
    mb, pb, bb, rb = b.moments_host(), b.populations(), b.balance(), b.residual()
    gas = np.asarray(p["mask"]).ravel() == W.GAS
    assert np.array_equal(ma, mb)
    assert np.array_equal(pa[:, :, gas], pb[:, :, gas])
    # the ledger's totals are summed with FP64 atomics (order varies between launches):
    # equal to rounding; the fixed-order reduction gives the same bits. The residuals are
    # differences of those totals, so their rounding is relative to the totals' size
    scale = abs(ba["E_gas"]) + abs(ba["H_solid"])
    derived = {"residual": scale, "solid_residual": scale,
               "eps_paper": scale / max(abs(ba["Q_reaction"]), 1e-300)}
    for k, v in ba.items():
        atol = 1e-12 * derived[k] if k in derived else 0.0
        np.testing.assert_allclose(np.asarray(v), np.asarray(bb[k]), rtol=1e-12, atol=atol, err_msg=k)
    ta, tb = a.totals_static(), b.totals_static()
    for k in ta:
        assert np.array_equal(np.asarray(ta[k]), np.asarray(tb[k])), k
    assert ra == pytest.approx(rb, rel=1e-12)  # residual sums use FP64 atomics too
    assert bb["steps"] == 65
    a.close()
    b.close()


def test_load_rejects_other_problem_and_missing_file(tmp_path):
    fdlbm = _fdlbm()
    a = fdlbm.Solver(W.channel(nx=48, n_gas=12, wall=3))
    a.step(3)
    path = str(tmp_path / "a.ck")
    a.save(path)
    other = fdlbm.Solver(W.channel(nx=48, n_gas=12, wall=3, u_inlet=0.01))
    with pytest.raises(fdlbm.FdlbmError) as ei:
        other.load_state(path)
    assert ei.value.status == -1
    with pytest.raises(fdlbm.FdlbmError) as ei:
        other.load_state(str(tmp_path / "missing.ck"))
    assert ei.value.status == -8
    a.close()
    other.close()


def test_restart_fields_warm_start():
    """The state of one solver as initial fields of another (fdlbm_set_fields): the new
    solver starts from the same moment fields (equilibrium populations of them)."""
    fdlbm = _fdlbm()
    p = W.channel(nx=64, n_gas=16, wall=4)
    a = fdlbm.Solver(p)
    a.step(120)
    f = a.restart_fields()
    ma = a.moments_host().astype(np.float64)
    b = fdlbm.Solver(p)
    b.set_fields(f)
    mb = b.moments_host().astype(np.float64)
    ns = a.ns
    for row in list(range(ns, 2 * ns)) + [2 * ns, 2 * ns + 1, 2 * ns + 2, 2 * ns + 3]:
        scale = np.abs(ma[row]).max()
        assert np.abs(ma[row] - mb[row]).max() <= 2e-6 * scale, row
    a.close()
    b.close()
