"""Fault paths of the CUDA solver, through the C ABI, on the GPU: the wall-density
iteration cap (non-converged wall nodes are counted in the ledger, as the oracle counts
them), initial fields outside the equilibrium's range, and the strict geometry mode that
rejects the concave corners and narrow gaps the paper excludes (FDLBM_EGEOM). No case
faults the device: every failure is a status returned by the host or a count."""
import pytest

import oracle
from paper_1804_07588_gb300 import workloads as W
from parity import assert_parity

pytestmark = pytest.mark.gpu


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


def test_wall_iteration_cap_counts_nonconverged_like_the_oracle():
    """rho_w_maxit = 1: one Jacobi update per catalytic wall node cannot meet the 1e-8
    tolerance, so after one step every catalytic wall node is counted as non-converged,
    on the GPU and in the oracle (both start from the non-reactive wall density on the
    first step), and the fields still agree."""
    fdlbm = _fdlbm()
    p = W.channel(nx=48, n_gas=12, wall=4, rho_w_maxit=1)
    s = fdlbm.Solver(p)
    o = oracle.Oracle(p)
    s.step(1)
    o.step(1)
    nw = int((o.classes() == 3).sum())
    assert s.balance()["noconv"] == o.balance()["noconv"] == nw
    assert_parity(s, o, what="rho_w_maxit = 1")
    s.close()


def test_default_cap_converges():
    fdlbm = _fdlbm()
    p = W.channel(nx=48, n_gas=12, wall=4)
    s = fdlbm.Solver(p)
    o = oracle.Oracle(p)
    s.step(20)
    o.step(20)
    assert s.balance()["noconv"] == 0 and o.balance()["noconv"] == 0
    s.close()


def test_initial_fields_outside_the_equilibrium_are_rejected():
    """One node with T_lat + M_CO2 u^2 >= 1 in the initial fields: EINVAL naming it."""
    fdlbm = _fdlbm()
    p = W.periodic_box(16, 12)
    init = W.random_fields(p, seed=3)
    init["u"][0, 37] = 0.2
    p["init"] = init
    with pytest.raises(fdlbm.FdlbmError) as ei:
        fdlbm.Solver(p)
    assert ei.value.status == -1 and "node 37" in str(ei.value)
    init["u"][0, 37] = 0.0
    init["X"][:, 5] *= 1.01
    with pytest.raises(fdlbm.FdlbmError) as ei:
        fdlbm.Solver(p)
    assert ei.value.status == -1 and "node 5" in str(ei.value)


def test_strict_geometry():
    """A periodic box over a planar catalytic slab passes the strict mode; a digitised disk
    packing (concave staircase corners) is rejected with FDLBM_EGEOM, and accepted without
    it. (A channel's inlet corners also need the linear fallback: the strict mode rejects
    them too.)"""
    fdlbm = _fdlbm()
    s = fdlbm.Solver(W.periodic_box(48, 20, solid_rows=4), strict_geometry=True)
    s.close()
    with pytest.raises(fdlbm.FdlbmError) as ei:
        fdlbm.Solver(W.channel(nx=48, n_gas=12, wall=4), strict_geometry=True)
    assert ei.value.status == -2
    p = W.porous_disks(nx=100, ny=60, porosity=0.75, rmin=3.0, rmax=7.0, seed=7)
    with pytest.raises(fdlbm.FdlbmError) as ei:
        fdlbm.Solver(p, strict_geometry=True)
    assert ei.value.status == -2 and "strict geometry" in str(ei.value)
    fdlbm.Solver(p).close()
