"""Host-side validation of fdlbm_create (no GPU needed: every check below fails before
the library touches a device). Each case takes a valid problem, breaks one input, and
expects FDLBM_EINVAL (-1) with a message naming the input."""
import copy
import ctypes as C

import pytest

from paper_1804_07588_gb300 import fdlbm
from paper_1804_07588_gb300 import workloads as W

EINVAL = -1


def _create_status(p):
    L = fdlbm.load()
    keep = []
    g, spec, ns, tr, kin, fields = fdlbm.create_args(p, keep)
    h = C.c_void_p()
    st = L.fdlbm_create(C.byref(g), spec, ns, C.byref(tr), C.byref(kin), C.byref(fields), None, C.byref(h))
    assert not h.value
    return st, L.fdlbm_last_error().decode()


def _channel():
    return W.channel(nx=32, n_gas=8, wall=4)


def _with_species(p, j, **kw):
    q = copy.deepcopy(p)
    q["species"][j].update(kw)
    return q


@pytest.mark.parametrize("case, what", [
    (lambda p: _with_species(p, 0, tau1=0.0), "tau1"),
    (lambda p: _with_species(p, 2, tau2=-0.5), "tau2"),
    (lambda p: _with_species(p, 4, X_init=0.7), "sum to 1"),
    (lambda p: _with_species(p, 4, X_inlet=0.9), "sum to 1"),
    (lambda p: _with_species(p, 0, X_init=-0.1), "[0, 1]"),
    (lambda p: dict(p, T_inlet_K=3.0 * p["T0_K"] * 1.01), "equilibrium"),
    (lambda p: dict(p, u_inlet=0.2), "equilibrium"),
    (lambda p: dict(p, T_init_K=3.0 * p["T0_K"]), "equilibrium"),
    (lambda p: dict(p, Pr=0.0), "Pr"),
    (lambda p: dict(p, rho_w_maxit=0), "rho_w_maxit"),
    (lambda p: dict(p, alpha_s=0.3), "alpha_s"),
])
def test_create_rejects_invalid_inputs(case, what):
    st, msg = _create_status(case(_channel()))
    assert st == EINVAL, (st, msg)
    assert what.split()[0].lower() in msg.lower() or what in msg, msg


def test_heaviest_species_sets_the_velocity_limit():
    """1 - M u^2 - T > 0 for the heaviest species (CO2, 21.83 times H2's mass) at the inlet
    temperature T = 1/3 holds up to u = 0.1747: u_inlet = 0.18 is outside."""
    st, msg = _create_status(dict(_channel(), u_inlet=0.18))
    assert st == EINVAL and "equilibrium" in msg
