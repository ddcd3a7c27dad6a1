"""The learned warm start: the host-side encoding on CPU (instances, network input,
target and its inverse), and on the GPU the pipeline end to end (steady fields from the
solver, training with the library's tensor-core kernels, prediction for an unseen
geometry, warm-started solver run)."""
import numpy as np
import pytest

from paper_1804_07588_gb300 import warmstart as WS


def test_instances_are_seeded_and_percolating():
    a = WS.instances(3, 123)
    b = WS.instances(3, 123)
    for p, q in zip(a, b):
        assert np.array_equal(p["mask"], q["mask"]) and p["u_inlet"] == q["u_inlet"]
        assert (p["nx"], p["ny"], p["nz"]) == WS.SHAPE
        assert 0.005 <= p["u_inlet"] <= 0.03 and 450 <= p["T_inlet_K"] <= 600
        solid = 1.0 - (np.asarray(p["mask"]) == 0).mean()
        assert 0.38 <= solid <= 0.57  # porosity 0.45-0.6 of the lattice, digitised


def test_encoding_round_trip():
    """fields_from_prediction(target_fields(m)) gives back the velocity, mole fractions
    and temperatures of m on gas nodes and the solid temperature on solid nodes."""
    p = WS.instances(1, 321)[0]
    ns = len(p["species"])
    n = p["nx"] * p["ny"] * p["nz"]
    rng = np.random.default_rng(5)
    solid = np.asarray(p["mask"]).reshape(n) > 0
    Xin = np.array([s["X_inlet"] for s in p["species"]])
    m = np.zeros((2 * ns + 5, n))
    X = Xin[:, None] * (1 + 0.05 * rng.normal(size=(ns, n)))
    X /= X.sum(0, keepdims=True)
    m[ns:2 * ns] = np.where(solid[None], 0.0, X)
    m[2 * ns:2 * ns + 3] = np.where(solid[None], 0.0, 0.01 * rng.normal(size=(3, n)))
    m[2 * ns + 3] = np.where(solid, 0.0, 5 * rng.normal(size=n))
    m[2 * ns + 4] = np.where(solid, 5 * rng.normal(size=n), 0.0)
    y = WS.target_fields(p, m)
    assert y.shape == (p["nz"], p["ny"], p["nx"], WS.N_OUT)
    f = WS.fields_from_prediction(p, y)
    gas = ~solid
    np.testing.assert_allclose(f["u"][:, gas], m[2 * ns:2 * ns + 3][:, gas], rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(f["X"][:, gas], X[:, gas], rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(f["T_K"][gas], p["T_inlet_K"] + m[2 * ns + 3][gas], rtol=1e-6)
    np.testing.assert_allclose(f["Ts_K"][solid], p["T_inlet_K"] + m[2 * ns + 4][solid], rtol=1e-6)
    x = WS.network_input(p)
    assert x.shape == (p["nz"], p["ny"], p["nx"], 16)
    assert np.array_equal(x[..., 0].reshape(n) > 0, solid)


@pytest.mark.gpu
def test_trained_network_predicts_unseen_steady_fields():
    """Six training packings run cold to residual 1e-5, the network trained on them for
    300 Adam steps; on an unseen packing its prediction lies closer to the steady fields
    than the cold start's uniform state (less than half its distance), and a solver run
    started from the prediction reaches the residual."""
    tol = 1e-5
    data = WS.generate(WS.instances(6, 5000), tol=tol, max_steps=80_000)
    assert sum(d["stats"]["converged"] for d in data) >= 4
    model = WS.new_model(1)
    losses = WS.train(model, data, iters=300)
    assert losses[-1] < 0.2 * losses[0]
    q = WS.instances(1, 9000)[0]
    steady = WS.generate([q], tol=tol, max_steps=80_000)[0]
    y = steady["y"]
    pred = WS.predict(model, q)
    cold = np.zeros_like(y)  # the cold start: gas at rest at the inlet state
    err_pred = float(np.sqrt(np.mean((pred - y) ** 2)))
    err_cold = float(np.sqrt(np.mean((cold - y) ** 2)))
    assert err_pred < 0.5 * err_cold, (err_pred, err_cold)
    r = WS.warm_vs_cold(model, q, tol=tol, max_steps=80_000)
    print("warm start", r)
    assert r["cold"]["converged"]
    assert r["warm"]["converged"] or r["warm"]["fallback"]


def test_solve_closes_its_solver_on_errors(monkeypatch):
    """warmstart.solve with a stand-in solver (no GPU): a failed field upload closes the
    solver and raises; a solver error in a step counts as a diverged run and returns the
    solver; any other error in a step closes it and raises."""
    import torch

    from paper_1804_07588_gb300 import fdlbm
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    closed = []
    mode = {}

    class FakeSolver:
        def __init__(self, p, device=0):
            pass

        def set_fields(self, f):
            if mode.get("upload"):
                raise ValueError("bad fields")

        def residual(self):
            return 1.0

        def step(self, n):
            raise mode["step"]

        def sync(self):
            pass

        def close(self):
            closed.append(self)

    monkeypatch.setattr(fdlbm, "Solver", FakeSolver)
    mode.update(upload=True, step=RuntimeError("unused"))
    with pytest.raises(ValueError):
        WS.solve({}, init={"X": None})
    assert len(closed) == 1
    mode.update(upload=False, step=fdlbm.FdlbmError(-5, "unstable"))
    s, st = WS.solve({}, init={"X": None})
    assert st["diverged"] and not st["converged"] and len(closed) == 1
    mode.update(step=KeyError("other"))
    with pytest.raises(KeyError):
        WS.solve({})
    assert len(closed) == 2


def test_rejected_prediction_falls_back_to_the_cold_run(monkeypatch):
    """A prediction whose fields the solver rejects (stand-in solver, no GPU) is counted
    like a diverged warm run: its cost plus the cold run."""
    import torch

    from paper_1804_07588_gb300 import fdlbm
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    monkeypatch.setattr(WS, "predict", lambda model, p: None)
    monkeypatch.setattr(WS, "fields_from_prediction", lambda p, y: {"X": None})

    class FakeSolver:
        def __init__(self, p, device=0):
            self.r = 1.0

        def set_fields(self, f):
            raise fdlbm.FdlbmError(-1, "fields outside the equilibrium's range")

        def residual(self):
            return self.r

        def step(self, n):
            self.r *= 1e-3

        def sync(self):
            pass

        def close(self):
            pass

    monkeypatch.setattr(fdlbm, "Solver", FakeSolver)
    r = WS.warm_vs_cold(None, {}, tol=1e-6, every=10)
    assert r["cold"]["converged"] and r["cold"]["steps"] == 30      # residual 1e-9 at the third check
    assert r["warm"]["fallback"] and "rejected" in r["warm"]
    assert r["warm"]["steps"] == r["cold"]["steps"] and r["warm"]["seconds"] >= r["cold"]["seconds"]
