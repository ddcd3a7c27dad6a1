"""Batched stepping through the C ABI (fdlbm_batch_*): members of different sizes,
geometries and parameters advanced in one launch per step give the same bits as each
member stepped on its own (same kernels, same per-block ledger slots), and a member
matches the FP64 oracle."""
import numpy as np
import pytest

from paper_1804_07588_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _fdlbm():
    from paper_1804_07588_gb300 import fdlbm
    return fdlbm


def _problems():
    a = W.channel(nx=64, n_gas=16, wall=4)
    b = W.porous_disks(nx=100, ny=60, porosity=0.75, rmin=3.0, rmax=7.0, seed=7, u_inlet=0.01)
    b["init"] = W.random_fields(b, seed=51, du=0.005)
    c = W.periodic_box(40, 28, solid_rows=5)
    c["init"] = W.random_fields(c, seed=52)
    d = W.channel(nx=48, n_gas=12, wall=3, u_inlet=0.03, coupling=W.PAPER)
    return [a, b, c, d]


def _same(s, t):
    assert np.array_equal(s.moments_host(), t.moments_host())
    assert np.array_equal(s.populations(), t.populations())
    bs, bt = s.balance(), t.balance()
    for k in ("Q_reaction", "Q_wall", "Q_couple", "Q_fixedT", "noconv", "steps"):
        assert bs[k] == bt[k], k


@pytest.mark.parametrize("steps", [37, 40])
def test_batch_matches_members_stepped_alone(steps):
    fdlbm = _fdlbm()
    probs = _problems()
    batched = [fdlbm.Solver(p) for p in probs]
    alone = [fdlbm.Solver(p) for p in probs]
    batch = fdlbm.Batch(batched)
    assert len(batch) == 4
    batch.step(steps)            # >= 16: graph replay plus single launches
    for s in alone:
        s.step(steps)
    for s, t in zip(batched, alone):
        _same(s, t)
    batch.close()


def test_batch_remove_and_members_stepped_outside():
    fdlbm = _fdlbm()
    probs = _problems()[:3]
    batched = [fdlbm.Solver(p) for p in probs]
    alone = [fdlbm.Solver(p) for p in probs]
    batch = fdlbm.Batch(batched)
    batch.step(20)
    batch.remove(batched[1])
    assert len(batch) == 2
    batch.step(5)
    batched[0].step(3)           # a member stepped on its own in between
    batch.step(18)
    alone[0].step(46)
    alone[1].step(20)
    alone[2].step(43)
    for s, t in zip(batched, alone):
        _same(s, t)
    batch.close()


def test_batch_fp16_members():
    fdlbm = _fdlbm()
    probs = _problems()[:2]
    batched = [fdlbm.Solver(p, storage="fp16") for p in probs]
    alone = [fdlbm.Solver(p, storage="fp16") for p in probs]
    batch = fdlbm.Batch(batched)
    batch.step(33)
    for s in alone:
        s.step(33)
    for s, t in zip(batched, alone):
        assert np.array_equal(s.moments_host(), t.moments_host())
    batch.close()


def test_batch_rejects_incompatible_members():
    fdlbm = _fdlbm()
    p = W.channel(nx=48, n_gas=12, wall=3)
    q = W.channel(nx=48, n_gas=12, wall=3, reactions=[])
    q["species"] = q["species"][:4]
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Batch([fdlbm.Solver(p), fdlbm.Solver(q)])
    s = fdlbm.Solver(p)
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Batch([s, s])
    with pytest.raises(fdlbm.FdlbmError):
        fdlbm.Batch([fdlbm.Solver(p), fdlbm.Solver(p, storage="bf16")])


def test_batch_member_matches_the_oracle():
    """Every member of a batch after 300 batched steps against the FP64 oracle of the same
    problem (the parity bar of the solver stepped alone)."""
    import oracle
    from parity import assert_parity
    fdlbm = _fdlbm()
    probs = _problems()
    members = [fdlbm.Solver(p) for p in probs]
    b = fdlbm.Batch(members)
    b.step(300)
    for s in members:
        s.sync()
    b.close()
    for p, s in zip(probs, members):
        o = oracle.Oracle(p)
        o.step(300)
        assert_parity(s, o, what="batch member")
        s.close()


def test_batch_runs_members_to_steady_and_removes_them():
    """Six small beds of uneven size and inlet velocity run to residual 1e-5 in one batch:
    a member below the tolerance leaves the batch at the check where it got there and is
    not advanced further (its step count stays there), the others go on; at least four of
    the six get there within 100,000 steps."""
    fdlbm = _fdlbm()
    probs = W.batch_instances(n=6, seed=77, nx_range=(96, 160), ny_range=(48, 64), porosity=(0.5, 0.7),
                              u_inlet=(0.02, 0.03))
    solvers = [fdlbm.Solver(p) for p in probs]
    b = fdlbm.Batch(solvers)
    res = b.run_to_steady(tol=1e-5, every=1000, max_steps=100_000)
    remaining = len(b)
    b.close()
    conv = [r for r in res if r["converged"]]
    assert len(conv) >= 4, res
    assert remaining == len(res) - len(conv) - sum(r["unstable"] for r in res)
    for s, r in zip(solvers, res):
        assert not r["unstable"]
        assert s.info()["steps"] == r["steps"]
        if r["converged"]:
            assert r["residual"] < 1e-5
        else:
            assert r["steps"] == 100_000
        s.close()
    assert len({r["steps"] for r in conv}) > 1  # members leave at different times


@pytest.mark.parametrize("band, tile, order", [(8, 128, 0), (32, 192, 1), (5, 64, 1)])
def test_block_order_gives_the_same_bits(band, tile, order):
    """The step kernel's block order (band height, gas nodes per tile, wall blocks per
    band or last) changes which block does a node's work, not the node's arithmetic:
    populations and moments are bit-identical to the default order's; the FP64 ledger
    sums its per-block slots in another grouping, so it agrees to rounding."""
    fdlbm = _fdlbm()
    p = W.porous_disks(nx=192, ny=96, porosity=0.65, seed=41)
    p["init"] = W.random_fields(p, seed=9, du=0.005)
    a = fdlbm.Solver(p)
    b = fdlbm.Solver(p, band_rows=band, tile_entries=tile, wall_order=order)
    for s in (a, b):
        s.step(150)
        s.sync()
    assert np.array_equal(a.populations().view(np.uint32), b.populations().view(np.uint32))
    assert np.array_equal(a.moments_host().view(np.uint32), b.moments_host().view(np.uint32))
    la, lb = a.balance(), b.balance()
    fin = {k: v for k, v in la.items() if isinstance(v, float) and np.isfinite(v)}  # kept accounts only
    scale = max(abs(v) for v in fin.values())
    for k, v in fin.items():
        assert abs(v - lb[k]) <= 1e-12 * scale, k
    a.close()
    b.close()


def test_block_order_options_are_validated():
    fdlbm = _fdlbm()
    p = W.periodic_box(32, 16)
    for kw in ({"tile_entries": 100}, {"tile_entries": 32}, {"tile_entries": 512}, {"wall_order": 2}):
        with pytest.raises(fdlbm.FdlbmError):
            fdlbm.Solver(p, **kw)
