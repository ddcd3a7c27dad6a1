"""The slab decomposition of the D2Q9 and D3Q19 paths (x slabs, 3-column ghost strips
exchanged by point-to-point send/recv every step, FP64 all-reduce of the totals and the
residual), checked with the FP64 oracles as every rank's slab solver: gloo ranks on CPU,
world sizes 2 and 4. The gathered moment fields must equal the undecomposed oracle's bit
for bit; the all-reduced totals and residual equal it up to the order of the additions."""
import os
import pickle
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(name):
    from paper_1804_07588_gb300 import workloads as W
    if name == "channel":  # inlet, outlet, catalytic FD walls, fixed-T faces
        p = W.channel(nx=64, n_gas=12, wall=4)
        p["init"] = W.random_fields(p, seed=71, du=0.005)
        return p
    if name == "periodic":  # periodic x and y over a catalytic slab
        p = W.periodic_box(48, 16, solid_rows=4)
        p["init"] = W.random_fields(p, seed=72)
        return p
    if name == "porous":  # digitised disks cut by the slab boundaries, paper coupling
        p = W.porous_disks(nx=100, ny=60, porosity=0.75, rmin=3.0, rmax=7.0, seed=7, u_inlet=0.01, coupling=1)
        p["init"] = W.random_fields(p, seed=73, du=0.005)
        return p
    if name == "local_tau":  # relaxation times from each node's own moments (Wilke, mixture-averaged D)
        p = W.local_transport(W.channel(nx=64, n_gas=12, wall=4))
        p["init"] = W.random_fields(p, seed=77, du=0.005)
        return p
    if name == "channel3":  # D3Q19: inlet, outlet, catalytic FD walls in y, periodic z
        nx, ng, wall, nz = 40, 8, 3, 6
        mask = np.zeros((nz, ng + 2 * wall, nx), np.uint8)
        mask[:, :wall, :] = W.CATALYTIC
        mask[:, wall + ng:, :] = W.CATALYTIC
        p = W._base(3, nx, ng + 2 * wall, nz, mask,
                    [W.INLET, W.OUTLET, W.FIXED_T, W.FIXED_T, W.PERIODIC, W.PERIODIC],
                    u_inlet=0.02, inlet_profile=W.PLUG)
        p["init"] = W.random_fields(p, seed=74, du=0.005)
        return p
    if name == "periodic3":  # D3Q19, periodic in all three axes over a catalytic slab
        p = W.periodic_box3(24, 8, 6, solid_layers=2)
        p["init"] = W.random_fields(p, seed=75)
        return p
    if name == "spheres3":  # crop of the sphere packing (cut by every slab boundary)
        p = W.config2_crop(nx=32, ny=16, nz=16)
        p["init"] = W.random_fields(p, seed=76, du=0.005)
        return p
    raise KeyError(name)


def _solver_class(p):
    import oracle
    return oracle.Oracle3 if p["dim"] == 3 else oracle.Oracle


STEPS = 30


def _rank_main(rank, world, port, name, out, halo=None):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    from paper_1804_07588_gb300 import slabs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = _problem(name)
        run = slabs.SlabRunner(p, _solver_class(p), dist, halo=slabs.HALO if halo is None else halo)
        run.residual(10)
        run.step(10)
        r1 = run.residual(10)
        run.step(STEPS - 10)
        tot = run.totals()
        m = run.gather_moments()
        out.put((rank, pickle.dumps((m, tot, r1))))
    finally:
        dist.destroy_process_group()


def _run(name, world, halo=None):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, name, q, halo)) for r in range(world)]
    for pr in procs:
        pr.start()
    res = {}
    import queue
    while len(res) < world:
        try:
            r, blob = q.get(timeout=5)
            res[r] = pickle.loads(blob)
        except queue.Empty:
            dead = [pr.exitcode for pr in procs if pr.exitcode not in (None, 0)]
            assert not dead, f"a rank failed: exit codes {dead}"
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    return res


def test_partition_is_even_and_covers_the_lattice():
    from paper_1804_07588_gb300 import slabs
    parts = slabs.partition(50, 4)
    assert parts[0][0] == 0 and parts[-1][1] == 50
    assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
    assert max(b - a for a, b in parts) - min(b - a for a, b in parts) <= 1
    assert slabs.HALO == 3
    with pytest.raises(ValueError):
        slabs.partition(11, 4)  # slabs narrower than the ghost depth


@pytest.mark.parametrize("name, world", [("channel", 2), ("channel", 4), ("periodic", 2), ("periodic", 4),
                                         ("porous", 2), ("porous", 4), ("local_tau", 2), ("channel3", 2),
                                         ("periodic3", 4),
                                         ("spheres3", 2), ("spheres3", 4)])
def test_slabs_bitwise_equal_to_monolithic(name, world):
    res = _run(name, world)
    m_slab, tot, r1 = res[0]
    p = _problem(name)
    o = _solver_class(p)(p)
    o.residual(10)
    o.step(10)
    r1_mono = o.residual(10)
    o.step(STEPS - 10)
    m_mono = o.moments()
    assert np.array_equal(m_slab, m_mono), np.abs(m_slab - m_mono).max()
    b = o.balance()
    for k in ("E_gas", "H_solid"):
        assert abs(tot[k] - b[k]) <= 1e-12 * abs(b[k]), (k, tot[k], b[k])
    for k in ("mass", "moles"):
        np.testing.assert_allclose(tot[k], b[k], rtol=1e-12)
    assert abs(r1 - r1_mono) <= 1e-10 * r1_mono, (r1, r1_mono)
    # every rank reports the same all-reduced totals
    for r in range(1, world):
        assert res[r][0] is None
        assert res[r][1]["E_gas"] == tot["E_gas"]


@pytest.mark.parametrize("name", ["porous", "channel3"])
def test_one_column_less_of_ghosts_breaks_the_decomposition(name):
    """The ghost depth is the reach of one step and no more than needed: with HALO - 1
    columns the gathered fields differ from the undecomposed run."""
    from paper_1804_07588_gb300 import slabs
    m_slab = _run(name, 2, halo=slabs.HALO - 1)[0][0]
    p = _problem(name)
    o = _solver_class(p)(p)
    o.step(STEPS)
    assert not np.array_equal(m_slab, o.moments())
