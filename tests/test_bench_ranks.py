"""The multi-rank logic of bench.py on CPU: two gloo ranks (replicas) agree on the
slowest rank's time and report the whole job's throughput; the reference arm runs on
rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = [40.0, 55.0][rank]
    t = bench.max_over_ranks(my_ms, dist)
    v = bench.whole_job_value(5, 1000, 100, world, t)
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, t, v))


def test_two_gloo_ranks_max_time_and_whole_job_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v in res:
        assert t == 55.0
        # 2 ranks x 5 species x 1000 gas nodes x 100 steps in 55 ms
        assert v == pytest.approx(2 * 5 * 1000 * 100 / 0.055 / 1e6)


def test_single_rank_value_has_no_collective():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.whole_job_value(5, 313539, 1000, 1, 119.0) == pytest.approx(13173.9, rel=1e-4)


def test_reference_arm_other_ranks_do_nothing(capsys):
    import sys
    sys.path.insert(0, ROOT)
    import argparse

    import bench
    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_traffic_record_holds_for_its_source_and_listed_equivalents():
    import bench
    rec = {"kernel_source_sha": "aaaa", "also_valid_for": [{"sha": "bbbb", "why": "unchanged kernels"}]}
    assert bench.traffic_record_holds(rec, "aaaa") and bench.traffic_record_holds(rec, "bbbb")
    assert not bench.traffic_record_holds(rec, "cccc")
    assert not bench.traffic_record_holds({"kernel_source_sha": "aaaa"}, "bbbb")


def test_steady_runs_close_their_solver_when_a_step_raises(monkeypatch):
    """bench.run_to_steady and bench.precision_handoff close the solver they created
    when a step raises, and let the error through (a stand-in solver, no GPU)."""
    import torch

    import bench
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    closed = []

    class Boom(RuntimeError):
        pass

    class FakeSolver:
        def __init__(self, p, device=0, storage="fp32"):
            pass

        def set_fields(self, f):
            pass

        def residual(self):
            return float("inf")

        def step(self, n):
            raise Boom("step failed")

        def sync(self):
            pass

        def restart_fields(self):
            return {}

        def close(self):
            closed.append(self)

    class FakeModule:
        Solver = FakeSolver

    with pytest.raises(Boom):
        bench.run_to_steady(FakeModule, {}, init={"X": None})
    assert len(closed) == 1
    with pytest.raises(Boom):
        bench.precision_handoff(FakeModule, {}, "fp16")
    assert len(closed) == 2
