#!/usr/bin/env python
"""Benchmark of the coupled FD-LBM solver on the 2D porous catalytic bed
(D2Q9, 1024 x 512 nodes, catalytic FD-solid disks r ~ U[6, 12], porosity 0.6, five
species CO/H2O/CO2/H2/N2 with water-gas shift on the disk surfaces, FP32 storage).

A step is one time step of the whole scheme: one launch of the step kernel, whose
blocks run the gas update and the wall + solid update. Timing: W untimed warm-up steps, then K timed steps, each preceded by an L2
flush (a 256 MB write, untimed) and bracketed by CUDA events on the solver's stream.
Prints ONE JSON line (rank 0). ``--impl reference`` times the FP64 CPU oracle instead
on a bounded crop of the same bed.

Multi-GPU (torchrun, N > 1): the problem does not need more than one GPU; every rank
runs an independent replica of the bed and the line reports the aggregate throughput
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "species-MLUPS & % HBM roofline; time-to-steady (res 1e-6) warm vs cold"
UNIT = "species-MLUPS"
# D2Q9: read 9 + write 9 populations per species-node, 4 bytes each in FP32 storage, 2 in
# BF16 / FP16 storage
BYTES_PER_VALUE = {"fp32": 4, "bf16": 2, "fp16": 2}
WORKLOAD = "porous-bed-d2q9-1024x512-5species-fp32"


WORKLOAD3 = "porous-bed-d3q19-256x128x128-5species-fp32"


def workload_name(storage, three_d=False, size="256x128x128"):
    w = WORKLOAD3.replace("256x128x128", size) if three_d else WORKLOAD
    return w if storage == "fp32" else w.replace("-fp32", f"-{storage}-storage")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="fdlbm", choices=["fdlbm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-steady", action="store_true", help="skip the time-to-steady runs")
    ap.add_argument("--workload", default="bed", choices=["bed", "batch", "bed3d"],
                    help="bed: the 1024x512 porous bed; batch: 64 independent porous beds of uneven "
                         "size stepped together (one launch per step); bed3d: the D3Q19 256x128x128 "
                         "sphere packing")
    ap.add_argument("--size", default="256x128x128",
                    help="bed3d lattice nx x ny x nz (the same sphere recipe; 256x128x128 by default)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="population storage (FP32 arithmetic in every case)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_source_hash(three_d=False):
    """Hash of the sources of the step kernel of the D2Q9 (or D3Q19) path."""
    h = hashlib.sha256()
    files = ("fdlbm_device.cuh", "fdlbm3d_device.cuh", "fdlbm3d_kernels.cu", "fdlbm_internal.h") if three_d else \
        ("fdlbm_device.cuh", "fdlbm_kernels.cu", "fdlbm_internal.h")
    for f in files:
        with open(os.path.join(ROOT, "paper_1804_07588_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(three_d=False):
    """DRAM bytes per step-kernel launch from the committed ncu summary, or None when the
    kernel source changed since the counters were taken."""
    name = "step_kernel3_traffic.json" if three_d else "step_kernel_traffic.json"
    path = os.path.join(ROOT, "profiles", name)
    try:
        with open(path) as f:
            d = json.load(f)
    except Exception:
        return None
    if d.get("kernel_source_sha") != kernel_source_hash(three_d):
        return None
    return d.get("dram_bytes_per_launch")


class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def crop_problem(n_target: int):
    """A bounded sample of the benchmark bed: the top-left crop of the same seeded disk
    packing with the last two columns opened for the outlet."""
    import numpy as np

    from paper_1804_07588_gb300 import workloads as W
    full = W.config1()
    side = max(32, int(math.sqrt(n_target)) // 8 * 8)
    w, h = min(side, 1024), min(side, 512)
    mask = full["mask"].reshape(512, 1024)[:h, :w].copy()
    mask[:, w - 2:] = W.GAS
    p = W._base(2, w, h, 1, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC],
                u_inlet=full["u_inlet"], inlet_profile=W.PLUG)
    return p, f"top-left {w}x{h} crop of the 1024x512 bed (same disk packing), outlet opened"


def oracle_throughput(seconds: float = 10.0, n_target: int = 16384, max_steps=None, three_d=False):
    import oracle
    if three_d:
        from paper_1804_07588_gb300 import workloads as W
        p = W.config2_crop()
        desc = "64x32x32 corner crop of the 256x128x128 sphere packing (same seed), outlet opened"
        o = oracle.Oracle3(p)
    else:
        p, desc = crop_problem(n_target)
        o = oracle.Oracle(p)
    n_gas = o.counts()["gas"]
    ns = len(p["species"])
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if max_steps is not None and steps >= max_steps:
            break
        if max_steps is None and el >= seconds and steps >= 3:
            break
    el = time.perf_counter() - t0
    return ns * n_gas * steps / el / 1e6, f"{desc}, {steps} steps, {n_gas} gas nodes", el


def max_over_ranks(x: float, dist=None, device="cpu") -> float:
    """The largest x over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ns: int, n_gas: int, steps: int, world: int, total_ms: float) -> float:
    """species-MLUPS of all replicas: every rank advances its own lattice `steps` times."""
    return ns * n_gas * steps * world / (total_ms * 1e-3) / 1e6


def run_to_steady(fdlbm, p, init=None, tol=1e-6, every=500, max_steps=400_000, device=0, storage="fp32"):
    """Steps and wall time (host clock around the whole loop, synchronised) for the solver
    to reach the steady-state residual tol, checked every `every` steps."""
    import torch
    s = fdlbm.Solver(p, device=device, storage=storage)
    if init is not None:
        s.set_fields(init)
    s.residual()
    torch.cuda.synchronize(device)
    t0 = time.perf_counter()
    steps, r = 0, float("inf")
    while steps < max_steps:
        s.step(every)
        steps += every
        r = s.residual()
        if r < tol:
            break
    s.sync()
    el = time.perf_counter() - t0
    return s, {"steps": steps, "seconds": el, "residual": r, "converged": r < tol}


def time_to_steady(fdlbm, workloads, device=0):
    """Cold start vs warm start on the catalytic channel (128x32 gas, 8-node walls): cold
    from the uniform initial fields, warm from the steady state of a neighbouring
    operating point (inlet velocity 0.018 instead of 0.02) passed through
    fdlbm_set_fields."""
    p = workloads.config0()
    near = workloads.config0(u_inlet=0.018)
    s_near, _ = run_to_steady(fdlbm, near, device=device)
    warm_init = s_near.restart_fields()
    s_near.close()
    s, cold = run_to_steady(fdlbm, p, device=device)
    s.close()
    s, warm = run_to_steady(fdlbm, p, init=warm_init, device=device)
    s.close()
    # Cold starts with 16-bit population storage (FP32 arithmetic), against the FP32 cold
    # start above; stochastic rounding can hold the residual above the tolerance, so
    # these runs are capped and report whether they converged.
    reduced = {}
    for storage in ("fp16", "bf16"):
        try:
            s, r = run_to_steady(fdlbm, p, device=device, storage=storage, max_steps=100_000)
            s.close()
            reduced[storage] = r
        except Exception as e:  # reported in the line, the benchmark itself goes on
            reduced[storage] = {"error": str(e)[:200]}
    return {"workload": "catalytic channel 128x32 gas + 2x8 solid rows, 5 species", "tol": 1e-6,
            "check_every": 500, "cold": cold, "warm": warm,
            "cold_fp16_storage": reduced["fp16"], "cold_bf16_storage": reduced["bf16"],
            "warm_start": "steady state of the channel at inlet velocity 0.018 (a neighbouring "
                          "operating point); the learned warm start is not built"}


def run_batch(args, rank, world, local_rank):
    """64 independent porous beds (256..1024 x 128..256, porosity 0.6-0.7, inlet 0.005-0.03,
    450-600 K) advanced together by one batch (one kernel launch per step from a captured
    graph) against the same solvers stepped one launch each per step. Host clock around
    K synchronised steps; the working set (GBs) is far larger than L2."""
    import torch

    from paper_1804_07588_gb300 import fdlbm, workloads
    if world > 1 and rank != 0:
        return
    dev = local_rank
    torch.cuda.set_device(dev)
    probs = workloads.batch_instances()
    solvers = [fdlbm.Solver(p, device=dev, storage=args.storage, band_rows="auto") for p in probs]
    infos = [s.info() for s in solvers]
    ns = infos[0]["ns"]
    units = sum(ns * i["n_gas"] for i in infos)
    batch = fdlbm.Batch(solvers)
    batch.step(args.warmup)
    for s in solvers:
        s.sync()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev)
    clocks.start()
    t0 = time.perf_counter()
    batch.step(args.steps)
    for s in solvers:
        s.sync()
    el_batch = time.perf_counter() - t0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in solvers:
            s.step(1)
    for s in solvers:
        s.sync()
    el_seq = time.perf_counter() - t0
    clk = clocks.stop()
    batch.close()
    value = units * args.steps / el_batch / 1e6
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": el_batch / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batch-64-porous-d2q9-5species-{args.storage}-storage", "instances": len(solvers),
                   "nodes": int(sum(i["n_nodes"] for i in infos)), "gas_nodes": int(sum(i["n_gas"] for i in infos)),
                   "l2": "working set far larger than L2", "timing": "host clock around synchronised steps",
                   "band_rows": "autotuned per member (nearest entry of the GB300 table)"},
        "sequential": {"value": units * args.steps / el_seq / 1e6, "ms_per_step": el_seq / args.steps * 1e3,
                       "what": "the same solvers stepped one launch each per step"},
        "gpu_launches": 2 * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    for s in solvers:
        s.close()


def run_reference(args, rank, world):
    if rank != 0:
        return
    # each step a bounded sample: the crop is sized so that W + K oracle steps take about
    # a minute or two on one host core.
    total = max(args.steps + args.warmup, 1)
    n_target = int(max(1024, min(65536, 40e6 / total)))
    import oracle
    p, desc = crop_problem(n_target)
    o = oracle.Oracle(p)
    n_gas = o.counts()["gas"]
    ns = len(p["species"])
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    value = ns * n_gas * args.steps / el / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": el / max(args.steps, 1) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc, "oracle": "plain FP64 C, one host core"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_fdlbm(args, rank, world, local_rank):
    import torch

    from paper_1804_07588_gb300 import fdlbm, workloads
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local_rank}"))
    dev = local_rank
    torch.cuda.set_device(dev)
    three_d = args.workload == "bed3d"
    if three_d:
        nx3, ny3, nz3 = (int(v) for v in args.size.split("x"))
        p = workloads.config2(nx=nx3, ny=ny3, nz=nz3)
    else:
        p = workloads.config1()
    Q = 19 if three_d else 9
    s = fdlbm.Solver(p, device=dev, storage=args.storage)
    info = s.info()
    ns = info["ns"]
    n_gas = info["n_gas"]
    stream = s.stream
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float32, device=f"cuda:{dev}")  # 256 MB > L2
    s.step(args.warmup)
    s.sync()
    s.profile(True)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize(dev)
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
        starts[k].record(stream)
        s.step(1)
        ends[k].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    total_ms = sum(a.elapsed_time(b) for a, b in zip(starts, ends))
    ms_step, timed = s.kernel_times()
    s.profile(False)
    s.sync()
    total_ms = max_over_ranks(total_ms, dist, device=f"cuda:{dev}")
    value = whole_job_value(ns, n_gas, args.steps, world, total_ms)
    step_kernel_ms = ms_step / max(timed, 1)
    alg_bytes = 2 * Q * BYTES_PER_VALUE[args.storage] * ns * n_gas
    achieved = alg_bytes / (step_kernel_ms * 1e-3) / 1e9
    peak, peak_kind = measured_peaks()

    e2e = None
    if not args.no_e2e:
        import numpy as np
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s2 = fdlbm.Solver(p, device=dev, storage=args.storage)
        s2.step(args.steps)
        m = s2.moments_host()
        s2.sync()
        el = time.perf_counter() - t0
        n = info["n_nodes"]
        if three_d:
            # mask, FP64 initial fields (X, u, T, Ts, C), inlet state, 64-bit code words of the
            # padded lattice, gas list, solid list, block table
            blocks = (n_gas + 127) // 128 + (info["n_wall"] + info["n_solid"]) // 128 + p["nz"] + 1
            pitch = (p["nx"] + 8 + 31) // 32 * 32
            plane = pitch * (p["ny"] + 6) * (p["nz"] + 6)
            h2d = n + 8 * (ns + 6) * n + 8 * (ns + 2) + 8 * plane + 8 * n_gas + \
                4 * (info["n_wall"] + info["n_solid"]) + 16 * blocks
        else:
            h2d = 4 * n + 4 * (info["n_wall"] + info["n_solid"]) + 8 * (ns + 5) * n + 8 * (p["ny"] + ns + 1) + n
        d2h = m.nbytes
        e2e = {"value": ns * n_gas * args.steps / el / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "what": "whole job through the C ABI: fdlbm_create from host arrays (geometry, "
                       "initial fields), K steps, moment fields read back to host"}
        s2.close()
        del np

    tts = None
    if rank == 0 and not args.no_steady and not three_d:
        tts = time_to_steady(fdlbm, workloads, device=dev)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, el = oracle_throughput(seconds=10.0, three_d=three_d)
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
               "seconds": round(el, 2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_name(args.storage, three_d, args.size), "nx": p["nx"], "ny": p["ny"],
                       **({"nz": p["nz"], "lattice": "D3Q19"} if three_d else {"lattice": "D2Q9"}),
                       "porosity": 0.5 if three_d else 0.6,
                       "storage": {"fp32": "FP32 deviations", "bf16": "BF16 deviations, stochastic rounding",
                                   "fp16": "FP16 deviations (power-of-two scale per species), stochastic "
                                           "rounding"}[args.storage],
                       "species": ns, "gas_nodes": n_gas, "wall_nodes": info["n_wall"],
                       "solid_nodes": info["n_solid"], "l2": "flushed (256 MB write) before every timed step",
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "roofline": {"bound": "hbm", "kernel": "step_kernel", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": ncu_traffic(three_d) if args.storage == "fp32" else None,
                         "peak_kind": peak_kind + " copy bandwidth",
                         "alg_bytes_per_launch": alg_bytes, "kernel_ms_per_launch": step_kernel_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps,
            "time_to_steady": tts,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    s.close()
    if dist is not None:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch":
        run_batch(args, rank, world, local_rank)
        return
    run_fdlbm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
