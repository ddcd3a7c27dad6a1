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
    ap.add_argument("--no-variants", action="store_true", help="skip the 3D and 16-bit storage workloads")
    ap.add_argument("--workload", default="bed", choices=["bed", "batch", "bed3d"],
                    help="bed: the 1024x512 porous bed; batch: 64 independent porous beds of uneven "
                         "size stepped together (one launch per step); bed3d: the D3Q19 256x128x128 "
                         "sphere packing")
    ap.add_argument("--size", default="256x128x128",
                    help="bed3d lattice nx x ny x nz (the same sphere recipe; 256x128x128 by default)")
    ap.add_argument("--storage", default="fp32", choices=["fp32", "bf16", "fp16"],
                    help="population storage (FP32 arithmetic in every case)")
    ap.add_argument("--steady-cap", type=int, default=0,
                    help="batch workload: after the timed steps, run every member to residual 1e-6 "
                         "(members leave the batch once there) for at most this many steps; 0: skip")
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


def traffic_record_holds(rec, sha):
    """A traffic record holds for the source it was captured on and for the later sources
    it lists under also_valid_for, each with the reason the measured kernels are unchanged."""
    return rec.get("kernel_source_sha") == sha or any(v.get("sha") == sha for v in rec.get("also_valid_for", []))


def variant_traffic(name, three_d):
    """DRAM bytes per step of a bench variant from the committed ncu table, or None when the
    kernel source changed since the counters were taken."""
    try:
        with open(os.path.join(ROOT, "profiles", "variant_traffic.json")) as f:
            e = json.load(f)["variants"][name]
    except Exception:
        return None
    return e["dram_bytes_per_step"] if traffic_record_holds(e, kernel_source_hash(three_d)) else None


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
    if not traffic_record_holds(d, kernel_source_hash(three_d)):
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


def crop_problem(n_target: int, x0: int = 0):
    """A bounded sample of the benchmark bed: the crop at columns x0.. of the top rows of
    the same seeded disk packing, with the last two columns opened for the outlet."""
    import numpy as np

    from paper_1804_07588_gb300 import workloads as W
    full = W.config1()
    side = max(32, int(math.sqrt(n_target)) // 8 * 8)
    w, h = min(side, 1024 - x0), min(side, 512)
    mask = full["mask"].reshape(512, 1024)[:h, x0:x0 + w].copy()
    mask[:, w - 2:] = W.GAS
    p = W._base(2, w, h, 1, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC],
                u_inlet=full["u_inlet"], inlet_profile=W.PLUG)
    return p, f"{w}x{h} crop at column {x0} of the top rows of the 1024x512 bed (same disk packing), outlet opened"


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
    try:
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
    except BaseException:
        s.close()                       # the caller never sees this solver
        raise
    return s, {"steps": steps, "seconds": el, "residual": r, "converged": r < tol}


def time_to_steady(fdlbm, workloads, device=0):
    """Cold start vs warm start on the catalytic channel (128x32 gas, 8-node walls): cold
    from the uniform initial fields, warm from the steady state of a neighbouring
    operating point (inlet velocity 0.018 instead of 0.02) passed through
    fdlbm_set_fields."""
    p = workloads.config0()
    near = workloads.config0(u_inlet=0.018)
    s_near, _ = run_to_steady(fdlbm, near, device=device)
    try:
        warm_init = s_near.restart_fields()
    finally:
        s_near.close()
    s, cold = run_to_steady(fdlbm, p, device=device)
    s.close()
    s, warm = run_to_steady(fdlbm, p, init=warm_init, device=device)
    s.close()
    # 16-bit population storage (FP32 arithmetic): its stochastic rounding holds the
    # residual at a floor above the tolerance (about 1e-4 FP16, 1e-3 BF16 on this
    # channel), so the run hands over to FP32 storage once the 16-bit residual stops
    # falling, and FP32 finishes to the tolerance.
    reduced = {}
    for storage in ("fp16", "bf16"):
        try:
            reduced[storage] = precision_handoff(fdlbm, p, storage, device=device)
        except Exception as e:  # reported in the line, the benchmark itself goes on
            reduced[storage] = {"error": str(e)[:200]}
    return {"workload": "catalytic channel 128x32 gas + 2x8 solid rows, 5 species", "tol": 1e-6,
            "check_every": 500, "cold": cold, "warm": warm,
            "fp16_then_fp32": reduced["fp16"], "bf16_then_fp32": reduced["bf16"],
            "warm_start": "steady state of the channel at inlet velocity 0.018 (a neighbouring operating point)"}


def precision_handoff(fdlbm, p, storage, device=0, tol=1e-6, every=500, stall_checks=8, max_steps=200_000):
    """Cold start with 16-bit storage until its residual stops falling (no new minimum
    in `stall_checks` checks), then the state (restart fields) goes to an FP32-storage
    solver that runs to tol. Steps and wall time of both phases and in total."""
    import torch
    s = fdlbm.Solver(p, device=device, storage=storage)
    try:
        s.residual()
        torch.cuda.synchronize(device)
        t0 = time.perf_counter()
        steps, best, since = 0, float("inf"), 0
        while steps < max_steps:
            s.step(every)
            steps += every
            r = s.residual()
            if r < tol:
                break
            if r < best:
                best, since = r, 0
            else:
                since += 1
                if since >= stall_checks:
                    break
        init = s.restart_fields()
    finally:
        s.close()
    t16 = time.perf_counter() - t0
    s32, rest = run_to_steady(fdlbm, p, init=init, tol=tol, device=device)
    s32.close()
    return {"storage": storage, "steps_16bit": steps, "residual_16bit": r, "seconds_16bit": t16,
            "steps_fp32": rest["steps"], "seconds_fp32": rest["seconds"], "steps": steps + rest["steps"],
            "seconds": t16 + rest["seconds"], "residual": rest["residual"], "converged": rest["converged"]}


def learned_warm_start(device=0, n_train=12, n_test=3, tol=1e-5, max_steps=100_000, iters=600):
    """The learned warm start end to end on the GPU: steady fields of n_train seeded
    64x32x32 sphere packings from cold solver runs, the U-Net trained on them with the
    library's kernels, then on n_test unseen packings the steps and wall time to the
    residual tol from a cold start and from the network's prediction (with the cold
    fallback). tol is 1e-5 here: these packings need about 200k steps to reach 1e-6 (one
    run shows a slow transient that delays it further), more than a benchmark run holds."""
    from paper_1804_07588_gb300 import warmstart as WS
    t0 = time.perf_counter()
    train_p = WS.instances(n_train, 5000)
    test_p = WS.instances(n_test, 9000)
    data = WS.generate(train_p, tol=tol, max_steps=max_steps, device=device)
    t_gen = time.perf_counter() - t0
    model = WS.new_model(1)
    t0 = time.perf_counter()
    losses = WS.train(model, data, iters=iters)
    t_train = time.perf_counter() - t0
    study = [WS.warm_vs_cold(model, q, tol=tol, max_steps=max_steps, device=device) for q in test_p]
    cold_steps = sum(r["cold"]["steps"] for r in study)
    warm_steps = sum(r["warm"]["steps"] for r in study)
    return {"workload": f"D3Q19 {WS.SHAPE[0]}x{WS.SHAPE[1]}x{WS.SHAPE[2]} sphere packings, porosity 0.45-0.6, "
                        "inlet 0.005-0.03, 450-600 K", "tol": tol, "train_instances": n_train,
            "train_converged": sum(d["stats"]["converged"] for d in data), "data_seconds": t_gen,
            "train_iterations": iters, "train_seconds": t_train, "loss_first": losses[0], "loss_last": losses[-1],
            "network": f"4-level 3D U-Net {list(WS.CHANNELS)} channels, bf16, tcgen05 kernels",
            "test": [{"cold_steps": r["cold"]["steps"], "cold_seconds": r["cold"]["seconds"],
                      "cold_converged": r["cold"]["converged"], "warm_steps": r["warm"]["steps"],
                      "warm_seconds": r["warm"]["seconds"], "warm_converged": r["warm"]["converged"],
                      "fallback": r["warm"]["fallback"]} for r in study],
            "steps_ratio_warm_over_cold": warm_steps / max(cold_steps, 1),
            "seconds_ratio_warm_over_cold": sum(r["warm"]["seconds"] for r in study) /
            max(sum(r["cold"]["seconds"] for r in study), 1e-9)}


def measure(fdlbm, p, storage, steps, warmup, dev, flush, Q):
    """Species-MLUPS of one workload (L2 flushed before each timed step) and the roofline
    of its step launches: algorithmic bytes (2 Q populations per species-node) over the
    CUDA-event time of the step's kernels."""
    import torch
    s = fdlbm.Solver(p, device=dev, storage=storage, band_rows="auto" if p["dim"] == 2 else 0)
    info = s.info()
    ns, n_gas = info["ns"], info["n_gas"]
    s.step(warmup)
    s.sync()
    s.profile(True)
    st = s.stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for a, b in ev:
        with torch.cuda.stream(st):
            flush.zero_()
        a.record(st)
        s.step(1)
        b.record(st)
    torch.cuda.synchronize(dev)
    ms = sum(a.elapsed_time(b) for a, b in ev)
    kms, timed = s.kernel_times()
    s.close()
    peak, peak_kind = measured_peaks()
    alg = 2 * Q * BYTES_PER_VALUE[storage] * ns * n_gas
    k = kms / max(timed, 1)
    return {"value": ns * n_gas * steps / (ms * 1e-3) / 1e6, "unit": UNIT, "ms_per_step": ms / steps,
            "steps": steps, "gas_nodes": n_gas,
            "roofline": {"bound": "hbm", "achieved": alg / (k * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                         "frac": alg / (k * 1e-3) / 1e9 / peak, "peak_kind": peak_kind + " copy bandwidth",
                         "alg_bytes_per_launch": alg, "kernel_ms_per_step": k, "traffic": None}}


def _oracle_worker(args):
    """One host core: the oracle on its own crop of the bed for a fixed time."""
    offset, seconds, three_d = args
    sys.path.insert(0, ROOT)
    import oracle
    if three_d:
        from paper_1804_07588_gb300 import workloads as W
        p = W.config2_crop()
        o = oracle.Oracle3(p)
    else:
        p, _ = crop_problem(16384, x0=offset)
        o = oracle.Oracle(p)
    n_gas = o.counts()["gas"]
    ns = len(p["species"])
    t0 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t0 < seconds or steps < 3:
        o.step(1)
        steps += 1
    return ns * n_gas * steps / (time.perf_counter() - t0) / 1e6


def oracle_all_cores(seconds=10.0, three_d=False):
    """The oracle, single-threaded as it stands, run concurrently by one process per host
    core on disjoint crops of the bed; the sum of their species-MLUPS."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(n) as pool:
        rates = pool.map(_oracle_worker, [(128 * (i % 7), seconds, three_d) for i in range(n)])
    return float(sum(rates)), n


def run_batch(args, rank, world, local_rank):
    """64 independent porous beds (256..1024 x 128..256, porosity 0.4-0.7, inlet 0.005-0.03,
    450-600 K) advanced together by one batch (one kernel launch per step from a captured
    graph) against the same solvers stepped one launch each per step. Host clock around
    K synchronised steps; the working set (GBs) is far larger than L2."""
    import numpy as np
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
    steady = None
    if args.steady_cap > 0:
        t0 = time.perf_counter()
        res = batch.run_to_steady(tol=1e-6, every=1000, max_steps=args.steady_cap)
        el = time.perf_counter() - t0
        r = np.array([x["residual"] for x in res])
        steady = {"tol": 1e-6, "cap_steps": args.steady_cap, "seconds": el,
                  "converged": int(sum(x["converged"] for x in res)), "unstable": int(sum(x["unstable"] for x in res)),
                  "members": len(res), "residual_median": float(np.median(r)), "residual_max": float(r.max()),
                  "steps_of_converged": [x["steps"] for x in res if x["converged"]],
                  "what": "after the timed steps, members run on in the batch and leave it at residual 1e-6"}
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
    if steady is not None:
        line["to_steady"] = steady
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
    single = ns * n_gas * args.steps / el / 1e6
    # the host's cores together: one single-threaded oracle process per core on its own
    # crop for as long as the single-core run took (at least 5 s)
    value, ncores = oracle_all_cores(seconds=max(5.0, min(el, 60.0)))
    ms_step = ns * n_gas / value / 1e3  # time of one crop step at the aggregate rate
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": desc,
                   "oracle": f"plain FP64 C, single-threaded, {ncores} concurrent processes on the host's cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": ncores, "kind": "oracle",
                         "sample": f"{ncores} concurrent single-threaded oracle processes, each on its own "
                                   f"crop of the bed (the first: {desc})",
                         "single_core": {"value": single, "steps": args.steps, "seconds": el}},
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
    s = fdlbm.Solver(p, device=dev, storage=args.storage, band_rows="auto" if not three_d else 0)
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
        s2 = fdlbm.Solver(p, device=dev, storage=args.storage, band_rows="auto" if not three_d else 0)
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
    learned = None
    if rank == 0 and not args.no_steady and not three_d:
        tts = time_to_steady(fdlbm, workloads, device=dev)
        try:
            learned = learned_warm_start(device=dev)
        except Exception as e:  # reported in the line, the benchmark itself goes on
            learned = {"error": str(e)[:300]}
        tts["learned_warm_start"] = learned

    # the other workloads of the hot path, each with its own roofline (same timing rules)
    variants = None
    if rank == 0 and not three_d and args.storage == "fp32" and not args.no_variants:
        variants = {}
        for name, q, storage, k, w, Qv in (
                ("bed_bf16_storage", p, "bf16", 20, 5, 9), ("bed_fp16_storage", p, "fp16", 20, 5, 9),
                ("bed3d_256x128x128_fp32", None, "fp32", 10, 3, 19),
                ("bed3d_256x128x128_bf16_storage", None, "bf16", 10, 3, 19)):
            try:
                if q is None:
                    q = workloads.config2()
                variants[name] = measure(fdlbm, q, storage, k, w, dev, flush, Qv)
                variants[name]["roofline"]["traffic"] = variant_traffic(name, Qv == 19)
            except Exception as e:
                variants[name] = {"error": str(e)[:200]}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, el = oracle_throughput(seconds=10.0, three_d=three_d)
        vall, ncores = oracle_all_cores(seconds=10.0, three_d=three_d)
        cpu = {"value": vall, "unit": UNIT, "cores": ncores, "kind": "oracle",
               "sample": f"{ncores} concurrent single-threaded oracle processes, each on its own crop of the bed "
                         f"({desc.split(',')[0]} and its shifted copies), 10 s",
               "single_core": {"value": v, "sample": desc, "seconds": round(el, 2)}}

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
                       **({} if three_d else {"block_order": {"band_rows": s.band_rows, "tile_entries": s.tile_entries,
                                                              "wall_order": s.wall_order,
                                                              "from": "autotuner table (tuning_gb300.json)"}}),
                       "parallelism": "replicas" if world > 1 else "single-gpu"},
            "roofline": {"bound": "hbm", "kernel": "step_kernel", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "traffic": ncu_traffic(three_d) if args.storage == "fp32" else None,
                         "peak_kind": peak_kind + " copy bandwidth",
                         "alg_bytes_per_launch": alg_bytes, "kernel_ms_per_launch": step_kernel_ms},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * (2 if (three_d and p["energy_correction"]) else 1),
            "variants": variants,
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
