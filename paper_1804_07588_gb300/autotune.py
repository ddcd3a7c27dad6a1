"""Autotuner for the step kernel's block order.

The one launch of a time step runs, per band of rows, the gas blocks of the band and then
its wall blocks (so that the wall blocks find their neighbours' populations in L2); the
band height (`band_rows`) is the tunable. `sweep` times candidate heights on
representative porous beds on the current GPU and writes a JSON table keyed by lattice
size, porosity, species count and storage; `lookup` returns the height of the nearest
table entry for a problem (8 when there is no table). Solvers created with
band_rows="auto" use it.

Run the sweep on the target GPU:  python -m paper_1804_07588_gb300.autotune --out FILE
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
CANDIDATES = (4, 8, 16, 32, 64)
DEFAULT_BAND = 8


def _porosity(p: dict) -> float:
    return float((np.asarray(p["mask"]) == 0).mean())


def _key(p: dict, storage: str) -> dict:
    return {"nx": int(p["nx"]), "ny": int(p["ny"]), "porosity": round(_porosity(p), 3),
            "ns": len(p["species"]), "storage": storage}


def measure(p: dict, storage: str, band_rows: int, steps: int = 100, repeats: int = 3, device: int = 0) -> float:
    """Microseconds per step of the step kernel (CUDA events on the solver's stream; the
    best of `repeats` runs of `steps` steps after 10 warm-up steps)."""
    from . import fdlbm
    s = fdlbm.Solver(p, device=device, storage=storage, band_rows=band_rows)
    s.step(10)
    s.sync()
    best = math.inf
    for _ in range(repeats):
        s.profile(True)
        s.step(steps)
        s.sync()
        ms, n = s.kernel_times()
        best = min(best, ms / max(n, 1) * 1e3)
    s.profile(False)
    s.close()
    return best


def tune(p: dict, storage: str = "fp32", candidates=CANDIDATES, steps: int = 100, device: int = 0) -> dict:
    times = {int(b): measure(p, storage, b, steps=steps, device=device) for b in candidates}
    best = min(times, key=times.get)
    entry = _key(p, storage)
    entry.update({"band_rows": best, "us_per_step": times})
    return entry


def representative_problems():
    """Porous beds spanning the sizes and porosities the solver is run on."""
    from . import workloads
    out = []
    for (nx, ny) in ((256, 128), (512, 192), (512, 256), (1024, 256), (1024, 512)):
        for por in (0.6, 0.7):
            out.append(workloads.porous_disks(nx=nx, ny=ny, porosity=por, seed=5000 + nx + ny))
    return out


def sweep(out: str, storages=("fp32",), steps: int = 100, device: int = 0) -> list:
    entries = []
    for storage in storages:
        for p in representative_problems():
            e = tune(p, storage, steps=steps, device=device)
            print(json.dumps(e), flush=True)
            entries.append(e)
    with open(out, "w") as f:
        json.dump({"kernel": "step_kernel", "entries": entries}, f, indent=1)
    return entries


def lookup(p: dict, storage: str = "fp32", table: str | None = None) -> int:
    """band_rows of the nearest entry (log lattice size, porosity) with the same species
    count and storage; DEFAULT_BAND without a matching table entry."""
    path = table or TABLE
    try:
        with open(path) as f:
            entries = json.load(f)["entries"]
    except (OSError, ValueError, KeyError):
        return DEFAULT_BAND
    k = _key(p, storage)
    cands = [e for e in entries if e["ns"] == k["ns"] and e["storage"] == storage] or \
            [e for e in entries if e["storage"] == storage]
    if not cands:
        return DEFAULT_BAND

    def dist(e):
        return (abs(math.log(e["nx"] * e["ny"]) - math.log(k["nx"] * k["ny"])) +
                4.0 * abs(e["porosity"] - k["porosity"]))
    return int(min(cands, key=dist)["band_rows"])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--storage", nargs="+", default=["fp32"])
    ap.add_argument("--steps", type=int, default=100)
    args = ap.parse_args()
    sweep(args.out, storages=args.storage, steps=args.steps)


if __name__ == "__main__":
    main()
