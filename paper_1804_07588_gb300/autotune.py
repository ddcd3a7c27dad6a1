"""Autotuner for the D2Q9 step kernel's block order.

The one launch of a time step runs gas tiles (a band of rows x a column range, with the
one-node halo ring the energy correction needs) and wall and solid blocks. Three
tunables shape it: the band height (`band_rows`, also the tiles' height), the gas nodes
per tile (`tile_entries`, also the block size: smaller tiles mean more blocks per SM and
more halo work) and the block order (`wall_order`: each band's wall blocks right after its
gas tiles, or all wall blocks last). `sweep` times every combination of the candidate
values on representative porous beds on the current GPU and writes a JSON table keyed by
lattice size, porosity, species count and storage; `lookup` returns the best combination
of the nearest table entry for a problem (the defaults when there is no table). Solvers
created with band_rows="auto" use it.

Run the sweep on the target GPU:  python -m paper_1804_07588_gb300.autotune --out FILE
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning_gb300.json")
BANDS = (8, 16, 32)
TILE_ENTRIES = (128, 192, 256)
WALL_ORDERS = (0, 1)
DEFAULT = (16, 256, 0)  # band_rows, tile_entries, wall_order


def _porosity(p: dict) -> float:
    return float((np.asarray(p["mask"]) == 0).mean())


def _key(p: dict, storage: str) -> dict:
    return {"nx": int(p["nx"]), "ny": int(p["ny"]), "porosity": round(_porosity(p), 3),
            "ns": len(p["species"]), "storage": storage}


def measure(p: dict, storage: str, band_rows: int, tile_entries: int = 0, wall_order: int = 0, steps: int = 100,
            repeats: int = 3, device: int = 0) -> float:
    """Microseconds per step of the step kernel (CUDA events on the solver's stream; the
    best of `repeats` runs of `steps` steps after 10 warm-up steps)."""
    from . import fdlbm
    s = fdlbm.Solver(p, device=device, storage=storage, band_rows=band_rows, tile_entries=tile_entries,
                     wall_order=wall_order)
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


def tune(p: dict, storage: str = "fp32", bands=BANDS, tiles=TILE_ENTRIES, orders=WALL_ORDERS, steps: int = 100,
         device: int = 0) -> dict:
    """Step time of every (band_rows, tile_entries, wall_order) combination; the entry
    holds the fastest and all timings."""
    times = {}
    for b in bands:
        for t in tiles:
            for o in orders:
                times[f"{b},{t},{o}"] = measure(p, storage, b, t, o, steps=steps, device=device)
    best = min(times, key=times.get)
    b, t, o = (int(v) for v in best.split(","))
    entry = _key(p, storage)
    entry.update({"band_rows": b, "tile_entries": t, "wall_order": o, "us_per_step": times,
                  "us_default": times.get(f"{DEFAULT[0]},{DEFAULT[1]},{DEFAULT[2]}")})
    return entry


def _boolean_bed(nx: int, ny: int, por: float, seed: int) -> dict:
    from . import workloads as W
    while True:
        try:
            mask, _ = W.disk_mask_boolean(nx, ny, por, 6.0, 12.0, seed)
            break
        except ValueError:
            seed += 1
    return W._base(2, nx, ny, 1, mask, [W.INLET, W.OUTLET, W.PERIODIC, W.PERIODIC], u_inlet=0.01,
                   inlet_profile=W.PLUG)


def representative_problems():
    """Porous beds spanning the sizes and porosities the solver is run on."""
    from . import workloads
    out = []
    for (nx, ny) in ((256, 128), (512, 192), (512, 256), (1024, 256), (1024, 512)):
        for por in (0.45, 0.7):
            out.append(workloads.porous_disks(nx=nx, ny=ny, porosity=por, seed=5000 + nx + ny) if por >= 0.6 else
                       _boolean_bed(nx, ny, por, 5000 + nx + ny))
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


def lookup(p: dict, storage: str = "fp32", table: str | None = None) -> tuple:
    """(band_rows, tile_entries, wall_order) of the nearest entry (log lattice size,
    porosity) with the same species count and storage; DEFAULT without a matching table
    entry."""
    path = table or TABLE
    try:
        with open(path) as f:
            entries = json.load(f)["entries"]
    except (OSError, ValueError, KeyError):
        return DEFAULT
    k = _key(p, storage)
    cands = [e for e in entries if e["ns"] == k["ns"] and e["storage"] == storage] or \
            [e for e in entries if e["storage"] == storage]
    if not cands:
        return DEFAULT

    def dist(e):
        return (abs(math.log(e["nx"] * e["ny"]) - math.log(k["nx"] * k["ny"])) +
                4.0 * abs(e["porosity"] - k["porosity"]))
    e = min(cands, key=dist)
    return int(e["band_rows"]), int(e.get("tile_entries", DEFAULT[1])), int(e.get("wall_order", DEFAULT[2]))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=TABLE)
    ap.add_argument("--storage", nargs="+", default=["fp32"])
    ap.add_argument("--steps", type=int, default=100)
    args = ap.parse_args()
    sweep(args.out, storages=args.storage, steps=args.steps)


if __name__ == "__main__":
    main()
