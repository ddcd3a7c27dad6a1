"""Autotuner table lookup (host logic, no GPU)."""
import json

from paper_1804_07588_gb300 import autotune, workloads as W


def _table(tmp_path, entries):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"kernel": "step_kernel", "entries": entries}))
    return str(path)


def _entry(nx, ny, por, band, ns=5, storage="fp32", tile=None, order=None):
    e = {"nx": nx, "ny": ny, "porosity": por, "ns": ns, "storage": storage, "band_rows": band}
    if tile is not None:
        e["tile_entries"] = tile
    if order is not None:
        e["wall_order"] = order
    return e


def test_lookup_nearest_size_and_porosity(tmp_path):
    t = _table(tmp_path, [_entry(256, 128, 0.6, 8, tile=128, order=1), _entry(1024, 512, 0.6, 16, tile=256, order=0),
                          _entry(1024, 512, 0.7, 32, tile=192, order=1)])
    small = W.periodic_box(250, 130, solid_rows=50)
    assert autotune.lookup(small, table=t) == (8, 128, 1)
    big = W.periodic_box(1000, 500, solid_rows=150)           # porosity 0.7
    assert autotune.lookup(big, table=t) == (32, 192, 1)


def test_lookup_matches_storage_and_species(tmp_path):
    t = _table(tmp_path, [_entry(512, 256, 0.7, 8, storage="fp16", tile=128, order=0),
                          _entry(512, 256, 0.7, 32, tile=256, order=1)])
    p = W.periodic_box(512, 256, solid_rows=76)
    assert autotune.lookup(p, "fp16", table=t) == (8, 128, 0)
    assert autotune.lookup(p, "fp32", table=t) == (32, 256, 1)
    assert autotune.lookup(p, "bf16", table=t) == autotune.DEFAULT


def test_lookup_of_band_only_entries_keeps_default_tiles(tmp_path):
    """Entries of a table that tuned the band height alone: the other two tunables take
    their defaults."""
    t = _table(tmp_path, [_entry(512, 256, 0.7, 32)])
    p = W.periodic_box(512, 256, solid_rows=76)
    assert autotune.lookup(p, table=t) == (32, autotune.DEFAULT[1], autotune.DEFAULT[2])


def test_lookup_without_table_is_default(tmp_path):
    p = W.periodic_box(64, 32)
    assert autotune.lookup(p, table=str(tmp_path / "missing.json")) == autotune.DEFAULT


def test_sweep_covers_every_combination(monkeypatch):
    """tune() times every (band_rows, tile_entries, wall_order) combination and keeps the
    fastest (measure replaced by a fake timing)."""
    calls = []

    def fake(p, storage, b, t, o, steps=100, device=0):
        calls.append((b, t, o))
        return 100.0 + abs(b - 16) + abs(t - 192) / 32 + 3 * o

    monkeypatch.setattr(autotune, "measure", fake)
    e = autotune.tune(W.periodic_box(64, 32), "fp32")
    assert len(calls) == len(autotune.BANDS) * len(autotune.TILE_ENTRIES) * len(autotune.WALL_ORDERS)
    assert (e["band_rows"], e["tile_entries"], e["wall_order"]) == (16, 192, 0)
    assert e["us_default"] == fake(None, None, 16, 256, 0)


def test_committed_table_gives_swept_orders_for_the_bench_bed():
    """The table shipped with the package answers for the 1024x512 bench bed in every
    storage type, with values from the sweep sets (not the default fallback's path)."""
    import os
    assert os.path.exists(autotune.TABLE)
    p = W.config1()
    for storage in ("fp32", "bf16", "fp16"):
        b, t, o = autotune.lookup(p, storage)
        assert b in autotune.BANDS and t in autotune.TILE_ENTRIES and o in autotune.WALL_ORDERS
