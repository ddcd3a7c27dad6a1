"""Autotuner table lookup (host logic, no GPU)."""
import json

from paper_1804_07588_gb300 import autotune, workloads as W


def _table(tmp_path, entries):
    path = tmp_path / "t.json"
    path.write_text(json.dumps({"kernel": "step_kernel", "entries": entries}))
    return str(path)


def _entry(nx, ny, por, band, ns=5, storage="fp32"):
    return {"nx": nx, "ny": ny, "porosity": por, "ns": ns, "storage": storage, "band_rows": band}


def test_lookup_nearest_size_and_porosity(tmp_path):
    t = _table(tmp_path, [_entry(256, 128, 0.6, 4), _entry(1024, 512, 0.6, 16), _entry(1024, 512, 0.7, 32)])
    small = W.periodic_box(250, 130, solid_rows=50)
    assert autotune.lookup(small, table=t) == 4
    big = W.periodic_box(1000, 500, solid_rows=150)           # porosity 0.7
    assert autotune.lookup(big, table=t) == 32


def test_lookup_matches_storage_and_species(tmp_path):
    t = _table(tmp_path, [_entry(512, 256, 0.7, 4, storage="fp16"), _entry(512, 256, 0.7, 64)])
    p = W.periodic_box(512, 256, solid_rows=76)
    assert autotune.lookup(p, "fp16", table=t) == 4
    assert autotune.lookup(p, "fp32", table=t) == 64
    assert autotune.lookup(p, "bf16", table=t) == autotune.DEFAULT_BAND


def test_lookup_without_table_is_default(tmp_path):
    p = W.periodic_box(64, 32)
    assert autotune.lookup(p, table=str(tmp_path / "missing.json")) == autotune.DEFAULT_BAND
