"""Host-side parts of autotuning that need no GPU: table keys, persistence,
the ctypes mirror of mg_tuning, and the text summary."""
import ctypes as C
import json

import pytest

from paper_2206_11294_gb300 import inputs as I
from paper_2206_11294_gb300.autotune import TuningTable, describe, table_key
from paper_2206_11294_gb300 import binding as B


def _tuning(levels=5):
    return dict(levels=levels, sweep=["colour", "fused", "fused", "colour", "colour"][:levels],
                tile=[0, 1, 2, 0, 0][:levels], tail_level=3, tail_ctas=8, persistent=1, overlap=0)


def test_key_depends_on_shape_precision_and_cycle_not_on_spacing():
    g1 = I.Grid(dim=2, axisym=0, n=(256, 128, 1), h=1e-3)
    g2 = I.Grid(dim=2, axisym=1, n=(256, 128, 1), h=5e-5, r0=1e-3)
    g3 = I.Grid(dim=2, axisym=0, n=(128, 256, 1), h=1e-3)
    k1 = table_key("GPU", g1, "fp64")
    assert k1 == table_key("GPU", g2, "fp64")                 # spacing, axis and origin: same kernels
    assert k1 != table_key("GPU", g3, "fp64")
    assert k1 != table_key("GPU", g1, "mixed")
    assert k1 != table_key("GPU", g1, "fp64", nu1=1)
    assert k1 != table_key("GPU", g1, "fp64", coarse_min=8)
    assert k1 != table_key("Other GPU", g1, "fp64")
    assert table_key("GPU", g1.as_dict(), "fp64") == k1
    assert table_key("GPU", B.make_grid(g1), "fp64") == k1
    assert "256x128" in k1 and "2d" in k1
    g4 = I.Grid(dim=3, axisym=0, n=(64, 32, 16), h=1e-3)
    assert "64x32x16" in table_key("GPU", g4, "mixed")


def test_table_roundtrip(tmp_path):
    path = str(tmp_path / "tuning.json")
    t = TuningTable(path)
    assert t.lookup("k") is None
    t.store("k", _tuning(), 0.25)
    t.save()
    t2 = TuningTable(path)
    e = t2.lookup("k")
    assert e["tuning"] == _tuning() and e["vcycle_ms"] == 0.25
    raw = json.load(open(path))
    assert raw["format"] == 1 and "k" in raw["entries"]
    mem = TuningTable(None)
    mem.store("a", _tuning(), 1.0)
    mem.save()                                   # no path: nothing written
    assert mem.lookup("a")["vcycle_ms"] == 1.0


def test_table_rejects_foreign_file(tmp_path):
    p = tmp_path / "x.json"
    p.write_text(json.dumps({"entries": {}}))
    with pytest.raises(ValueError):
        TuningTable(str(p))


def test_ctypes_mirror_roundtrip():
    t = B.MgTuning.from_dict(_tuning())
    assert t.sweep[1] == B.MG_SWEEP_FUSED and t.sweep[0] == B.MG_SWEEP_COLOUR
    assert t.as_dict() == _tuning()
    # layout of the C struct: levels, sweep[32], tile[32], tail_level, tail_ctas, persistent, overlap (all int)
    assert C.sizeof(B.MgTuning) == 4 * (1 + 2 * B.MG_MAX_LEVELS + 4)
    assert B.MgTuning.tail_ctas.offset == 4 * (1 + 2 * B.MG_MAX_LEVELS + 1)
    assert B.MgTuning.persistent.offset == 4 * (1 + 2 * B.MG_MAX_LEVELS + 2)
    assert B.MgTuning.overlap.offset == 4 * (1 + 2 * B.MG_MAX_LEVELS + 3)
    # an entry stored before the overlap field existed reads as the library's default, 1
    d = _tuning()
    del d["overlap"]
    assert B.MgTuning.from_dict(d).overlap == 1


def test_sweep_names_roundtrip():
    d = _tuning()
    d["sweep"] = ["async", "fused", "colour", "fused2", "colour"]
    assert B.MgTuning.from_dict(d).as_dict() == d
    assert describe(d).startswith("sweeps [A0,F1,C,P0,C]")


def test_describe():
    assert describe(_tuning()) == "sweeps [C,F1,F2,C,C], tail from L3 on 8 CTAs, persistent waves, plain stream order"
    assert describe(dict(_tuning(), overlap=1)) == "sweeps [C,F1,F2,C,C], tail from L3 on 8 CTAs, persistent waves"
    d = dict(_tuning(), overlap=1)
    d["tail_level"] = 5
    d["persistent"] = 0
    assert describe(d).endswith("tail none")
