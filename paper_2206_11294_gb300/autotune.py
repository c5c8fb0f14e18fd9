"""Table of autotuned kernel choices, keyed by device and hierarchy shape.

The search is native (mg_autotune in the library): it captures each
candidate -- per level the sweep kernel and fused tile shape, then the extent
and cluster size of the V-cycle tail -- as a CUDA graph and times it on the
device.  Every candidate computes the same result bit for bit, so a table
entry changes speed only.

This module keys the outcome by what determines it (device name, dimension,
grid size, precision, cycle shape, coarsest size), keeps it as JSON, and
applies a stored entry to a new hierarchy of the same key instead of measuring
again.  Spacing, coefficients and boundary values do not enter the key: the
kernels' work does not depend on them.
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Optional


def table_key(device_name: str, grid, precision: str, nu1: int = 2, nu2: int = 2, coarse_min: int = 4,
              inner_cycles: int = 1, cycle: str = "V") -> str:
    """Key of a hierarchy.  `grid` is an inputs.Grid, a dict with its keys, or a binding.MgGrid."""
    if hasattr(grid, "_fields_"):          # ctypes MgGrid
        dim, n = int(grid.dim), tuple(int(v) for v in grid.n)
    elif isinstance(grid, dict):
        dim, n = int(grid["dim"]), tuple(int(v) for v in grid["n"])
    else:
        dim, n = int(grid.dim), tuple(int(v) for v in grid.n)
    shape = "x".join(str(v) for v in n[:dim])
    inner = f"/i{inner_cycles}" if precision == "mixed" else ""
    return f"{device_name}|{dim}d|{shape}|{precision}{inner}|{cycle}({nu1},{nu2})|cmin{coarse_min}"


class TuningTable:
    """JSON-backed map key -> {"tuning": mg_tuning as a dict, "vcycle_ms": float}.

    path None keeps the table in memory only.  Thread-safe; save() writes
    atomically (temporary file, then rename)."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, dict] = {}
        self._lock = threading.Lock()
        self.measured = 0
        self.reused = 0
        if path and os.path.exists(path):
            with open(path) as f:
                data = json.load(f)
            if not isinstance(data, dict) or data.get("format") != 1:
                raise ValueError(f"{path}: not a tuning table (format 1)")
            self.entries = dict(data["entries"])

    def lookup(self, key: str) -> Optional[dict]:
        with self._lock:
            e = self.entries.get(key)
            return None if e is None else dict(e)

    def store(self, key: str, tuning: dict, vcycle_ms: float):
        with self._lock:
            self.entries[key] = {"tuning": tuning, "vcycle_ms": float(vcycle_ms)}

    def save(self):
        if not self.path:
            return
        with self._lock:
            data = {"format": 1, "entries": self.entries}
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)

    def key_of(self, solver) -> str:
        import torch
        o = solver.options
        prec = "mixed" if int(o.precision) == 1 else "fp64"
        return table_key(torch.cuda.get_device_name(solver.device), solver.grid, prec, int(o.nu1), int(o.nu2),
                         int(o.coarse_min), int(o.inner_cycles), "VWF"[int(o.cycle)])

    def tune(self, solver, reps: int = 10) -> dict:
        """Applies the stored choices for this solver's key, or measures them
        (the solver must have coefficients) and stores the result."""
        key = self.key_of(solver)
        e = self.lookup(key)
        if e is not None and e["tuning"].get("levels") == len(solver.levels()):
            solver.set_tuning(e["tuning"])
            self.reused += 1
            return e["tuning"]
        tuning, ms = solver.autotune(reps)
        self.store(key, tuning, ms)
        self.measured += 1
        return tuning


def describe(tuning: dict) -> str:
    """Short text form: per level C (colour), C2 (colour, two rows per thread), F<tile> (fused),
    A<tile> (TMA-fed fused) or P<tile> (fused pairs of sweeps), then the tail; "plain stream order"
    where the kernels do not launch as programmatic dependents."""
    code = {"colour": lambda t: "C", "colour2": lambda t: "C2", "async": lambda t: f"A{t}", "fused": lambda t: f"F{t}",
            "fused2": lambda t: f"P{t}"}
    lv = ",".join(code[s](t) for s, t in zip(tuning["sweep"], tuning["tile"]))
    tail = "none" if tuning["tail_level"] >= tuning["levels"] else \
        f"from L{tuning['tail_level']} on {tuning['tail_ctas']} CTAs"
    waves = ", persistent waves" if tuning.get("persistent") else ""
    order = ", plain stream order" if tuning.get("overlap", 1) == 0 else ""
    return f"sweeps [{lv}], tail {tail}{waves}{order}"
