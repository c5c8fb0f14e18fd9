"""FP64 CPU oracle for the coupled solve on a refined-patch (adaptive) grid (test infrastructure).

Only the tests and the benchmark's CPU-baseline leg may import it.  The
arithmetic lives in ``composite_oracle.c`` (plain C, ``-O2 -ffp-contract=off``,
one thread, reusing ``coupled_oracle.c``); this file compiles it and marshals
numpy arrays.  A composite grid is a base grid (a mapping as for the uniform
oracle, 2D Cartesian) plus ``box`` = ((i0, i1), (j0, j1)), the base cells
refined 2:1 into the patch.

- ``patch_grid``   the patch as a uniform grid (cells, spacing, the domain's boundary kinds on its outer sides)
- ``apply``        y = L(x) of Eqs. 27-28 on the composite grid
- ``dense_solve``  exact solution by Gaussian elimination (small grids)
- ``fac_solve``    defect correction with FAC cycles, a fixed number of steps
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

from . import OrcGrid, _grid, _dp, _c64, _faces

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "composite_oracle.c")
_DEP = os.path.join(_HERE, "coupled_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libcomposite_oracle.so")
_lock = threading.Lock()
_lib = None


class OrcCGrid(C.Structure):
    _fields_ = [("base", OrcGrid), ("box", (C.c_int * 2) * 2)]


def build(force: bool = False) -> str:
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    stale = not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(p) for p in (_SRC, _DEP))
    if force or stale:
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-I", _HERE, "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def configure(lib):
    dp = C.POINTER(C.c_double)
    cp = C.POINTER(OrcCGrid)
    pa3 = dp * 3
    lib.orc_cf_apply.argtypes = [cp, dp, pa3, pa3, dp, pa3, pa3, dp, dp, dp, dp, C.c_int]
    lib.orc_cf_apply.restype = None
    lib.orc_cf_fac_solve.argtypes = [cp, dp, pa3, pa3, dp, pa3, pa3, dp, dp, dp, dp, C.c_int, C.c_int, C.c_int,
                                     C.c_int, dp]
    lib.orc_cf_fac_solve.restype = C.c_int
    lib.orc_cf_dense_solve.argtypes = [cp, dp, pa3, pa3, dp, pa3, pa3, dp, dp, dp, dp]
    lib.orc_cf_dense_solve.restype = C.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(C.CDLL(build()))
    return _lib


def _cgrid(base, box) -> OrcCGrid:
    s = OrcCGrid()
    s.base = _grid(base)
    for a in range(2):
        for q in range(2):
            s.box[a][q] = int(box[a][q])
    return s


def patch_grid(base, box) -> dict:
    """The patch as a uniform grid mapping: n = 2 x the box, h / 2, the base's
    boundary kinds and values on sides where the box reaches the domain
    boundary (interface sides are reported as walls: their flux is the
    composite one)."""
    get = (lambda k: base[k]) if isinstance(base, dict) else (lambda k: getattr(base, k))
    n = list(get("n")) + [1] * (3 - len(get("n")))
    bc = [list(s) for s in get("bc")]
    bcT = [list(s) for s in get("bcT")]
    bcp = [list(s) for s in get("bcp")]
    m = [2 * (box[a][1] - box[a][0]) for a in range(2)] + [1]
    for a in range(2):
        for s, touches in ((0, box[a][0] == 0), (1, box[a][1] == n[a])):
            if not touches:
                bc[a][s], bcT[a][s], bcp[a][s] = 0, 0.0, 0.0
    return dict(dim=2, axisym=0, n=m, h=float(get("h")) / 2, r0=0.0, bc=bc, bcT=bcT, bcp=bcp)


def _args(base, box, lamb, fab, fkb, lamf, faf, fkf):
    cg = _cgrid(base, box)
    keep = []
    lamb, lamf = _c64(lamb), _c64(lamf)
    pab, k1 = _faces(fab)
    pkb, k2 = _faces(fkb)
    paf, k3 = _faces(faf)
    pkf, k4 = _faces(fkf)
    keep += [lamb, lamf, k1, k2, k3, k4]
    return cg, (C.byref(cg), _dp(lamb), pab, pkb, _dp(lamf), paf, pkf), keep


def apply(base, box, lamb, fab, fkb, lamf, faf, fkf, xb, xf, homogeneous=False):
    """(yb, yf): L(x) on the valid base cells (covered cells 0) and on the patch."""
    cg, a, keep = _args(base, box, lamb, fab, fkb, lamf, faf, fkf)
    xb, xf = _c64(xb), _c64(xf)
    yb, yf = np.empty_like(xb), np.empty_like(xf)
    _load().orc_cf_apply(*a, _dp(xb), _dp(xf), _dp(yb), _dp(yf), int(homogeneous))
    return yb, yf


def dense_solve(base, box, lamb, fab, fkb, lamf, faf, fkf, bb, bf):
    cg, a, keep = _args(base, box, lamb, fab, fkb, lamf, faf, fkf)
    bb, bf = _c64(bb), _c64(bf)
    xb, xf = np.zeros_like(bb), np.zeros_like(bf)
    rc = _load().orc_cf_dense_solve(*a, _dp(bb), _dp(bf), _dp(xb), _dp(xf))
    if rc:
        raise RuntimeError(f"composite dense solve failed ({rc})")
    return xb, xf


def fac_solve(base, box, lamb, fab, fkb, lamf, faf, fkf, bb, bf, xb0, xf0, cycles, nu1=2, nu2=2, coarse_min=4):
    """(xb, xf, hist): `cycles` defect-correction steps with one FAC cycle each;
    hist[k] = L2 norms of the (T, p) residuals over the valid base cells, then
    over the patch, before step k and after the last."""
    cg, a, keep = _args(base, box, lamb, fab, fkb, lamf, faf, fkf)
    bb, bf = _c64(bb), _c64(bf)
    xb, xf = _c64(xb0).copy(), _c64(xf0).copy()
    hist = np.zeros(4 * (cycles + 1))
    rc = _load().orc_cf_fac_solve(*a, _dp(bb), _dp(bf), _dp(xb), _dp(xf), int(nu1), int(nu2), int(coarse_min),
                                  int(cycles), _dp(hist))
    if rc:
        raise RuntimeError(f"composite FAC solve failed ({rc})")
    return xb, xf, hist.reshape(-1, 4)
