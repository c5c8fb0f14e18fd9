"""FP64 CPU oracle for the coupled pressure-temperature solve (test infrastructure).

This package is test infrastructure: only the tests, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA library never
calls it and shares no code with it.  The arithmetic lives in
``coupled_oracle.c`` (plain C, ``-O2 -ffp-contract=off``, one thread); this file
only compiles it with gcc and marshals numpy arrays through ctypes.

Functions (each follows Sec. 3 of the paper, Eqs. 27-34 and the
defect-correction loop after them; see the C file for the exact statements):

- ``apply_paper``     y = L(x), the paper's two-row operator (Eqs. 27-28)
- ``dense_solve``     exact solution of L(x) = b by Gaussian elimination
- ``mg_solve``        defect-correction loop with V(nu1, nu2) cycles
- ``rbgs_sweeps``     in-place red-black block Gauss-Seidel sweeps
- ``wjac_sweeps``     weighted block Jacobi sweeps
- ``residual_norms``  the per-field stopping norm ||D^-1 r||_2
- ``level_coeffs``    coarse-level blocks and faces of the hierarchy
- ``apply_rows``      L(x) at selected cells (residual checks of large solutions)
- ``restrict``        a fine residual restricted to the coarse right-hand side
- ``prolong_add``     a coarse correction interpolated and added to fine unknowns
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "coupled_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libcoupled_oracle.so")
_LIB_OMP = os.path.join(_BUILD, "libcoupled_oracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

BC_WALL, BC_DIRICHLET, BC_AXIS = 0, 1, 2


class OrcGrid(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("axisym", C.c_int),
        ("n", C.c_int * 3),
        ("h", C.c_double),
        ("r0", C.c_double),
        ("bc", (C.c_int * 2) * 3),
        ("bcT", (C.c_double * 2) * 3),
        ("bcp", (C.c_double * 2) * 3),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C99, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def build_threaded(force: bool = False) -> str:
    """The same source with -fopenmp, for timing the oracle on every host core
    (comparisons use the single-thread build)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_OMP) or os.path.getmtime(_LIB_OMP) < os.path.getmtime(_SRC):
        tmp = _LIB_OMP + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_OMP)
    return _LIB_OMP


def configure(lib):
    """Declares the argument types of an oracle library (also used by the tests
    that load a deliberately mutated copy)."""
    dp = C.POINTER(C.c_double)
    gp = C.POINTER(OrcGrid)
    pa3 = dp * 3
    lib.orc_apply_paper.argtypes = [gp, dp, pa3, pa3, dp, dp, C.c_int]
    lib.orc_apply_paper.restype = None
    lib.orc_dense_solve.argtypes = [gp, dp, pa3, pa3, dp, dp]
    lib.orc_dense_solve.restype = C.c_int
    lib.orc_mg_solve.argtypes = [gp, dp, pa3, pa3, dp, dp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, dp, C.c_int,
                                 C.c_int, C.c_double]
    lib.orc_mg_solve.restype = C.c_int
    lib.orc_rbgs_sweeps.argtypes = [gp, dp, pa3, pa3, dp, dp, C.c_int]
    lib.orc_rbgs_sweeps.restype = C.c_int
    lib.orc_wjac_sweeps.argtypes = [gp, dp, pa3, pa3, dp, dp, C.c_int, C.c_double]
    lib.orc_wjac_sweeps.restype = C.c_int
    lib.orc_residual_norms.argtypes = [gp, dp, pa3, pa3, dp, dp, dp]
    lib.orc_residual_norms.restype = C.c_int
    lib.orc_num_levels.argtypes = [gp, C.c_int]
    lib.orc_num_levels.restype = C.c_int
    lib.orc_level_coeffs.argtypes = [gp, dp, pa3, pa3, C.c_int, C.c_int, dp, pa3, pa3]
    lib.orc_level_coeffs.restype = C.c_int
    lib.orc_apply_rows.argtypes = [gp, dp, pa3, pa3, dp, C.POINTER(C.c_long), C.c_long, dp]
    lib.orc_apply_rows.restype = None
    lib.orc_restrict.argtypes = [gp, dp, dp]
    lib.orc_restrict.restype = C.c_int
    lib.orc_prolong_add.argtypes = [gp, dp, dp]
    lib.orc_prolong_add.restype = C.c_int
    lib.orc_threads.argtypes = []
    lib.orc_threads.restype = C.c_int
    return lib


def compile_source(src: str, out: str) -> str:
    """Compiles an oracle source file with the oracle's flags."""
    subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                           "-o", out, src, "-lm"])
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = configure(C.CDLL(build()))
    return _lib


def _grid(g) -> OrcGrid:
    """g: a mapping/object with dim, axisym, n, h, r0, bc, bcT, bcp."""
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    s = OrcGrid()
    s.dim = int(get("dim"))
    s.axisym = int(get("axisym"))
    n = list(get("n")) + [1] * (3 - len(get("n")))
    for a in range(3):
        s.n[a] = int(n[a])
    s.h = float(get("h"))
    s.r0 = float(get("r0"))
    bc, bcT, bcp = get("bc"), get("bcT"), get("bcp")
    for a in range(3):
        for side in range(2):
            s.bc[a][side] = int(bc[a][side])
            s.bcT[a][side] = float(bcT[a][side])
            s.bcp[a][side] = float(bcp[a][side])
    return s


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _c64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _faces(fs):
    keep = [_c64(f) for f in fs] + [np.zeros(1)] * (3 - len(fs))
    arr = (C.POINTER(C.c_double) * 3)(*[_dp(f) for f in keep])
    return arr, keep


def _ncells(g) -> int:
    s = _grid(g)
    return s.n[0] * s.n[1] * s.n[2]


def apply_paper(g, lam, fa, fk, x, homogeneous: bool = False) -> np.ndarray:
    lib = _load()
    gs = _grid(g)
    lam, x = _c64(lam), _c64(x)
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    y = np.empty_like(x)
    lib.orc_apply_paper(C.byref(gs), _dp(lam), pa, pk, _dp(x), _dp(y), int(homogeneous))
    return y


def dense_solve(g, lam, fa, fk, b) -> np.ndarray:
    lib = _load()
    gs = _grid(g)
    lam, b = _c64(lam), _c64(b)
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    x = np.empty_like(b)
    rc = lib.orc_dense_solve(C.byref(gs), _dp(lam), pa, pk, _dp(b), _dp(x))
    if rc != 0:
        raise RuntimeError(f"oracle dense solve failed ({rc})")
    return x


CYCLES = {"V": 0, "W": 1, "F": 2}
SMOOTHERS = {"rbgs": 0, "wjac": 1}


def _load_threaded():
    global _lib_omp
    with _lock:
        if _lib_omp is None:
            _lib_omp = configure(C.CDLL(build_threaded()))
    return _lib_omp


def threads(threaded: bool = False) -> int:
    """Threads the oracle's loops run on (the threaded build: OMP_NUM_THREADS or every core)."""
    return int((_load_threaded() if threaded else _load()).orc_threads())


def mg_solve(g, lam, fa, fk, b, x0, nu1=2, nu2=2, coarse_min=4, max_cycles=50, rtol=1e-10, cycle="V",
             smoother="rbgs", omega=0.8, threaded=False):
    """Returns (x, cycles, history) where history[k] = per-field norms before cycle k.  cycle: V, W or F;
    smoother: rbgs (red-black block Gauss-Seidel) or wjac (weighted block Jacobi with weight omega).
    threaded: run the OpenMP build (timing only; its norms are summed in another order)."""
    lib = _load_threaded() if threaded else _load()
    gs = _grid(g)
    lam, b = _c64(lam), _c64(b)
    x = _c64(x0).copy()
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    hist = np.zeros(2 * (max_cycles + 1))
    rc = lib.orc_mg_solve(C.byref(gs), _dp(lam), pa, pk, _dp(b), _dp(x), int(nu1), int(nu2),
                          int(coarse_min), int(max_cycles), float(rtol), _dp(hist), CYCLES[cycle],
                          SMOOTHERS[smoother], float(omega))
    if rc < 0:
        raise RuntimeError(f"oracle mg solve failed ({rc})")
    return x, rc, hist.reshape(-1, 2)[: rc + 1]


def rbgs_sweeps(g, lam, fa, fk, b, x0, sweeps=1) -> np.ndarray:
    lib = _load()
    gs = _grid(g)
    lam, b = _c64(lam), _c64(b)
    x = _c64(x0).copy()
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    if lib.orc_rbgs_sweeps(C.byref(gs), _dp(lam), pa, pk, _dp(b), _dp(x), int(sweeps)):
        raise RuntimeError("oracle sweeps failed")
    return x


def wjac_sweeps(g, lam, fa, fk, b, x0, sweeps=1, omega=0.8) -> np.ndarray:
    lib = _load()
    gs = _grid(g)
    lam, b = _c64(lam), _c64(b)
    x = _c64(x0).copy()
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    if lib.orc_wjac_sweeps(C.byref(gs), _dp(lam), pa, pk, _dp(b), _dp(x), int(sweeps), float(omega)):
        raise RuntimeError("oracle sweeps failed")
    return x


def residual_norms(g, lam, fa, fk, b, x) -> np.ndarray:
    lib = _load()
    gs = _grid(g)
    lam, b, x = _c64(lam), _c64(b), _c64(x)
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    out = np.zeros(2)
    if lib.orc_residual_norms(C.byref(gs), _dp(lam), pa, pk, _dp(b), _dp(x), _dp(out)):
        raise RuntimeError("oracle norms failed")
    return out


def num_levels(g, coarse_min=4) -> int:
    gs = _grid(g)
    return int(_load().orc_num_levels(C.byref(gs), int(coarse_min)))


def level_coeffs(g, lam, fa, fk, level, coarse_min=4):
    """(lambda (N_l x 4), fa_l, fk_l) of hierarchy level ``level`` (physical form)."""
    lib = _load()
    gs = _grid(g)
    dim = gs.dim
    n = [gs.n[0], gs.n[1], gs.n[2]]
    for _ in range(level):
        for a in range(dim):
            n[a] //= 2
    N = n[0] * n[1] * n[2]
    B = np.zeros(4 * N)
    fa_o, fk_o = [], []
    for a in range(3):
        m = 1
        if a < dim:
            for q in range(3):
                m *= n[q] + 1 if q == a else n[q]
        fa_o.append(np.zeros(m))
        fk_o.append(np.zeros(m))
    lam = _c64(lam)
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    poa = (C.POINTER(C.c_double) * 3)(*[_dp(f) for f in fa_o])
    pok = (C.POINTER(C.c_double) * 3)(*[_dp(f) for f in fk_o])
    rc = lib.orc_level_coeffs(C.byref(gs), _dp(lam), pa, pk, int(coarse_min), int(level),
                              _dp(B), poa, pok)
    if rc:
        raise RuntimeError(f"oracle level_coeffs failed ({rc})")
    return B.reshape(N, 4), fa_o[:dim], fk_o[:dim]


def apply_rows(g, lam, fa, fk, x, ids) -> np.ndarray:
    """L(x) (Eqs. 27-28, with the Dirichlet values) at cells ``ids``: [len(ids), 2]."""
    lib = _load()
    gs = _grid(g)
    lam, x = _c64(lam), _c64(x)
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    pa, ka = _faces(fa)
    pk, kk = _faces(fk)
    out = np.empty((ids.size, 2))
    lib.orc_apply_rows(C.byref(gs), _dp(lam), pa, pk, _dp(x), ids.ctypes.data_as(C.POINTER(C.c_long)),
                       int(ids.size), _dp(out))
    return out


def _coarse_cells(g) -> int:
    gs = _grid(g)
    n = [gs.n[0], gs.n[1], gs.n[2]]
    for a in range(gs.dim):
        if n[a] % 2:
            raise ValueError("every n_a must be even to coarsen")
        n[a] //= 2
    return n[0] * n[1] * n[2]


def restrict(g, r) -> np.ndarray:
    """The coarse right-hand side [N_c, 2] that a V-cycle forms from the fine residual r [N, 2] on grid g."""
    lib = _load()
    gs = _grid(g)
    r = _c64(r)
    out = np.empty((_coarse_cells(g), 2))
    if lib.orc_restrict(C.byref(gs), _dp(r), _dp(out)):
        raise RuntimeError("oracle restriction failed")
    return out


def prolong_add(g, uc, uf) -> np.ndarray:
    """uf + P uc: the coarse correction uc [N_c, 2] interpolated onto grid g and added to uf [N, 2]."""
    lib = _load()
    gs = _grid(g)
    uc = _c64(uc)
    if uc.shape[0] != _coarse_cells(g):
        raise ValueError("uc has the wrong number of cells")
    out = _c64(uf).copy()
    if lib.orc_prolong_add(C.byref(gs), _dp(uc), _dp(out)):
        raise RuntimeError("oracle prolongation failed")
    return out
