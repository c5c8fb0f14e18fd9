"""ctypes binding of libcoupledmg.so (include/coupledmg.h): argument marshalling only.

Every step of the solve runs in the library's CUDA kernels.  PyTorch supplies
device memory (the handle's workspace) and the CUDA stream.  If the library is
missing this module raises: there is no CPU or Python fallback.

Arrays may be numpy arrays (host; the library copies them to the device
inside the call) or CUDA torch tensors (device; used in place).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libcoupledmg.so")

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_OOM, MG_ERR_BUDGET, MG_ERR_INVALID_COEFF = 0, 1, 2, 3, 4
MG_ERR_NOT_CONVERGED, MG_ERR_TIMEOUT, MG_ERR_CUDA, MG_ERR_STATE = 5, 6, 7, 8
MG_FP64, MG_MIXED = 0, 1
STATUS_NAMES = {0: "MG_OK", 1: "MG_ERR_INVALID_ARG", 2: "MG_ERR_OOM", 3: "MG_ERR_BUDGET",
                4: "MG_ERR_INVALID_COEFF", 5: "MG_ERR_NOT_CONVERGED", 6: "MG_ERR_TIMEOUT",
                7: "MG_ERR_CUDA", 8: "MG_ERR_STATE"}

# every entry point the header declares (checked by the CPU tests)
EXPORTS = ["mg_default_options", "mg_workspace_size", "mg_create", "mg_set_coeffs", "mg_solve",
           "mg_apply", "mg_smooth", "mg_residual_norms", "mg_set_device", "mg_levels", "mg_destroy",
           "mg_last_error", "mg_set_timing", "mg_counters", "mg_residual_norms_noalloc",
           "mg_batch_create", "mg_batch_solve", "mg_batch_counters", "mg_batch_destroy", "mg_set_stream",
           "mg_batch_set_coeffs", "mg_get_tuning", "mg_set_tuning", "mg_autotune", "mg_batch_get_tuning",
           "mg_batch_set_tuning", "mg_batch_autotune", "mg_assemble_async", "mg_correct_async",
           "mg_energy_async", "mg_momentum_create", "mg_momentum_set_coeffs", "mg_momentum_apply",
           "mg_momentum_solve", "mg_momentum_destroy", "mg_momentum_rhs_async", "mg_provisional_async",
           "mg_fp64_fma_rate", "mg_copy_h2d_async", "mg_solve_async", "mg_solve_async_stats", "mg_composite_create",
           "mg_composite_set_coeffs", "mg_composite_apply", "mg_composite_solve", "mg_composite_autotune",
           "mg_composite_destroy"]

MG_MAX_LEVELS = 32
MG_SWEEP_COLOUR, MG_SWEEP_FUSED, MG_SWEEP_ASYNC, MG_SWEEP_COLOUR2, MG_SWEEP_FUSED2 = 1, 2, 3, 4, 5
_SWEEP_NAMES = {MG_SWEEP_COLOUR: "colour", MG_SWEEP_FUSED: "fused", MG_SWEEP_ASYNC: "async",
                MG_SWEEP_COLOUR2: "colour2", MG_SWEEP_FUSED2: "fused2"}
_SWEEP_CODES = {v: k for k, v in _SWEEP_NAMES.items()}
TILE_SHAPES = [(64, 16), (32, 16), (32, 8)]      # fused tile shapes by index (cells x, y)


class MgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class MgGrid(C.Structure):
    _fields_ = [("dim", C.c_int), ("axisym", C.c_int), ("n", C.c_int * 3), ("h", C.c_double),
                ("r0", C.c_double), ("bc", (C.c_int * 2) * 3), ("bc_T", (C.c_double * 2) * 3),
                ("bc_p", (C.c_double * 2) * 3)]


class MgOptions(C.Structure):
    _fields_ = [("nu1", C.c_int), ("nu2", C.c_int), ("precision", C.c_int), ("rtol", C.c_double),
                ("max_cycles", C.c_int), ("coarse_min", C.c_int), ("inner_cycles", C.c_int), ("cycle", C.c_int),
                ("smoother", C.c_int), ("omega", C.c_double), ("fp64_jump_ratio", C.c_double),
                ("coarse_solve", C.c_int)]


class MgStats(C.Structure):
    _fields_ = [("cycles", C.c_int), ("outer", C.c_int), ("r0", C.c_double * 2),
                ("rfinal", C.c_double * 2), ("seconds", C.c_double), ("status", C.c_int),
                ("levels", C.c_int), ("fp64_cells", C.c_longlong)]

    def as_dict(self) -> dict:
        return dict(cycles=self.cycles, outer=self.outer, r0=list(self.r0), rfinal=list(self.rfinal),
                    seconds=self.seconds, status=STATUS_NAMES.get(self.status, self.status),
                    levels=self.levels, fp64_cells=int(self.fp64_cells))


class MgTuning(C.Structure):
    _fields_ = [("levels", C.c_int), ("sweep", C.c_int * MG_MAX_LEVELS), ("tile", C.c_int * MG_MAX_LEVELS),
                ("tail_level", C.c_int), ("tail_ctas", C.c_int), ("persistent", C.c_int), ("overlap", C.c_int)]

    def as_dict(self) -> dict:
        n = self.levels
        return dict(levels=n, sweep=[_SWEEP_NAMES.get(int(self.sweep[l]), "colour") for l in range(n)],
                    tile=[int(self.tile[l]) for l in range(n)], tail_level=int(self.tail_level),
                    tail_ctas=int(self.tail_ctas), persistent=int(self.persistent), overlap=int(self.overlap))

    @staticmethod
    def from_dict(d: dict) -> "MgTuning":
        t = MgTuning()
        t.levels = int(d.get("levels", len(d["sweep"])))
        for l, s in enumerate(d["sweep"]):
            t.sweep[l] = _SWEEP_CODES[s] if s in _SWEEP_CODES else int(s)
        for l, s in enumerate(d["tile"]):
            t.tile[l] = int(s)
        t.tail_level = int(d["tail_level"])
        t.tail_ctas = int(d["tail_ctas"])
        t.persistent = int(d.get("persistent", 0))
        t.overlap = int(d.get("overlap", 1))      # the library's default where an entry predates the field
        return t


class MgBatchTuning(C.Structure):
    _fields_ = [("depths", C.c_int), ("sweep", C.c_int * MG_MAX_LEVELS), ("tile", C.c_int * MG_MAX_LEVELS),
                ("blocks_per_sm", C.c_int)]

    def as_dict(self) -> dict:
        n = self.depths
        return dict(depths=n, sweep=["fused" if self.sweep[d] == MG_SWEEP_FUSED else "colour" for d in range(n)],
                    tile=[int(self.tile[d]) for d in range(n)], blocks_per_sm=int(self.blocks_per_sm))

    @staticmethod
    def from_dict(d: dict) -> "MgBatchTuning":
        t = MgBatchTuning()
        t.depths = int(d.get("depths", len(d["sweep"])))
        for l, s in enumerate(d["sweep"]):
            t.sweep[l] = MG_SWEEP_FUSED if s in ("fused", MG_SWEEP_FUSED) else MG_SWEEP_COLOUR
        for l, s in enumerate(d["tile"]):
            t.tile[l] = int(s)
        t.blocks_per_sm = int(d["blocks_per_sm"])
        return t


class MgPhase(C.Structure):
    _fields_ = [("Gamma", C.c_double), ("Pi", C.c_double), ("b", C.c_double), ("q", C.c_double),
                ("cp", C.c_double), ("cv", C.c_double), ("k", C.c_double), ("mu", C.c_double)]


class MgMomentumStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("cycles", C.c_int), ("r0", C.c_double), ("rfinal", C.c_double),
                ("seconds", C.c_double), ("status", C.c_int), ("jacobi", C.c_int), ("nu", C.c_double)]

    def as_dict(self) -> dict:
        return dict(iterations=self.iterations, cycles=self.cycles, r0=self.r0, rfinal=self.rfinal,
                    seconds=self.seconds, status=STATUS_NAMES.get(self.status, self.status),
                    jacobi=bool(self.jacobi), nu=self.nu)


class MgState(C.Structure):
    _fields_ = [("C", C.c_void_p), ("m1", C.c_void_p), ("m2", C.c_void_p), ("E", C.c_void_p),
                ("mom", C.c_void_p * 3), ("uf", C.c_void_p * 3)]


class MgAssembly(C.Structure):
    _fields_ = [("lam", C.c_void_p), ("rhs", C.c_void_p), ("x0", C.c_void_p),
                ("face_alpha", C.c_void_p * 3), ("face_k", C.c_void_p * 3)]


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH):
    """Loads the library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libcoupledmg.so not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        pa3 = C.c_void_p * 3
        sig = {
            "mg_default_options": ([C.POINTER(MgOptions)], C.c_int),
            "mg_workspace_size": ([C.POINTER(MgGrid), C.POINTER(MgOptions), C.POINTER(C.c_size_t)], C.c_int),
            "mg_create": ([C.POINTER(MgGrid), C.POINTER(MgOptions), P, C.c_size_t, P, C.POINTER(P)], C.c_int),
            "mg_set_coeffs": ([P, P, pa3, pa3, C.c_int], C.c_int),
            "mg_solve": ([P, P, P, C.c_int, C.POINTER(MgStats)], C.c_int),
            "mg_apply": ([P, P, P, C.c_int], C.c_int),
            "mg_smooth": ([P, P, P, C.c_int, C.c_int], C.c_int),
            "mg_residual_norms": ([P, P, P, C.c_int, dp], C.c_int),
            "mg_set_device": ([C.c_int], C.c_int),
            "mg_levels": ([P, C.POINTER(C.c_int), C.POINTER(C.c_int)], C.c_int),
            "mg_destroy": ([P], C.c_int),
            "mg_last_error": ([], C.c_char_p),
            "mg_set_timing": ([P, C.c_int], C.c_int),
            "mg_residual_norms_noalloc": ([C.POINTER(MgGrid), P, pa3, pa3, P, P, P, P], C.c_int),
            "mg_batch_create": ([C.c_int, C.POINTER(P), C.POINTER(P)], C.c_int),
            "mg_batch_solve": ([P, C.POINTER(P), C.POINTER(P), C.c_int, C.POINTER(MgStats)], C.c_int),
            "mg_batch_counters": ([P, C.POINTER(C.c_longlong)], C.c_int),
            "mg_batch_destroy": ([P], C.c_int),
            "mg_set_stream": ([P, P], C.c_int),
            "mg_batch_set_coeffs": ([P, C.POINTER(P), C.POINTER(P), C.POINTER(P), C.c_int], C.c_int),
            "mg_counters": ([P, C.POINTER(C.c_longlong), C.POINTER(C.c_double), C.POINTER(C.c_longlong),
                             C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)], C.c_int),
            "mg_get_tuning": ([P, C.POINTER(MgTuning)], C.c_int),
            "mg_set_tuning": ([P, C.POINTER(MgTuning)], C.c_int),
            "mg_autotune": ([P, C.c_int, C.POINTER(MgTuning), dp], C.c_int),
            "mg_batch_get_tuning": ([P, C.POINTER(MgBatchTuning)], C.c_int),
            "mg_batch_set_tuning": ([P, C.POINTER(MgBatchTuning)], C.c_int),
            "mg_batch_autotune": ([P, C.c_int, C.POINTER(MgBatchTuning), dp], C.c_int),
            "mg_assemble_async": ([C.POINTER(MgGrid), MgPhase * 2, C.c_double, C.c_int, C.POINTER(MgState),
                                   C.POINTER(MgAssembly), P], C.c_int),
            "mg_correct_async": ([C.POINTER(MgGrid), C.c_double, C.c_double, P, P, P, pa3, pa3, pa3, P, P, P], C.c_int),
            "mg_energy_async": ([C.POINTER(MgGrid), C.POINTER(MgPhase), C.c_double, P, P, P, P, pa3, P, P, P, P, P],
                                C.c_int),
            "mg_momentum_create": ([C.POINTER(MgGrid), C.c_int, C.POINTER(MgOptions), P, C.POINTER(P)], C.c_int),
            "mg_momentum_set_coeffs": ([P, C.c_double, P, P], C.c_int),
            "mg_momentum_apply": ([P, pa3, pa3], C.c_int),
            "mg_momentum_solve": ([P, pa3, pa3, C.c_double, C.c_int, C.POINTER(MgMomentumStats)], C.c_int),
            "mg_momentum_destroy": ([P], C.c_int),
            "mg_momentum_rhs_async": ([C.POINTER(MgGrid), C.c_double, C.c_double, pa3, P, P, P, pa3, P], C.c_int),
            "mg_provisional_async": ([C.POINTER(MgGrid), C.c_double, P, P, pa3, pa3, P], C.c_int),
            "mg_fp64_fma_rate": ([P, C.c_int, dp], C.c_int),
            "mg_copy_h2d_async": ([P, P, C.c_size_t, P], C.c_int),
            "mg_solve_async": ([P, P, P, P], C.c_int),
            "mg_solve_async_stats": ([P, C.POINTER(MgStats)], C.c_int),
            "mg_composite_create": ([C.POINTER(MgGrid), (C.c_int * 2) * 2, C.POINTER(MgOptions), P, C.POINTER(P)],
                                    C.c_int),
            "mg_composite_set_coeffs": ([P, P, pa3, pa3, P, pa3, pa3], C.c_int),
            "mg_composite_apply": ([P, P, P, P, P], C.c_int),
            "mg_composite_solve": ([P, P, P, P, P, C.c_int, dp], C.c_int),
            "mg_composite_autotune": ([P, C.c_int, dp], C.c_int),
            "mg_composite_destroy": ([P], C.c_int),
        }
        for name, (args, res) in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = res
        _lib = lib
    return _lib


def last_error() -> str:
    return load().mg_last_error().decode()


def check(status: int, allow=(MG_OK,)) -> int:
    if status not in allow:
        raise MgError(status, last_error())
    return status


def make_grid(g) -> MgGrid:
    """From an inputs.Grid, a dict with the same keys, or an MgGrid."""
    if isinstance(g, MgGrid):
        return g
    get = (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))
    s = MgGrid()
    s.dim, s.axisym = int(get("dim")), int(get("axisym"))
    n = list(get("n")) + [1] * (3 - len(get("n")))
    for a in range(3):
        s.n[a] = int(n[a])
    s.h, s.r0 = float(get("h")), float(get("r0"))
    bc, bT, bp = get("bc"), get("bcT"), get("bcp")
    for a in range(3):
        for side in range(2):
            s.bc[a][side] = int(bc[a][side])
            s.bc_T[a][side] = float(bT[a][side])
            s.bc_p[a][side] = float(bp[a][side])
    return s


CYCLES = {"V": 0, "W": 1, "F": 2}
SMOOTHERS = {"rbgs": 0, "wjac": 1}
COARSE = {"auto": 0, "inverse": 1}


def make_options(precision="fp64", rtol=1e-10, max_cycles=50, nu1=2, nu2=2, coarse_min=4,
                 inner_cycles=1, cycle="V", smoother="rbgs", omega=0.8, fp64_jump_ratio=2.0,
                 coarse="auto") -> MgOptions:
    o = MgOptions()
    check(load().mg_default_options(C.byref(o)))
    o.precision = MG_MIXED if precision in ("mixed", MG_MIXED) else MG_FP64
    o.rtol, o.max_cycles, o.nu1, o.nu2 = float(rtol), int(max_cycles), int(nu1), int(nu2)
    o.coarse_min, o.inner_cycles = int(coarse_min), int(inner_cycles)
    o.cycle = CYCLES[cycle] if isinstance(cycle, str) else int(cycle)
    o.smoother = SMOOTHERS[smoother] if isinstance(smoother, str) else int(smoother)
    o.omega = float(omega)
    o.fp64_jump_ratio = float(fp64_jump_ratio)
    o.coarse_solve = COARSE[coarse] if isinstance(coarse, str) else int(coarse)
    return o


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, on_device: bool, dtype=np.float64):
    """(pointer, keepalive) for a numpy array or a CPU torch tensor (host; pinned
    CPU tensors give the fastest copies) or a CUDA tensor (device)."""
    if on_device:
        import torch
        if not (_is_torch(a) and a.is_cuda and a.dtype == torch.float64 and a.is_contiguous()):
            raise TypeError("device arrays must be contiguous float64 CUDA tensors")
        return C.c_void_p(a.data_ptr()), a
    if _is_torch(a):
        import torch
        if not (a.dtype == torch.float64 and a.is_contiguous()):
            raise TypeError("host tensors must be contiguous float64")
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return C.c_void_p(arr.ctypes.data), arr


def _side(*arrays) -> bool:
    flags = {_is_torch(a) and a.is_cuda for a in arrays if a is not None}
    if len(flags) > 1:
        raise TypeError("mix of host and device arrays in one call")
    return flags.pop() if flags else False


def residual_norms_noalloc(grid, lam, fa, fk, b, x, out, stream=None) -> None:
    """mg_residual_norms_noalloc: every array a contiguous float64 CUDA tensor;
    out (2 values) receives the per-field norms.  No device allocation."""
    import torch
    g = make_grid(grid)
    pa = (C.c_void_p * 3)()
    pk = (C.c_void_p * 3)()
    for a in range(g.dim):
        pa[a] = _ptr(fa[a], True)[0]
        pk[a] = _ptr(fk[a], True)[0]
    if stream is None:
        stream = torch.cuda.current_stream()
    check(load().mg_residual_norms_noalloc(C.byref(g), _ptr(lam, True)[0], pa, pk, _ptr(b, True)[0],
                                           _ptr(x, True)[0], _ptr(out, True)[0], C.c_void_p(stream.cuda_stream)))


def copy_h2d(dst, src, stream=None):
    """mg_copy_h2d_async: dst (CUDA tensor) <- src (page-locked CPU tensor of the
    same size in bytes), copied by a kernel on `stream` (default: the current
    one); returns dst.  Asynchronous, like a non-blocking copy."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nbytes or not dst.is_contiguous() or not src.is_contiguous():
        raise ValueError("copy_h2d: contiguous tensors of the same size in bytes")
    check(load().mg_copy_h2d_async(C.c_void_p(dst.data_ptr()), C.c_void_p(src.data_ptr()), C.c_size_t(nbytes),
                                   C.c_void_p(stream.cuda_stream)))
    return dst


def fp64_fma_rate(repeats: int = 5, stream=None) -> float:
    """mg_fp64_fma_rate: the current device's measured FP64 FMA rate, G instructions per second."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    out = C.c_double()
    check(load().mg_fp64_fma_rate(C.c_void_p(stream.cuda_stream), int(repeats), C.byref(out)))
    return out.value


def make_phase(ph) -> MgPhase:
    """From an object or dict with Gamma, Pi, b, q, cp, cv, k and optionally mu (0 if absent)."""
    get = (lambda key: ph.get(key, 0.0)) if isinstance(ph, dict) else (lambda key: getattr(ph, key, 0.0))
    return MgPhase(*(float(get(key)) for key in ("Gamma", "Pi", "b", "q", "cp", "cv", "k", "mu")))


MG_ASSEMBLE_LAMBDA4_PRINTED, MG_ASSEMBLE_HARMONIC_K = 1, 2
MG_MOMENTUM_NO_SLIP, MG_MOMENTUM_MULTIGRID, MG_MOMENTUM_KRYLOV = 1, 2, 4


def assemble(grid, phases, dt: float, C_, m1, m2, E, mom: Sequence, uf: Sequence, out: dict,
             lambda4_printed: bool = False, harmonic_k: bool = False, stream=None) -> None:
    """mg_assemble_async: every array a contiguous float64 CUDA tensor.  out holds
    "lam" (N x 4), "b" (N x 2), optionally "x0" (N x 2), and per-axis lists
    "fa", "fk"; they are written in place, in the order of `stream` (the call
    does not wait for the work)."""
    import torch
    g = make_grid(grid)
    keep = []

    def dev(a):
        p, k_ = _ptr(a, True)
        keep.append(k_)
        return p

    st = MgState()
    st.C, st.m1, st.m2, st.E = dev(C_), dev(m1), dev(m2), dev(E)
    res = MgAssembly()
    res.lam, res.rhs = dev(out["lam"]), dev(out["b"])
    res.x0 = dev(out["x0"]) if out.get("x0") is not None else None
    for a in range(g.dim):
        st.mom[a] = dev(mom[a])
        st.uf[a] = dev(uf[a])
        res.face_alpha[a] = dev(out["fa"][a])
        res.face_k[a] = dev(out["fk"][a])
    ph = (MgPhase * 2)(make_phase(phases[0]), make_phase(phases[1]))
    if stream is None:
        stream = torch.cuda.current_stream()
    flags = (MG_ASSEMBLE_LAMBDA4_PRINTED if lambda4_printed else 0) | (MG_ASSEMBLE_HARMONIC_K if harmonic_k else 0)
    check(load().mg_assemble_async(C.byref(g), ph, float(dt), flags, C.byref(st), C.byref(res),
                             C.c_void_p(stream.cuda_stream)))


def correct(grid, dt: float, sigma: float, x, C_, kappa, fa: Sequence, uf_star: Sequence, uf_out: Sequence, p1, p2,
            stream=None) -> None:
    """mg_correct_async: every array a contiguous float64 CUDA tensor; uf_out, p1, p2 are written in the order of
    `stream` (the call does not wait for the work)."""
    import torch
    g = make_grid(grid)
    pa, pu, po = (C.c_void_p * 3)(), (C.c_void_p * 3)(), (C.c_void_p * 3)()
    for a in range(g.dim):
        pa[a] = _ptr(fa[a], True)[0]
        pu[a] = _ptr(uf_star[a], True)[0]
        po[a] = _ptr(uf_out[a], True)[0]
    if stream is None:
        stream = torch.cuda.current_stream()
    check(load().mg_correct_async(C.byref(g), float(dt), float(sigma), _ptr(x, True)[0], _ptr(C_, True)[0],
                            _ptr(kappa, True)[0], pa, pu, po, _ptr(p1, True)[0], _ptr(p2, True)[0],
                            C.c_void_p(stream.cuda_stream)))


def energy(grid, phases, dt: float, x, C_, p1, p2, uf: Sequence, E1, E2, E1_out, E2_out, stream=None) -> None:
    """mg_energy_async: every array a contiguous float64 CUDA tensor; E1_out, E2_out (which may be E1, E2) are
    written in the order of `stream` (the call does not wait for the work)."""
    import torch
    g = make_grid(grid)
    pu = (C.c_void_p * 3)()
    for a in range(g.dim):
        pu[a] = _ptr(uf[a], True)[0]
    ph = (MgPhase * 2)(make_phase(phases[0]), make_phase(phases[1]))
    if stream is None:
        stream = torch.cuda.current_stream()
    d = lambda a: _ptr(a, True)[0]
    check(load().mg_energy_async(C.byref(g), ph, float(dt), d(x), d(C_), d(p1), d(p2), pu, d(E1), d(E2),
                                 d(E1_out), d(E2_out), C.c_void_p(stream.cuda_stream)))


class Solver:
    """One mg_handle: a grid, its device hierarchy and a stream."""

    def __init__(self, grid, precision="fp64", rtol=1e-10, max_cycles=50, nu1=2, nu2=2, coarse_min=4,
                 inner_cycles=1, device: Optional[int] = None, stream=None, torch_workspace: bool = True,
                 cycle="V", smoother="rbgs", omega=0.8, fp64_jump_ratio=2.0, coarse="auto"):
        import torch
        lib = load()
        self._lib = lib
        self.grid = make_grid(grid)
        self.options = make_options(precision, rtol, max_cycles, nu1, nu2, coarse_min, inner_cycles, cycle,
                                    smoother, omega, fp64_jump_ratio, coarse)
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        check(lib.mg_set_device(dev))
        nbytes = C.c_size_t()
        check(lib.mg_workspace_size(C.byref(self.grid), C.byref(self.options), C.byref(nbytes)))
        self.workspace_bytes = int(nbytes.value)
        self._ws = None
        ws_ptr = None
        if torch_workspace:
            self._ws = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=f"cuda:{dev}")
            ws_ptr = C.c_void_p(self._ws.data_ptr())
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        handle = C.c_void_p()
        check(lib.mg_create(C.byref(self.grid), C.byref(self.options), ws_ptr, self.workspace_bytes,
                            C.c_void_p(stream.cuda_stream), C.byref(handle)))
        self._h = handle
        self.N = self.grid.n[0] * self.grid.n[1] * self.grid.n[2]

    # -------------------------------------------------------------- sizes
    def nfaces(self, a: int) -> int:
        n = [self.grid.n[0], self.grid.n[1], self.grid.n[2]]
        n[a] += 1
        return n[0] * n[1] * n[2]

    @staticmethod
    def _numel(a) -> int:
        return int(a.numel()) if _is_torch(a) else int(np.asarray(a).size)

    def _need(self, a, count: int, what: str):
        if self._numel(a) != count:
            raise ValueError(f"{what}: expected {count} values, got {self._numel(a)}")

    # -------------------------------------------------------------- calls
    def set_coeffs(self, lam, fa: Sequence, fk: Sequence):
        self._need(lam, 4 * self.N, "lambda")
        if len(fa) < self.grid.dim or len(fk) < self.grid.dim:
            raise ValueError("one face array per axis is required")
        for a in range(self.grid.dim):
            self._need(fa[a], self.nfaces(a), f"face_alpha[{a}]")
            self._need(fk[a], self.nfaces(a), f"face_k[{a}]")
        dev = _side(lam, *fa[: self.grid.dim], *fk[: self.grid.dim])
        lp, keep = _ptr(lam, dev)
        pa = (C.c_void_p * 3)()
        pk = (C.c_void_p * 3)()
        keeps = [keep]
        for a in range(self.grid.dim):
            p1, k1 = _ptr(fa[a], dev)
            p2, k2 = _ptr(fk[a], dev)
            pa[a], pk[a] = p1, p2
            keeps += [k1, k2]
        check(self._lib.mg_set_coeffs(self._h, lp, pa, pk, int(dev)))

    def solve(self, b, x, allow_not_converged: bool = False) -> dict:
        """Solves in place: x (numpy float64 [N,2] or CUDA tensor) holds the
        initial guess and receives the result.  Returns the stats."""
        self._need(b, 2 * self.N, "rhs")
        self._need(x, 2 * self.N, "x")
        dev = _side(b, x)
        bp, bk = _ptr(b, dev)
        if not dev and not _is_torch(x):
            if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
                raise TypeError("host x must be a C-contiguous float64 numpy array (solved in place)")
        xp, xk = _ptr(x, dev)
        st = MgStats()
        allow = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        check(self._lib.mg_solve(self._h, bp, xp, int(dev), C.byref(st)), allow)
        return st.as_dict()

    def solve_async(self, b, x, event=None) -> None:
        """mg_solve_async: b and x contiguous float64 CUDA tensors; the solve is
        enqueued on the handle's stream and x holds the result once it has run.
        event: None or a torch.cuda.Event, recorded after the solve (keep b alive
        until then)."""
        self._need(b, 2 * self.N, "rhs")
        self._need(x, 2 * self.N, "x")
        bp, _ = _ptr(b, True)
        xp, _ = _ptr(x, True)
        ev = None
        if event is not None:
            if not event.cuda_event:           # torch creates the CUDA event on its first record
                event.record(self.stream)
            ev = C.c_void_p(event.cuda_event)
        check(self._lib.mg_solve_async(self._h, bp, xp, ev))

    def async_stats(self, allow_not_converged: bool = False) -> dict:
        """mg_solve_async_stats: waits for the last solve_async and returns its stats."""
        st = MgStats()
        allow = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        check(self._lib.mg_solve_async_stats(self._h, C.byref(st)), allow)
        return st.as_dict()

    def apply(self, x):
        self._need(x, 2 * self.N, "x")
        dev = _side(x)
        xp, xk = _ptr(x, dev)
        if dev:
            import torch
            y = torch.empty_like(x)
        else:
            y = np.empty_like(xk)
        yp, yk = _ptr(y, dev)
        check(self._lib.mg_apply(self._h, xp, yp, int(dev)))
        return y

    def smooth(self, b, x, sweeps: int = 1):
        self._need(b, 2 * self.N, "rhs")
        self._need(x, 2 * self.N, "x")
        if not _is_torch(x) and not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
            raise TypeError("host x must be a C-contiguous float64 numpy array (smoothed in place)")
        dev = _side(b, x)
        bp, bk = _ptr(b, dev)
        xp, xk = _ptr(x, dev)
        check(self._lib.mg_smooth(self._h, bp, xp, int(sweeps), int(dev)))
        return x

    def residual_norms(self, b, x) -> np.ndarray:
        self._need(b, 2 * self.N, "rhs")
        self._need(x, 2 * self.N, "x")
        dev = _side(b, x)
        bp, bk = _ptr(b, dev)
        xp, xk = _ptr(x, dev)
        out = (C.c_double * 2)()
        check(self._lib.mg_residual_norms(self._h, bp, xp, int(dev), out))
        return np.array(list(out))

    def set_stream(self, stream):
        """Runs this handle's later work on `stream` (a torch.cuda.Stream)."""
        check(self._lib.mg_set_stream(self._h, C.c_void_p(stream.cuda_stream)))
        self.stream = stream

    def set_timing(self, enable: bool = True):
        check(self._lib.mg_set_timing(self._h, int(enable)))

    def counters(self) -> dict:
        n, ms, sl, sw, sc = C.c_longlong(), C.c_double(), C.c_longlong(), C.c_longlong(), C.c_longlong()
        check(self._lib.mg_counters(self._h, C.byref(n), C.byref(ms), C.byref(sl), C.byref(sw), C.byref(sc)))
        return dict(launches=n.value, smooth_ms=ms.value, smooth_launches=sl.value, smooth_sweeps=sw.value,
                    smooth_cells=sc.value)

    def tuning(self) -> dict:
        """The handle's kernel choices (see mg_tuning in the header)."""
        t = MgTuning()
        check(self._lib.mg_get_tuning(self._h, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, tuning: dict):
        t = MgTuning.from_dict(tuning)
        check(self._lib.mg_set_tuning(self._h, C.byref(t)))

    def autotune(self, reps: int = 10):
        """Runs the library's autotuner on this hierarchy; returns (tuning, V-cycle ms)."""
        t = MgTuning()
        ms = C.c_double()
        check(self._lib.mg_autotune(self._h, int(reps), C.byref(t), C.byref(ms)))
        return t.as_dict(), ms.value

    def levels(self):
        n = C.c_int()
        sizes = (C.c_int * (3 * 32))()
        check(self._lib.mg_levels(self._h, C.byref(n), sizes))
        return [tuple(sizes[3 * l: 3 * l + 3]) for l in range(n.value)]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mg_destroy(self._h)
            self._h = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _ptr3(g, arrs):
    out = (C.c_void_p * 3)()
    for a in range(g.dim):
        out[a] = _ptr(arrs[a], True)[0]
    return out


def momentum_rhs(grid, dt: float, sigma: float, mom: Sequence, p, kappa, C_, R: Sequence, stream=None) -> None:
    """mg_momentum_rhs_async: every array a contiguous float64 CUDA tensor; R written in the order of `stream`."""
    import torch
    g = make_grid(grid)
    if stream is None:
        stream = torch.cuda.current_stream()
    check(load().mg_momentum_rhs_async(C.byref(g), float(dt), float(sigma), _ptr3(g, mom), _ptr(p, True)[0],
                                       _ptr(kappa, True)[0], _ptr(C_, True)[0], _ptr3(g, R),
                                       C.c_void_p(stream.cuda_stream)))


def provisional(grid, dt: float, rho, p, u_pred: Sequence, uf_out: Sequence, stream=None) -> None:
    """mg_provisional_async: every array a contiguous float64 CUDA tensor; uf_out written in the order of `stream`."""
    import torch
    g = make_grid(grid)
    if stream is None:
        stream = torch.cuda.current_stream()
    check(load().mg_provisional_async(C.byref(g), float(dt), _ptr(rho, True)[0], _ptr(p, True)[0],
                                      _ptr3(g, u_pred), _ptr3(g, uf_out), C.c_void_p(stream.cuda_stream)))


class Momentum:
    """mg_momentum: the implicit momentum predictor (rho/dt) u - div(mu (grad u + grad u^T)) = R on one grid.
    Arrays are contiguous float64 CUDA tensors of the grid's cells, one per velocity component."""

    def __init__(self, grid, no_slip: bool = False, inner_cycles_per_step: int = 1, nu1=2, nu2=2,
                 coarse_min=4, device: Optional[int] = None, stream=None, multigrid_only: bool = False,
                 krylov: bool = False):
        import torch
        lib = load()
        self._lib = lib
        self.grid = make_grid(grid)
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        check(lib.mg_set_device(dev))
        opt = make_options("fp64", 0.0, inner_cycles_per_step, nu1, nu2, coarse_min)
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        handle = C.c_void_p()
        flags = ((MG_MOMENTUM_NO_SLIP if no_slip else 0) | (MG_MOMENTUM_MULTIGRID if multigrid_only else 0) |
                 (MG_MOMENTUM_KRYLOV if krylov else 0))
        check(lib.mg_momentum_create(C.byref(self.grid), flags, C.byref(opt),
                                     C.c_void_p(stream.cuda_stream), C.byref(handle)))
        self._h = handle

    def _list(self, v):
        arr = (C.c_void_p * 3)()
        for a in range(self.grid.dim):
            arr[a] = _ptr(v[a], True)[0]
        return arr

    def set_coeffs(self, dt: float, rho, mu) -> None:
        check(self._lib.mg_momentum_set_coeffs(self._h, float(dt), _ptr(rho, True)[0], _ptr(mu, True)[0]))

    def apply(self, u: Sequence, y: Sequence) -> None:
        check(self._lib.mg_momentum_apply(self._h, self._list(u), self._list(y)))

    def solve(self, R: Sequence, u: Sequence, rtol: float = 1e-10, max_iters: int = 100,
              allow_not_converged: bool = False) -> dict:
        st = MgMomentumStats()
        allow = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        check(self._lib.mg_momentum_solve(self._h, self._list(R), self._list(u), float(rtol), int(max_iters),
                                          C.byref(st)), allow)
        return st.as_dict()

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mg_momentum_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Batch:
    """mg_batch over existing Solvers (same dim, options, stream): one set of
    launches per V-cycle stage for all of them."""

    def __init__(self, solvers: Sequence["Solver"]):
        self._lib = load()
        self.solvers = list(solvers)
        hs = (C.c_void_p * len(self.solvers))(*[s._h for s in self.solvers])
        out = C.c_void_p()
        check(self._lib.mg_batch_create(len(self.solvers), hs, C.byref(out)))
        self._b = out

    def set_coeffs(self, lams: Sequence, fas: Sequence, fks: Sequence):
        """Coefficients of every problem in one set of launches."""
        n = len(self.solvers)
        if not (len(lams) == len(fas) == len(fks) == n):
            raise ValueError("one coefficient set per problem")
        dev = _side(*lams, *[f for fa in fas for f in fa[:3]], *[f for fk in fks for f in fk[:3]])
        keep = []
        pl = (C.c_void_p * n)()
        pa = (C.c_void_p * (3 * n))()
        pk = (C.c_void_p * (3 * n))()
        for q, (s, lam, fa, fk) in enumerate(zip(self.solvers, lams, fas, fks)):
            s._need(lam, 4 * s.N, "lambda")
            p, k = _ptr(lam, dev)
            pl[q] = p
            keep.append(k)
            for a in range(s.grid.dim):
                s._need(fa[a], s.nfaces(a), f"face_alpha[{a}]")
                s._need(fk[a], s.nfaces(a), f"face_k[{a}]")
                p1, k1 = _ptr(fa[a], dev)
                p2, k2 = _ptr(fk[a], dev)
                pa[3 * q + a], pk[3 * q + a] = p1, p2
                keep += [k1, k2]
        check(self._lib.mg_batch_set_coeffs(self._b, pl, pa, pk, int(dev)))

    def solve(self, bs: Sequence, xs: Sequence, allow_not_converged: bool = False) -> list:
        n = len(self.solvers)
        if len(bs) != n or len(xs) != n:
            raise ValueError("one rhs and one x per problem")
        dev = _side(*bs, *xs)
        keep = []
        pb = (C.c_void_p * n)()
        px = (C.c_void_p * n)()
        for q, (s, b, x) in enumerate(zip(self.solvers, bs, xs)):
            s._need(b, 2 * s.N, "rhs")
            s._need(x, 2 * s.N, "x")
            if not dev and not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
                raise TypeError("host x must be C-contiguous float64 numpy arrays (solved in place)")
            p1, k1 = _ptr(b, dev)
            p2, k2 = _ptr(x, dev)
            pb[q], px[q] = p1, p2
            keep += [k1, k2]
        st = (MgStats * n)()
        allow = (MG_OK, MG_ERR_NOT_CONVERGED) if allow_not_converged else (MG_OK,)
        check(self._lib.mg_batch_solve(self._b, pb, px, int(dev), st), allow)
        return [st[q].as_dict() for q in range(n)]

    def tuning(self) -> dict:
        t = MgBatchTuning()
        check(self._lib.mg_batch_get_tuning(self._b, C.byref(t)))
        return t.as_dict()

    def set_tuning(self, tuning: dict):
        t = MgBatchTuning.from_dict(tuning)
        check(self._lib.mg_batch_set_tuning(self._b, C.byref(t)))

    def autotune(self, reps: int = 5):
        """The library's batch autotuner; returns (tuning, ms of one V-cycle of the whole batch)."""
        t = MgBatchTuning()
        ms = C.c_double()
        check(self._lib.mg_batch_autotune(self._b, int(reps), C.byref(t), C.byref(ms)))
        return t.as_dict(), ms.value

    def launches(self) -> int:
        n = C.c_longlong()
        check(self._lib.mg_batch_counters(self._b, C.byref(n)))
        return n.value

    def close(self):
        if getattr(self, "_b", None):
            self._lib.mg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Composite:
    """mg_composite: a refined-patch (adaptive) grid, base grid plus one 2:1 box."""

    def __init__(self, grid, box, nu1=2, nu2=2, coarse_min=4, device: Optional[int] = None, stream=None,
                 precision="fp64"):
        import torch
        lib = load()
        self._lib = lib
        self.grid = make_grid(grid)
        self.box = tuple(tuple(int(v) for v in box[a]) for a in range(2))
        dev = torch.cuda.current_device() if device is None else int(device)
        self.device = dev
        check(lib.mg_set_device(dev))
        if stream is None:
            stream = torch.cuda.current_stream(dev)
        self.stream = stream
        o = make_options(precision, 0.0, 1, nu1, nu2, coarse_min)
        b = ((C.c_int * 2) * 2)(*[(C.c_int * 2)(*self.box[a]) for a in range(2)])
        h = C.c_void_p()
        check(lib.mg_composite_create(C.byref(self.grid), b, C.byref(o), C.c_void_p(stream.cuda_stream), C.byref(h)))
        self._h = h
        self.Nb = self.grid.n[0] * self.grid.n[1]
        self.m = (2 * (self.box[0][1] - self.box[0][0]), 2 * (self.box[1][1] - self.box[1][0]))
        self.Nf = self.m[0] * self.m[1]

    @staticmethod
    def _dev(a):
        import torch
        if _is_torch(a) and a.is_cuda:
            return a
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()

    def set_coeffs(self, lam_b, fa_b, fk_b, lam_f, fa_f, fk_f):
        d = self._dev
        self._keep = [d(lam_b), [d(f) for f in fa_b], [d(f) for f in fk_b], d(lam_f), [d(f) for f in fa_f],
                      [d(f) for f in fk_f]]
        lb, fab, fkb, lf, faf, fkf = self._keep
        arr = lambda fs: (C.c_void_p * 3)(*[C.c_void_p(f.data_ptr()) for f in fs], None)
        check(self._lib.mg_composite_set_coeffs(self._h, C.c_void_p(lb.data_ptr()), arr(fab), arr(fkb),
                                                C.c_void_p(lf.data_ptr()), arr(faf), arr(fkf)))

    def apply(self, xb, xf):
        import torch
        xb, xf = self._dev(xb), self._dev(xf)
        yb, yf = torch.empty_like(xb), torch.empty_like(xf)
        check(self._lib.mg_composite_apply(self._h, C.c_void_p(xb.data_ptr()), C.c_void_p(xf.data_ptr()),
                                           C.c_void_p(yb.data_ptr()), C.c_void_p(yf.data_ptr())))
        return yb, yf

    def solve(self, bb, bf, xb, xf, cycles: int, norms: bool = True):
        """xb, xf: CUDA tensors solved in place (numpy arrays: copies returned).
        Returns (xb, xf, norms [cycles + 1, 4] or None)."""
        bb, bf, xb, xf = self._dev(bb), self._dev(bf), self._dev(xb), self._dev(xf)
        h = np.zeros(4 * (cycles + 1)) if norms else None
        check(self._lib.mg_composite_solve(self._h, C.c_void_p(bb.data_ptr()), C.c_void_p(bf.data_ptr()),
                                           C.c_void_p(xb.data_ptr()), C.c_void_p(xf.data_ptr()), int(cycles),
                                           h.ctypes.data_as(C.POINTER(C.c_double)) if norms else None))
        return xb, xf, (h.reshape(-1, 4) if norms else None)

    def autotune(self, reps: int = 5) -> float:
        """Kernel choices of the base hierarchy (mg_composite_autotune); returns the V-cycle's ms."""
        ms = C.c_double(0.0)
        check(self._lib.mg_composite_autotune(self._h, int(reps), C.byref(ms)))
        return ms.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mg_composite_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

