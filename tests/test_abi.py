"""C-ABI checks that need no GPU: the library builds, loads and exports every
symbol include/*.h declares; host-side argument validation and workspace
sizing (no device work)."""
import ctypes as C
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        names |= set(re.findall(r"^MG_API\s+[\w\s\*]+?\b(mg_\w+)\s*\(", src, flags=re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2206_11294_gb300 import build, binding
    build.build()
    return binding.load()


def test_every_declared_symbol_is_exported(lib):
    from paper_2206_11294_gb300 import binding
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert names == set(binding.EXPORTS), names ^ set(binding.EXPORTS)


def test_default_options(lib):
    from paper_2206_11294_gb300 import binding as B
    o = B.MgOptions()
    assert lib.mg_default_options(C.byref(o)) == 0
    assert (o.nu1, o.nu2, o.precision, o.max_cycles, o.coarse_min, o.inner_cycles) == (2, 2, 0, 50, 4, 1)
    assert o.rtol == 1e-10
    assert o.cycle == B.CYCLES["V"] == 0 and B.CYCLES == {"V": 0, "W": 1, "F": 2}
    assert o.smoother == B.SMOOTHERS["rbgs"] == 0 and o.omega == 0.8 and o.fp64_jump_ratio == 2.0
    assert o.coarse_solve == B.COARSE["auto"] == 0 and B.COARSE == {"auto": 0, "inverse": 1}


def test_cycle_option_validated(lib):
    st, _ = _size(lib, _grid(n=(64, 64, 1)), cycle="W")
    assert st == 0
    st, _ = _size(lib, _grid(n=(64, 64, 1)), cycle=3)
    assert st != 0


def _grid(**kw):
    from paper_2206_11294_gb300 import binding as B, inputs as I
    g = I.Grid(dim=kw.get("dim", 2), axisym=kw.get("axisym", 0), n=kw.get("n", (64, 64, 1)), h=kw.get("h", 1 / 64),
               r0=kw.get("r0", 0.0), bc=kw.get("bc", ((0, 0), (0, 0), (0, 0))))
    return B.make_grid(g)


def _size(lib, g, **okw):
    from paper_2206_11294_gb300 import binding as B
    o = B.make_options(**okw)
    n = C.c_size_t()
    st = lib.mg_workspace_size(C.byref(g), C.byref(o), C.byref(n))
    return st, n.value


def test_workspace_size_scales_with_levels(lib):
    st, a = _size(lib, _grid(n=(64, 64, 1)))
    st2, b = _size(lib, _grid(n=(128, 128, 1)))
    st3, c = _size(lib, _grid(n=(128, 128, 1)), precision="mixed")
    assert st == st2 == st3 == 0
    # hierarchy ~ 4/3 of the finest level; 4x the cells -> about 4x the bytes
    assert 3.5 < b / a < 4.5
    assert c > b


@pytest.mark.parametrize("kw,okw", [
    (dict(dim=4), {}),
    (dict(dim=2, n=(64, 64, 2)), {}),
    (dict(axisym=1, dim=3, n=(8, 8, 8)), {}),
    (dict(h=-1.0), {}),
    (dict(bc=((2, 0), (0, 0), (0, 0))), {}),                      # axis on a Cartesian grid
    (dict(axisym=1, r0=0.0, bc=((1, 0), (0, 0), (0, 0))), {}),   # Dirichlet on the axis
    (dict(n=(96, 160, 1)), {}),                                   # 6 x 10 x 2 coarse unknowns fine
    (dict(n=(1000, 1000, 1)), {}),                                # coarsest 125 x 125: too large
    ({}, dict(nu1=0, nu2=0)),
    ({}, dict(max_cycles=-1)),
    ({}, dict(smoother=2)),
    ({}, dict(smoother="wjac", omega=1.5)),
    ({}, dict(fp64_jump_ratio=0.5)),
    ({}, dict(fp64_jump_ratio=float("inf"))),
    ({}, dict(coarse=2)),
    ({}, dict(coarse=-1)),
])
def test_argument_validation(lib, kw, okw):
    st, _ = _size(lib, _grid(**kw), **okw)
    ok_cases = [dict(n=(96, 160, 1))]
    if kw in ok_cases and not okw:
        assert st == 0
    else:
        assert st == 1, lib.mg_last_error()
        assert len(lib.mg_last_error()) > 0


def test_product_path_has_no_oracle_dependency():
    """The package and the library never import, load or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2206_11294_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".cuh", ".h")):
            src = open(path).read()
            assert "import oracle" not in src and "coupled_oracle" not in src, path


def test_momentum_and_side_steps_validate_on_the_host(lib):
    """Argument checks of the momentum predictor and the steps around the solves, made before any device work."""
    from paper_2206_11294_gb300 import binding as B
    g = _grid(n=(64, 64, 1))
    h = C.c_void_p()
    assert lib.mg_momentum_create(C.byref(g), 8, None, None, C.byref(h)) == B.MG_ERR_INVALID_ARG
    assert not h.value
    o = B.make_options("mixed", 0.0, 1)
    assert lib.mg_momentum_create(C.byref(g), 0, C.byref(o), None, C.byref(h)) == B.MG_ERR_INVALID_ARG
    o = B.make_options("fp64", 0.0, 0)
    assert lib.mg_momentum_create(C.byref(g), 0, C.byref(o), None, C.byref(h)) == B.MG_ERR_INVALID_ARG
    assert lib.mg_momentum_create(C.byref(g), 0, None, None, None) == B.MG_ERR_INVALID_ARG
    assert lib.mg_momentum_set_coeffs(None, 1e-3, None, None) == B.MG_ERR_INVALID_ARG
    pa = (C.c_void_p * 3)()
    assert lib.mg_momentum_solve(None, pa, pa, 1e-10, 10, None) == B.MG_ERR_INVALID_ARG
    assert lib.mg_momentum_apply(None, pa, pa) == B.MG_ERR_INVALID_ARG
    assert lib.mg_momentum_destroy(None) == B.MG_OK
    for dt in (0.0, -1.0, float("nan")):
        assert lib.mg_momentum_rhs_async(C.byref(g), dt, 0.07, pa, None, None, None, pa, None) == B.MG_ERR_INVALID_ARG
        assert lib.mg_provisional_async(C.byref(g), dt, None, None, pa, pa, None) == B.MG_ERR_INVALID_ARG
        ph = (B.MgPhase * 2)()
        assert lib.mg_energy_async(C.byref(g), ph, dt, None, None, None, None, pa, None, None, None, None,
                                   None) == B.MG_ERR_INVALID_ARG
    assert "dt" in B.last_error()


@pytest.mark.parametrize("bad", [
    dict(bc=((7, 0), (0, 0), (0, 0))),                           # unknown boundary kind
    dict(bc=((0, 2), (0, 0), (0, 0))),                           # the axis on the high side
    dict(axisym=1, r0=0.1, bc=((2, 0), (0, 0), (0, 0))),         # the axis where r0 != 0
    dict(axisym=1, r0=float("nan")),
    dict(h=float("inf")),
])
def test_noalloc_checks_grids_like_mg_create(lib, bad):
    """The allocation-free norm applies mg_create's grid rules: a bad grid gets
    the same status from both, before any device work (dummy host pointers)."""
    from paper_2206_11294_gb300 import binding as B
    g = _grid(**bad)
    st_create, _ = _size(lib, g)
    dummy = (C.c_double * 8)()
    p = C.cast(dummy, C.c_void_p)
    pa = (C.c_void_p * 3)(p, p, p)
    st = lib.mg_residual_norms_noalloc(C.byref(g), p, pa, pa, p, p, p, None)
    assert st_create == st == B.MG_ERR_INVALID_ARG, (st_create, st, B.last_error())


def test_factored_coarse_solve_needs_no_inverse(lib):
    """With the default coarse solve a 31 x 31 coarsest level (n = 992: 1922
    unknowns, the windowed path) keeps its LU factors and no dense inverse:
    the workspace is smaller by the FP64 inverse (and its FP32 copy in mixed
    precision) than with MG_COARSE_INVERSE.  Small coarsest levels are the
    same either way."""
    nc = 2 * 31 * 31
    for prec, per in (("fp64", 8), ("mixed", 12)):
        st, auto = _size(lib, _grid(n=(992, 992, 1), h=1 / 992), precision=prec)
        st2, inv = _size(lib, _grid(n=(992, 992, 1), h=1 / 992), precision=prec, coarse="inverse")
        assert st == st2 == 0
        assert 0 <= (inv - auto) - per * nc * nc <= 4096
    st, a = _size(lib, _grid(n=(1024, 1024, 1), h=1 / 1024))
    st2, b = _size(lib, _grid(n=(1024, 1024, 1), h=1 / 1024), coarse="inverse")
    assert st == st2 == 0 and a == b


def test_binding_constants_match_the_header():
    """Every MG_* enum value the binding defines equals the header's, and the
    header's sweep kinds, status codes and flags all have a binding name."""
    from paper_2206_11294_gb300 import binding as B
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    text = open(os.path.join(root, "include", "coupledmg.h")).read()
    header = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(MG_[A-Z0-9_]+)\s*=\s*(-?\d+)", text)}
    assert header["MG_SWEEP_FUSED2"] == 5 and header["MG_ERR_STATE"] == 8
    bound = {k: getattr(B, k) for k in dir(B) if k.startswith("MG_") and isinstance(getattr(B, k), int)}
    for k, v in bound.items():
        if k in header:
            assert header[k] == v, k
    for k in header:
        named = k.startswith(("MG_SWEEP_", "MG_ERR_", "MG_ASSEMBLE_", "MG_MOMENTUM_"))
        if named or k in ("MG_OK", "MG_FP64", "MG_MIXED"):
            assert k in bound, k
