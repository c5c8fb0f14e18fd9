"""Planted mistakes: each mutant copy of the oracle (compiled on the CPU) must
fail at least one of the pins, so the pins would catch that kind of error in
the oracle itself (and, through the parity tests, in the CUDA path)."""
import contextlib
import os
import shutil
import tempfile

import ctypes as C
import numpy as np
import pytest

import fv_matrix as fv
from paper_2206_11294_gb300 import inputs as I

W, D, A = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS

MUTATIONS = {
    # Dirichlet boundary value at h instead of h/2
    "dirichlet_distance": ("sum += A * cf * (gv - u[2 * i]) / (0.5 * g->h);", "sum += A * cf * (gv - u[2 * i]) / g->h;"),
    # p-row of the defining operator loses l4 div(k grad T) (Eq. 28)
    "drop_l4_operator": ("y[2 * i + 1] = lapp + l[2] * p + l[3] * lapT;", "y[2 * i + 1] = lapp + l[2] * p;"),
    # the same term dropped only inside the multigrid's rows: the defect
    # correction still converges, so the sweep pin has to catch it
    "drop_l4_smoother": ("out[1] = lapp + l[2] * u[2 * i + 1] + l[3] * lapT;", "out[1] = lapp + l[2] * u[2 * i + 1];"),
    # axisymmetric r-face area taken at the cell centre
    "axi_face_area": ("return (a == 0 ? r_face(g, f[0]) : r_cell(g, c[0])) * g->h;",
                      "return (a == 0 ? r_cell(g, c[0]) : r_cell(g, c[0])) * g->h;"),
    # sign error in the 2x2 block solve
    "block_solve_sign": ("z[1] = (D[0] * s[1] - D[2] * s[0]) / det;", "z[1] = (D[0] * s[1] + D[2] * s[0]) / det;"),
    # prolongation weights 1/2 instead of 3/4 and 1/4
    "prolongation_weights": ("                    w *= 0.25;", "                    w *= 0.5;"),
}


@contextlib.contextmanager
def mutant(orc, name):
    old, new = MUTATIONS[name]
    src = open(os.path.join(os.path.dirname(orc.__file__), "coupled_oracle.c")).read()
    assert src.count(old) >= 1, name
    d = tempfile.mkdtemp()
    try:
        path = os.path.join(d, "m.c")
        open(path, "w").write(src.replace(old, new))
        lib = orc.configure(C.CDLL(orc.compile_source(path, os.path.join(d, "m.so"))))
        saved = orc._lib
        orc._lib = lib
        try:
            yield
        finally:
            orc._lib = saved
    finally:
        shutil.rmtree(d, ignore_errors=True)


def _pins_pass(orc) -> bool:
    """A few pins (closed-form modes, sparse assembly, dense vs multigrid,
    multigrid convergence); False as soon as one fails."""
    rng = np.random.default_rng(0)
    grids = [I.Grid(dim=2, axisym=0, n=(6, 10, 1), h=0.1, bc=((W, D), (D, W), (0, 0)),
                    bcT=((1, 2), (3, 4), (0, 0)), bcp=((5, 6), (7, 8), (0, 0))),
             I.Grid(dim=2, axisym=1, n=(4, 8, 1), h=0.1, bc=((A, D), (W, D), (0, 0)),
                    bcT=((0, 2), (3, 4), (0, 0)), bcp=((0, 6), (7, 8), (0, 0)))]
    for g in grids:
        lam = rng.standard_normal((g.N, 4))
        fa = [rng.uniform(0.5, 2, int(np.prod(g.face_shape(a)))) for a in range(g.dim)]
        fk = [rng.uniform(0.5, 2, int(np.prod(g.face_shape(a)))) for a in range(g.dim)]
        x = rng.standard_normal((g.N, 2))
        M, aff = fv.paper_operator(g, lam, fa, fk)
        ref = M @ x.reshape(-1) + aff
        if np.abs(orc.apply_paper(g.as_dict(), lam, fa, fk, x).reshape(-1) - ref).max() > 1e-12 * np.abs(ref).max():
            return False
        # one red-black sweep = the block Gauss-Seidel step of the assembled matrix
        b = rng.standard_normal((g.N, 2))
        x1 = orc.rbgs_sweeps(g.as_dict(), lam, fa, fk, b, x, sweeps=1)
        Md = M.toarray()
        rhs = b.reshape(-1) - aff
        idx = np.arange(g.N)
        red = ((idx % g.n[0] + idx // g.n[0]) % 2 == 0)
        order = np.concatenate([np.flatnonzero(red), np.flatnonzero(~red)])
        perm = np.stack([2 * order, 2 * order + 1], axis=1).reshape(-1)
        Mp, rp, xp = Md[perm][:, perm], rhs[perm], x.reshape(-1)[perm]
        Lo = np.zeros_like(Mp)
        for r in range(2 * g.N):
            Lo[r, : 2 * (r // 2) + 2] = Mp[r, : 2 * (r // 2) + 2]
        xn = np.linalg.solve(Lo, rp - (Mp - Lo) @ xp)
        gs = np.empty_like(xn)
        gs[perm] = xn
        if np.abs(x1.reshape(-1) - gs).max() > 1e-11 * np.abs(gs).max():
            return False
        p = I.random_coeff_problem(g, seed=7, dt=1e-5)
        xd = np.linalg.solve(fv.paper_operator(g, p.lam, p.fa, p.fk)[0].toarray(),
                             p.b.reshape(-1) - fv.paper_operator(g, p.lam, p.fa, p.fk)[1]).reshape(-1, 2)
        xm, cyc, _ = orc.mg_solve(g.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, coarse_min=2, max_cycles=80,
                                  rtol=1e-14)
        if np.linalg.norm(xm - xd) > 1e-10 * np.linalg.norm(xd - p.x0):
            return False
    p = I.stiff(I.bubble_2d, 64)
    x, cyc, hist = orc.mg_solve(p.grid.as_dict(), p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=40, rtol=1e-10)
    q = hist[1:, 1] / hist[:-1, 1]
    return cyc <= 20 and np.max(q[:-1]) < 0.3


def test_unmutated_oracle_passes_the_pins(orc):
    assert _pins_pass(orc)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutant_fails_a_pin(orc, name):
    with mutant(orc, name):
        assert not _pins_pass(orc), name


# Planted mistakes in the cycle variants, against the W/F pin (two coarse visits
# per level contract faster than one).
CYCLE_MUTATIONS = {
    # the second coarse visit of W- and F-cycles left out: every cycle is a V-cycle
    "no_second_visit": ("if (type != 0 && l + 1 < nlev - 1) {", "if (0 && l + 1 < nlev - 1) {"),
    # the second visit restarts the coarse correction from zero, discarding the first
    "second_visit_restarts": ("        rc = mgcycle(Ls, l + 1, nlev, nu1, nu2, type == 1 ? 1 : 0, sm);",
                              "        memset(Ls[l + 1].u, 0, sizeof(double) * 2 * Ls[l + 1].N);\n"
                              "        rc = mgcycle(Ls, l + 1, nlev, nu1, nu2, type == 1 ? 1 : 0, sm);"),
}


def _cycle_pins_pass(orc) -> bool:
    p = I.stiff(I.bubble_2d, 32)
    gd = p.grid.as_dict()
    rate = {}
    for c in "VW":
        _, _, hist = orc.mg_solve(gd, p.lam, p.fa, p.fk, p.b, p.x0, max_cycles=6, rtol=0.0, cycle=c)
        rate[c] = np.exp(np.log(hist[1:6] / hist[0:5]).mean(axis=0))
    return bool(np.all(rate["W"] <= 0.8 * rate["V"]))


def test_unmutated_oracle_passes_the_cycle_pin(orc):
    assert _cycle_pins_pass(orc)


@pytest.mark.parametrize("name", list(CYCLE_MUTATIONS))
def test_cycle_mutant_fails_the_pin(orc, name):
    MUTATIONS[name] = CYCLE_MUTATIONS[name]
    try:
        with mutant(orc, name):
            assert not _cycle_pins_pass(orc), name
    finally:
        del MUTATIONS[name]


# Planted mistakes in the grid transfers, against the transfer pins of
# test_oracle_pins.py (each only slows the multigrid down: no converged-solution
# pin sees it).
TRANSFER_MUTATIONS = {
    # restriction as a plain mean of the children, ignoring their volumes (r_i h^2 on axisymmetric grids)
    "restrict_plain_mean": ("            s0 += V * F->r[2 * f];\n            s1 += V * F->r[2 * f + 1];\n"
                            "            vsum += V;",
                            "            s0 += 1.0 * F->r[2 * f];\n            s1 += 1.0 * F->r[2 * f + 1];\n"
                            "            vsum += 1.0;"),
    # the Dirichlet ghost of the prolongation taken even (same value) instead of odd
    "prolong_no_dirichlet_sign": ("if (C->g.bc[a][side] == BC_DIRICHLET) sign = -sign;", "if (0) sign = -sign;"),
    # every ghost taken odd, the walls' and the axis's too
    "prolong_odd_wall_ghost": ("if (C->g.bc[a][side] == BC_DIRICHLET) sign = -sign;", "sign = -sign;"),
    # prolongation stencil leaning the wrong way (toward the far coarse neighbour)
    "prolong_wrong_side": ("int s[3] = {(c[0] & 1) ? 1 : -1, (c[1] & 1) ? 1 : -1, (c[2] & 1) ? 1 : -1};",
                           "int s[3] = {(c[0] & 1) ? -1 : 1, (c[1] & 1) ? -1 : 1, (c[2] & 1) ? -1 : 1};"),
}


def _transfer_pins_pass(orc) -> bool:
    import test_oracle_pins as P
    try:
        for name in P.TRANSFER_GRIDS:
            P.test_restriction_conserves_the_volume_integral(orc, name)
            P.test_prolongation_reproduces_multilinear_fields(orc, name)
        P.test_prolongation_boundary_ghosts(orc)
    except AssertionError:
        return False
    return True


def test_unmutated_oracle_passes_the_transfer_pins(orc):
    assert _transfer_pins_pass(orc)


@pytest.mark.parametrize("name", list(TRANSFER_MUTATIONS))
def test_transfer_mutant_fails_a_pin(orc, name):
    MUTATIONS[name] = TRANSFER_MUTATIONS[name]
    try:
        with mutant(orc, name):
            assert not _transfer_pins_pass(orc), name
    finally:
        del MUTATIONS[name]


# Planted mistakes in the weighted block Jacobi smoother, against its pin.
WJAC_MUTATIONS = {
    # the weight omega left out: every cell jumps to its block solution
    "wjac_undamped": ("for (long i = 0; i < 2 * L->N; i++) L->u[i] = L->u[i] + omega * (z[i] - L->u[i]);",
                      "for (long i = 0; i < 2 * L->N; i++) L->u[i] = z[i];"),
    # cells updated in place, so later cells see new neighbours (a Gauss-Seidel sweep)
    "wjac_in_place": ("        solve2(D, s, z + 2 * i);\n",
                      "        solve2(D, s, z + 2 * i);\n"
                      "        L->u[2 * i] = z[2 * i];\n        L->u[2 * i + 1] = z[2 * i + 1];\n"),
}


def _wjac_pins_pass(orc) -> bool:
    import test_oracle_pins as P
    try:
        for name in ("2d_mixed", "axi_axis", "3d_mixed"):
            P.test_wjac_sweep_is_damped_block_jacobi(orc, name, 0.8)
    except AssertionError:
        return False
    return True


def test_unmutated_oracle_passes_the_wjac_pin(orc):
    assert _wjac_pins_pass(orc)


@pytest.mark.parametrize("name", list(WJAC_MUTATIONS))
def test_wjac_mutant_fails_the_pin(orc, name):
    MUTATIONS[name] = WJAC_MUTATIONS[name]
    try:
        with mutant(orc, name):
            assert not _wjac_pins_pass(orc), name
    finally:
        del MUTATIONS[name]


# Planted mistakes in the refined-patch oracle (composite_oracle.c), against its pins.
COMPOSITE_MUTATIONS = {
    # the interface flux seen from the fine cell over h instead of the 1.5 h to the coarse centre
    "cf_interface_distance": ("sum += cf * (gu - u) / (1.5 * h * h);", "sum += cf * (gu - u) / (h * h);"),
    # the coarse field's tangential slope taken the wrong way
    "cf_tangential_sign": ("return uc + sgn * (up - um) / 8.0;", "return uc - sgn * (up - um) / 8.0;"),
    # the tangential offset taken as half a coarse cell instead of a quarter
    "cf_tangential_offset": ("return uc + sgn * (up - um) / 8.0;", "return uc + sgn * (up - um) / 4.0;"),
    # the base cell's interface flux with the wrong distance: no longer the fine faces' flux
    "cf_reflux_distance": ("sum += (0.5 * H) * cf * (uf - gu) / (1.5 * 0.5 * H) / (H * H);",
                           "sum += (0.5 * H) * cf * (uf - gu) / (0.5 * H) / (H * H);"),
    # the FAC cycle without the base correction's prolongation onto the patch
    "cf_fac_no_prolongation": ("        prolong_to_patch(cg, &P, Ls[0].u, P.u);\n", "\n"),
}


@contextlib.contextmanager
def composite_mutant(name):
    from oracle import composite as cf
    old, new = COMPOSITE_MUTATIONS[name]
    here = os.path.dirname(cf.__file__)
    src = open(os.path.join(here, "composite_oracle.c")).read()
    assert src.count(old) >= 1, name
    d = tempfile.mkdtemp()
    try:
        shutil.copy(os.path.join(here, "coupled_oracle.c"), os.path.join(d, "coupled_oracle.c"))
        path = os.path.join(d, "m.c")
        open(path, "w").write(src.replace(old, new))
        import subprocess
        subprocess.check_call(["gcc", "-std=c99", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-I", d, "-o", os.path.join(d, "m.so"), path, "-lm"])
        lib = cf.configure(C.CDLL(os.path.join(d, "m.so")))
        cf._load()
        saved = cf._lib
        cf._lib = lib
        try:
            yield
        finally:
            cf._lib = saved
    finally:
        shutil.rmtree(d, ignore_errors=True)


def _composite_pins_pass() -> bool:
    import test_oracle_composite as P
    try:
        for axis in (0, 1):
            for box in (((3, 8), (2, 7)), ((0, 6), (3, 9))):
                P.test_linear_fields_have_zero_laplacian(axis, box)
        P.test_conservation_with_walls(((3, 8), (2, 7)))
        P.test_fac_converges_to_the_dense_solution(True, None)
    except (AssertionError, RuntimeError):
        return False
    return True


def test_unmutated_oracle_passes_the_composite_pins():
    assert _composite_pins_pass()


@pytest.mark.parametrize("name", list(COMPOSITE_MUTATIONS))
def test_composite_mutant_fails_a_pin(name):
    with composite_mutant(name):
        assert not _composite_pins_pass(), name
