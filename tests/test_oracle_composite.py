"""Pins of the refined-patch (adaptive grid) oracle, composite_oracle.c (CPU).

The composite operator is checked against what the mathematics fixes:
  - fields linear in x or in y (and bilinear ones away from the domain
    boundary) have zero discrete Laplacian on every valid cell, through the
    coarse-fine interface too (the interface flux is the two-point difference
    between the fine centre and the coarse field at the fine cell's
    tangential position, 1.5 h away);
  - conservation: with walls the cell integrals of the divergence sum to
    zero for any field and coefficients (the base cells' interface fluxes are
    the fine faces' fluxes);
  - a patch covering the whole domain is the uniform fine grid of the
    uniform oracle;
  - FAC converges to the dense solution of the composite system;
  - the discrete solution converges to a continuous one at second order.
test_oracle_mutations.py plants mistakes in it."""
import math

import numpy as np
import pytest

import oracle as orc
from oracle import composite as cf
from paper_2206_11294_gb300 import inputs as I

W, D = I.BC_WALL, I.BC_DIRICHLET


def _g(d):
    return I.Grid(dim=2, axisym=0, n=tuple(d["n"]), h=d["h"], bc=tuple(map(tuple, d["bc"])),
                  bcT=tuple(map(tuple, d["bcT"])), bcp=tuple(map(tuple, d["bcp"])))


def _const_faces(g, c):
    return [np.full(int(np.prod(g.face_shape(a))), c) for a in range(2)]


def _rand_faces(g, rng):
    return [rng.uniform(0.5, 2.0, int(np.prod(g.face_shape(a)))) for a in range(2)]


def _centres(g, origin=(0.0, 0.0)):
    xs = origin[0] + (np.arange(g.n[0]) + 0.5) * g.h
    ys = origin[1] + (np.arange(g.n[1]) + 0.5) * g.h
    return np.meshgrid(xs, ys)


def _covered(base, box):
    cov = np.zeros((base.n[1], base.n[0]), bool)
    cov[box[1][0]: box[1][1], box[0][0]: box[0][1]] = True
    return cov.reshape(-1)


def _lam_part(lam, x):
    return np.stack([lam[:, 0] * x[:, 0] + lam[:, 1] * x[:, 1], lam[:, 2] * x[:, 1]], axis=1)


BOXES = [((3, 8), (2, 7)), ((0, 6), (3, 9)), ((5, 12), (0, 4)), ((0, 12), (0, 10)), ((4, 5), (4, 5))]


@pytest.mark.parametrize("box", BOXES)
@pytest.mark.parametrize("axis", [0, 1])
def test_linear_fields_have_zero_laplacian(axis, box):
    """u = a + b x (or + b y) with Dirichlet sides carrying its values across
    that axis and walls on the other: L(u) is the local terms alone on every
    valid cell (constant coefficients, random l1..l4)."""
    rng = np.random.default_rng(3 + axis)
    H = 0.1
    n = (12, 10, 1)
    L = n[axis] * H
    gT = (1.0, 1.0 + 3.0 * L)
    gp = (2.0, 2.0 - L)
    bc = [[W, W], [W, W], [0, 0]]
    bcT = [[0.0, 0.0], [0.0, 0.0], [0.0, 0.0]]
    bcp = [[0.0, 0.0], [0.0, 0.0], [0.0, 0.0]]
    bc[axis] = [D, D]
    bcT[axis] = list(gT)
    bcp[axis] = list(gp)
    base = I.Grid(dim=2, axisym=0, n=n, h=H, bc=tuple(map(tuple, bc)), bcT=tuple(map(tuple, bcT)),
                  bcp=tuple(map(tuple, bcp)))
    pg = _g(cf.patch_grid(base.as_dict(), box))
    lamb, lamf = rng.standard_normal((base.N, 4)), rng.standard_normal((pg.N, 4))
    ck, ca = 0.7, 1.9
    fkb, fab, fkf, faf = _const_faces(base, ck), _const_faces(base, ca), _const_faces(pg, ck), _const_faces(pg, ca)

    def field(g, origin):
        X = _centres(g, origin)[axis].reshape(-1)
        return np.stack([1.0 + 3.0 * X, 2.0 - X], axis=1)

    xb = field(base, (0.0, 0.0))
    xf = field(pg, (box[0][0] * H, box[1][0] * H))
    yb, yf = cf.apply(base.as_dict(), box, lamb, fab, fkb, lamf, faf, fkf, xb, xf)
    cov = _covered(base, box)
    scale = np.abs(xb).max() * (ck + ca) / (H / 2) ** 2
    if (~cov).any():
        assert np.abs((yb - _lam_part(lamb, xb))[~cov]).max() <= 1e-13 * scale
    assert np.abs(yf - _lam_part(lamf, xf)).max() <= 1e-13 * scale
    assert np.all(yb[cov] == 0.0)


def test_bilinear_field_zero_laplacian_away_from_the_boundary():
    rng = np.random.default_rng(5)
    H = 0.1
    base = I.Grid(dim=2, axisym=0, n=(14, 12, 1), h=H, bc=((W, W), (W, W), (0, 0)))
    box = ((4, 9), (3, 8))
    pg = _g(cf.patch_grid(base.as_dict(), box))
    lz = np.zeros((base.N, 4)), np.zeros((pg.N, 4))
    c = 1.3
    fb, ff = _const_faces(base, c), _const_faces(pg, c)

    def field(g, origin):
        X, Y = _centres(g, origin)
        u = (0.5 + 2.0 * X - 1.5 * Y + 4.0 * X * Y).reshape(-1)
        return np.stack([u, -2.0 * u], axis=1)

    xb, xf = field(base, (0.0, 0.0)), field(pg, (box[0][0] * H, box[1][0] * H))
    yb, yf = cf.apply(base.as_dict(), box, lz[0], fb, fb, lz[1], ff, ff, xb, xf)
    I_, J_ = np.meshgrid(np.arange(base.n[0]), np.arange(base.n[1]))
    inner = ((I_ > 0) & (I_ < base.n[0] - 1) & (J_ > 0) & (J_ < base.n[1] - 1)).reshape(-1) & ~_covered(base, box)
    scale = np.abs(xb).max() * c / (H / 2) ** 2
    assert np.abs(yb[inner]).max() <= 1e-12 * scale
    assert np.abs(yf).max() <= 1e-12 * scale


@pytest.mark.parametrize("box", BOXES)
def test_conservation_with_walls(box):
    """Walls everywhere, random coefficients and field: the cell integrals of
    div(c grad u) over the valid cells sum to zero (every flux, through the
    coarse-fine interface included, is counted once with each sign)."""
    rng = np.random.default_rng(7)
    H = 0.1
    base = I.Grid(dim=2, axisym=0, n=(12, 10, 1), h=H, bc=((W, W), (W, W), (0, 0)))
    pg = _g(cf.patch_grid(base.as_dict(), box))
    fab, fkb, faf, fkf = _rand_faces(base, rng), _rand_faces(base, rng), _rand_faces(pg, rng), _rand_faces(pg, rng)
    xb, xf = rng.standard_normal((base.N, 2)), rng.standard_normal((pg.N, 2))
    yb, yf = cf.apply(base.as_dict(), box, np.zeros((base.N, 4)), fab, fkb, np.zeros((pg.N, 4)), faf, fkf, xb, xf)
    cov = _covered(base, box)
    tot = (yb[~cov] * H * H).sum(axis=0) + (yf * (H / 2) ** 2).sum(axis=0)
    scale = np.abs(yb).max() * H * H + np.abs(yf).max() * H * H
    assert np.all(np.abs(tot) <= 1e-13 * scale * base.N)


def test_full_patch_is_the_uniform_fine_grid():
    """A box covering the whole domain leaves no base cell: the composite
    operator is the uniform oracle's on the fine grid."""
    rng = np.random.default_rng(9)
    base = I.Grid(dim=2, axisym=0, n=(6, 8, 1), h=0.2, bc=((D, W), (W, D), (0, 0)),
                  bcT=((1, 0), (0, 2), (0, 0)), bcp=((3, 0), (0, 4), (0, 0)))
    box = ((0, 6), (0, 8))
    pg = _g(cf.patch_grid(base.as_dict(), box))
    assert pg.bc == base.bc and pg.n == (12, 16, 1)
    lamb, lamf = rng.standard_normal((base.N, 4)), rng.standard_normal((pg.N, 4))
    fab, fkb, faf, fkf = _rand_faces(base, rng), _rand_faces(base, rng), _rand_faces(pg, rng), _rand_faces(pg, rng)
    xf = rng.standard_normal((pg.N, 2))
    yb, yf = cf.apply(base.as_dict(), box, lamb, fab, fkb, lamf, faf, fkf, np.zeros((base.N, 2)), xf)
    ref = orc.apply_paper(pg.as_dict(), lamf, faf, fkf, xf)
    assert np.abs(yf - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.all(yb == 0.0)


@pytest.mark.parametrize("stiff", [False, True])
@pytest.mark.parametrize("box", [None, ((0, 10), (6, 16)), ((4, 12), (0, 16))])
def test_fac_converges_to_the_dense_solution(stiff, box):
    kw = dict(length=6.4e-3, dt=1e-5) if stiff else {}
    b, p, box = I.composite_bubble(16, box=box, seed=11, n_bubbles=1, rmin=0.15, rmax=0.2, **kw)
    gd = b.grid.as_dict()
    xd_b, xd_f = cf.dense_solve(gd, box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b)
    xb, xf, hist = cf.fac_solve(gd, box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b, b.x0, p.x0, 40,
                                coarse_min=2)
    cov = _covered(b.grid, box)
    for f in range(2):
        dev = max(np.abs(xd_f[:, f] - p.x0[:, f]).max(), np.abs(xd_b[~cov, f] - b.x0[~cov, f]).max())
        assert np.abs(xf[:, f] - xd_f[:, f]).max() <= 1e-9 * dev
        assert np.abs(xb[~cov, f] - xd_b[~cov, f]).max() <= 1e-9 * dev
    # covered base cells report the mean of their children
    ch = xd_f.reshape(p.grid.n[1] // 2, 2, p.grid.n[0] // 2, 2, 2).mean(axis=(1, 3)).reshape(-1, 2)
    assert np.allclose(xd_b[cov], ch, rtol=1e-14)


def _continuous(n, box_frac):
    """Constant coefficients, walls, a smooth coupled solution; returns the
    composite problem and the exact values at its cell centres."""
    kT, a_, l1, l2, l3, l4 = 0.8, 1.3, -2.0, 0.3, -1.5, 0.2
    H = 1.0 / n
    base = I.Grid(dim=2, axisym=0, n=(n, n, 1), h=H, bc=((W, W), (W, W), (0, 0)))
    box = tuple((int(box_frac[a][0] * n), int(box_frac[a][1] * n)) for a in range(2))
    pg = _g(cf.patch_grid(base.as_dict(), box))

    def exact(g, origin):
        X, Y = _centres(g, origin)
        T = (np.cos(math.pi * X) * np.cos(math.pi * Y)).reshape(-1)
        p = (np.cos(2 * math.pi * X) * np.cos(math.pi * Y)).reshape(-1)
        lapT, lapp = -2 * math.pi ** 2 * T, -5 * math.pi ** 2 * p
        rhs = np.stack([kT * lapT + l1 * T + l2 * p, a_ * lapp + l3 * p + l4 * kT * lapT], axis=1)
        return np.stack([T, p], axis=1), rhs

    ub, bb = exact(base, (0.0, 0.0))
    uf, bf = exact(pg, (box[0][0] * H, box[1][0] * H))
    lam = lambda N: np.tile([l1, l2, l3, l4], (N, 1))
    return (base, box, pg, lam(base.N), _const_faces(base, a_), _const_faces(base, kT), lam(pg.N),
            _const_faces(pg, a_), _const_faces(pg, kT), bb, bf, ub, uf)


def test_second_order_convergence():
    """Max error at the valid cells' centres against the continuous solution,
    patch over a quarter of the domain off-centre: it falls by ~4 per halving
    of the spacing (fitted order >= 1.8)."""
    errs = []
    for n in (8, 16, 32, 64):
        base, box, pg, lamb, fab, fkb, lamf, faf, fkf, bb, bf, ub, uf = _continuous(n, ((0.25, 0.75), (0.375, 0.875)))
        xb, xf, hist = cf.fac_solve(base.as_dict(), box, lamb, fab, fkb, lamf, faf, fkf, bb, bf,
                                    np.zeros_like(bb), np.zeros_like(bf), 60, coarse_min=2)
        cov = _covered(base, box)
        errs.append(max(np.abs(xb[~cov] - ub[~cov]).max(), np.abs(xf - uf).max()))
    order = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(order >= 1.8), (errs, order)


def test_fac_with_the_patch_in_a_dirichlet_corner():
    """The patch in the corner of two Dirichlet sides: the prolongation's
    stencil reaches across both (odd ghosts in turn); FAC still reaches the
    dense solution."""
    bc = ((D, W), (D, W), (0, 0))
    bcT = ((305.0, 0.0), (295.0, 0.0), (0.0, 0.0))
    bcp = ((1.05e5, 0.0), (0.98e5, 0.0), (0.0, 0.0))
    b, p, box = I.composite_bubble(16, box=((0, 8), (0, 10)), seed=12, n_bubbles=1, rmin=0.1, rmax=0.15,
                                   length=6.4e-3, dt=1e-5, bc=bc, bcT=bcT, bcp=bcp)
    assert p.grid.bc[0][0] == D and p.grid.bc[1][0] == D
    gd = b.grid.as_dict()
    xd_b, xd_f = cf.dense_solve(gd, box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b)
    xb, xf, hist = cf.fac_solve(gd, box, b.lam, b.fa, b.fk, p.lam, p.fa, p.fk, b.b, p.b, b.x0, p.x0, 40,
                                coarse_min=2)
    for f in range(2):
        dev = np.abs(xd_f[:, f] - p.x0[:, f]).max()
        assert np.abs(xf[:, f] - xd_f[:, f]).max() <= 1e-9 * dev
