"""Seeded synthetic inputs for the coupled pressure-temperature solve.

This module holds no solver arithmetic: it only builds the data a caller hands
to the solver, from the paper's own definitions of those data.  Both the CUDA
path (tests, benchmark) and the CPU oracle (tests) consume exactly these arrays.

What it builds, for a cell-centred grid carrying gas bubbles in a liquid:

- the liquid volume fraction C per cell, a tanh profile of the signed distance
  to the union of the bubbles, about two cells wide;
- one-fluid averages  phi_bar = C phi_1 + (1 - C) phi_2  (Sec. 3, the
  one-fluid formulation) of rho c_p, beta, beta/(rho c_p) and of the bracket
  gamma/(rho c^2) - beta^2 T/(rho c_p) of Eq. 8;
- the per-cell coefficients (Eqs. 29-32)
      l1 = -rho c_p / dt,   l2 = beta T / dt,
      l3 = -(gamma/(rho c^2) - beta^2 T/(rho c_p)) / dt^2,
      l4 = beta/(rho c_p) / dt            (1/dt restored, see ``LAMBDA4``);
- the right-hand side (Eqs. 33-34) from provisional fields T_adv, p_adv:
      lambda_T = l1 T_adv + l2 p_adv,   lambda_p = l3 p_adv + div(u*)/dt,
  with div(u*) = 0 and (T_adv, p_adv) a background state plus a manufactured
  sinusoidal pair plus seeded relative N(0, 1e-3) noise;
- face coefficients 1/rho and k from the face volume fraction
  C_f = (C_left + C_right)/2 (the boundary faces take the adjacent cell's C).

Liquid: NASG water (Table 1: Gamma = 1.19, Pi = 7028e5 Pa, b = 6.61e-4 m^3/kg,
c_p = 4285, c_v = 3610); beta from Eq. 10 at (T, p) = (300 K, 1e5 Pa).
Gas: ideal (Gamma = gamma = 1.4, Pi = b = q = 0), so beta = 1/T by Eq. 10.

Arrays use the solver's layouts: cells x-fastest (index i + n0*(j + n1*k));
faces normal to axis a carry n_a + 1 entries along a.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BC_WALL, BC_DIRICHLET, BC_AXIS = 0, 1, 2

# Table 1 (NASG liquid water) and the ideal gas of the paper's test cases.
NASG_WATER = dict(Gamma=1.19, Pi=7028e5, b=6.61e-4, q=-1177788.0, cp=4285.0, cv=3610.0)
AIR = dict(cp=1005.0, cv=717.857142857)            # gamma = 1.4
T_INF, P_INF = 300.0, 1e5

# Eq. 32 as printed lacks the 1/dt that dividing Eq. 19 by dt gives (as Eqs. 31
# and 34 do).  The restored form is the default; the printed one is available.
LAMBDA4 = "restored"


def nasg_beta(T: float, p: float, Gamma: float, Pi: float, b: float, cv: float, **_) -> float:
    """Thermal dilation coefficient, Eq. 10."""
    return (Gamma - 1.0) * cv / ((Gamma - 1.0) * cv * T + b * (p + Pi))


@dataclasses.dataclass
class Phase:
    rho: float
    k: float
    rho_c2: float     # rho c^2
    cp: float
    cv: float
    beta: float

    @property
    def gamma(self) -> float:
        return self.cp / self.cv


def liquid(rho=1000.0, k=0.6, rho_c2=2.2e9) -> Phase:
    w = NASG_WATER
    return Phase(rho=rho, k=k, rho_c2=rho_c2, cp=w["cp"], cv=w["cv"],
                 beta=nasg_beta(T_INF, P_INF, **w))


def gas(rho=1.2, k=0.026, rho_c2=1.4e5) -> Phase:
    return Phase(rho=rho, k=k, rho_c2=rho_c2, cp=AIR["cp"], cv=AIR["cv"], beta=1.0 / T_INF)


@dataclasses.dataclass
class Grid:
    dim: int
    axisym: int
    n: Tuple[int, int, int]
    h: float
    r0: float = 0.0
    origin: Tuple[float, float, float] = (0.0, 0.0, 0.0)
    bc: Tuple[Tuple[int, int], ...] = ((0, 0), (0, 0), (0, 0))
    bcT: Tuple[Tuple[float, float], ...] = ((0.0, 0.0),) * 3
    bcp: Tuple[Tuple[float, float], ...] = ((0.0, 0.0),) * 3

    @property
    def N(self) -> int:
        return self.n[0] * self.n[1] * self.n[2]

    def as_dict(self) -> dict:
        return dict(dim=self.dim, axisym=self.axisym, n=list(self.n), h=self.h, r0=self.r0,
                    bc=[list(s) for s in self.bc], bcT=[list(s) for s in self.bcT],
                    bcp=[list(s) for s in self.bcp])

    def face_shape(self, a: int) -> Tuple[int, int, int]:
        """numpy shape (n2, n1, n0) with n_a + 1 along axis a."""
        s = [self.n[2], self.n[1], self.n[0]]
        s[2 - a] += 1
        return tuple(s)


@dataclasses.dataclass
class Problem:
    name: str
    grid: Grid
    lam: np.ndarray               # N x 4: l1..l4
    fa: List[np.ndarray]          # per axis (dim of them), 1/rho on faces
    fk: List[np.ndarray]          # per axis, k on faces
    b: np.ndarray                 # N x 2: (lambda_T, lambda_p)
    x0: np.ndarray                # N x 2: initial guess (T, p)
    meta: dict = dataclasses.field(default_factory=dict)


def _centres(g: Grid):
    """Cell-centre coordinates as (n2, n1, n0) arrays, one per axis."""
    ax = [g.origin[a] + (np.arange(g.n[a]) + 0.5) * g.h for a in range(3)]
    if g.axisym:
        ax[0] = g.r0 + (np.arange(g.n[0]) + 0.5) * g.h
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return [X, Y, Z]


def volume_fraction(g: Grid, centres: Sequence[Sequence[float]], radii: Sequence[float]) -> np.ndarray:
    """Liquid fraction C = (1 + tanh(d/h))/2, d = signed distance to the bubbles' union."""
    X = _centres(g)
    d = np.full(X[0].shape, np.inf)
    for c, R in zip(centres, radii):
        r2 = sum((X[a] - c[a]) ** 2 for a in range(g.dim))
        d = np.minimum(d, np.sqrt(r2) - R)
    return 0.5 * (1.0 + np.tanh(d / g.h))


def _face_C(Cc: np.ndarray, a: int) -> np.ndarray:
    ax = 2 - a
    pad = [(0, 0)] * 3
    pad[ax] = (1, 1)
    P = np.pad(Cc, pad, mode="edge")
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[ax] = slice(0, -1)
    hi[ax] = slice(1, None)
    return 0.5 * (P[tuple(lo)] + P[tuple(hi)])


def _mode(g: Grid, X) -> np.ndarray:
    """Manufactured shape: per axis cos for wall/axis pairs, sin for Dirichlet
    pairs, quarter waves for mixed pairs."""
    phi = np.ones(X[0].shape)
    for a in range(g.dim):
        lo, hi = g.bc[a]
        L = g.n[a] * g.h
        o = g.r0 if (g.axisym and a == 0) else g.origin[a]
        xi = (X[a] - o) / L
        dlo, dhi = lo == BC_DIRICHLET, hi == BC_DIRICHLET
        if not dlo and not dhi:
            phi = phi * np.cos(math.pi * xi)
        elif dlo and dhi:
            phi = phi * np.sin(math.pi * xi)
        elif dhi:
            phi = phi * np.cos(0.5 * math.pi * xi)
        else:
            phi = phi * np.sin(0.5 * math.pi * xi)
    return phi


def assemble(name: str, g: Grid, Cc: np.ndarray, liq: Phase, gs: Phase, dt: float,
             rng: np.random.Generator, a_T: float = 10.0, a_p: float = 1e3,
             lambda4: str = LAMBDA4) -> Problem:
    """Per-cell lambdas (Eqs. 29-32), RHS (Eqs. 33-34) and face coefficients."""
    X = _centres(g)
    T_adv_bg = T_INF
    # one-fluid averages (Sec. 3)
    avg = lambda f1, f2: Cc * f1 + (1.0 - Cc) * f2
    rho_cp = avg(liq.rho * liq.cp, gs.rho * gs.cp)
    beta = avg(liq.beta, gs.beta)
    b_over = avg(liq.beta / (liq.rho * liq.cp), gs.beta / (gs.rho * gs.cp))
    bracket = avg(liq.gamma / liq.rho_c2 - liq.beta ** 2 * T_adv_bg / (liq.rho * liq.cp),
                  gs.gamma / gs.rho_c2 - gs.beta ** 2 * T_adv_bg / (gs.rho * gs.cp))
    assert np.all(bracket > 0.0)
    phi = _mode(g, X)
    T_adv = (T_INF + a_T * phi) * (1.0 + 1e-3 * rng.standard_normal(phi.shape))
    p_adv = (P_INF + a_p * phi) * (1.0 + 1e-3 * rng.standard_normal(phi.shape))
    l1 = -rho_cp / dt                                     # Eq. 29
    l2 = beta * T_adv / dt                                # Eq. 30
    l3 = -bracket / dt ** 2                               # Eq. 31
    l4 = b_over / dt if lambda4 == "restored" else b_over  # Eq. 32
    lam_T = l1 * T_adv + l2 * p_adv                       # Eq. 33
    lam_p = l3 * p_adv + 0.0                              # Eq. 34, div(u*) = 0
    lam = np.stack([l1, l2, l3, l4], axis=-1).reshape(-1, 4)
    b = np.stack([lam_T, lam_p], axis=-1).reshape(-1, 2)
    x0 = np.empty_like(b)
    x0[:, 0] = T_INF
    x0[:, 1] = P_INF
    fa, fk = [], []
    for a in range(g.dim):
        Cf = _face_C(Cc, a)
        fa.append((1.0 / (Cf * liq.rho + (1.0 - Cf) * gs.rho)).reshape(-1))
        fk.append((Cf * liq.k + (1.0 - Cf) * gs.k).reshape(-1))
    return Problem(name=name, grid=g, lam=np.ascontiguousarray(lam), fa=fa, fk=fk,
                   b=np.ascontiguousarray(b), x0=x0, meta=dict(dt=dt))


def _walls(dim: int, axisym: int = 0):
    bc = [[BC_WALL, BC_WALL] for _ in range(3)]
    if axisym:
        bc[0][0] = BC_AXIS
    return tuple(tuple(s) for s in bc)


def _place_bubbles(rng: np.random.Generator, count: int, rmin: float, rmax: float, dim: int,
                   L: Sequence[float], max_tries: int = 10000):
    """Uniform centres, non-overlapping, at least R from every wall."""
    centres, radii = [], []
    tries = 0
    while len(centres) < count and tries < max_tries:
        tries += 1
        R = rng.uniform(rmin, rmax)
        c = [rng.uniform(R, L[a] - R) for a in range(dim)]
        if all(math.dist(c, c2) > R + R2 for c2, R2 in zip(centres, radii)):
            centres.append(c)
            radii.append(R)
    return centres, radii


def bubble_2d(n: int = 64, seed: int = 1, n_bubbles: int = 1, rmin: float = 0.25, rmax: float = 0.25,
              centred: bool = True, length: float = 1.0, dt: float = 1e-7, gas_rho: float = 1.2,
              ny: Optional[int] = None, name: str = "") -> Problem:
    """2D square (or n x ny) domain of side ``length``, walls on every side."""
    rng = np.random.default_rng(seed)
    ny = ny or n
    h = length / n
    g = Grid(dim=2, axisym=0, n=(n, ny, 1), h=h, bc=_walls(2))
    Ls = (n * h, ny * h)
    if centred and n_bubbles == 1:
        centres, radii = [[0.5 * Ls[0], 0.5 * Ls[1]]], [rmin * length]
    else:
        centres, radii = _place_bubbles(rng, n_bubbles, rmin * length, rmax * length, 2, Ls)
    Cc = volume_fraction(g, centres, radii)
    p = assemble(name or f"bubble2d_{n}x{ny}", g, Cc, liquid(), gas(rho=gas_rho), dt, rng)
    p.meta.update(centres=centres, radii=radii, seed=seed)
    return p


def bubble_axi(nr: int = 512, nz: int = 1024, seed: int = 3, R: float = 0.2, length: float = 1.0,
               dt: float = 1e-7, name: str = "") -> Problem:
    """Axisymmetric (r, z) grid, r in [0, length/2], z in [0, length], one bubble
    on the axis at mid-height; symmetry axis at r = 0, walls elsewhere."""
    rng = np.random.default_rng(seed)
    h = length / nz
    g = Grid(dim=2, axisym=1, n=(nr, nz, 1), h=h, r0=0.0, bc=_walls(2, axisym=1))
    Cc = volume_fraction(g, [[0.0, 0.5 * nz * h]], [R * length])
    p = assemble(name or f"axi_{nr}x{nz}", g, Cc, liquid(), gas(), dt, rng)
    p.meta.update(seed=seed)
    return p


def bubble_wall_3d(n: int = 256, seed: int = 4, R: float = 0.15, standoff: float = 0.2,
                   length: float = 1.0, dt: float = 1e-7, name: str = "") -> Problem:
    """3D cube: bubble of radius R centred ``standoff`` above a rigid wall at
    z = 0; the other five faces hold p = 1e5 Pa, T = 300 K (Dirichlet)."""
    rng = np.random.default_rng(seed)
    h = length / n
    D = BC_DIRICHLET
    bc = ((D, D), (D, D), (BC_WALL, D))
    vals_T = ((T_INF, T_INF),) * 3
    vals_p = ((P_INF, P_INF),) * 3
    g = Grid(dim=3, axisym=0, n=(n, n, n), h=h, bc=bc, bcT=vals_T, bcp=vals_p)
    c = [0.5 * length, 0.5 * length, standoff * length]
    Cc = volume_fraction(g, [c], [R * length])
    p = assemble(name or f"wall3d_{n}", g, Cc, liquid(), gas(), dt, rng)
    p.meta.update(seed=seed)
    return p


def stiff(p_fn, *args, length: float = 6.4e-3, dt: float = 1e-5, **kw) -> Problem:
    """Same geometry at the paper's bubble scale (domain 64 R0 with R0 = 0.1 mm)
    and a longer step, where the Laplacians dominate the p-row and the coarse
    levels carry the convergence.  Test-only workload."""
    return p_fn(*args, length=length, dt=dt, **kw)


def round_to(v: float, m: int) -> int:
    return max(m, int(round(v / m)) * m)


def batch_sizes(count: int = 256, seed: int = 5, lo: int = 64, hi: int = 1024, multiple: int = 32):
    """Log-uniform sizes in [lo, hi], rounded to a multiple (32: every size then
    coarsens to at most 31 x 31 cells, 1922 unknowns of the exact coarsest
    solve)."""
    rng = np.random.default_rng(seed)
    return [min(hi, round_to(math.exp(rng.uniform(math.log(lo), math.log(hi))), multiple))
            for _ in range(count)]


def batch_problems(count: int = 256, seed: int = 5, lo: int = 64, hi: int = 1024,
                   sizes: Optional[Sequence[int]] = None) -> List[Problem]:
    """Independent 2D problems, 1-8 bubbles each, density ratio exactly 1000."""
    rng = np.random.default_rng(seed)
    sizes = list(sizes) if sizes is not None else batch_sizes(count, seed, lo, hi)
    out = []
    for q, n in enumerate(sizes):
        nb = int(rng.integers(1, 9))
        out.append(bubble_2d(n=n, seed=int(rng.integers(1 << 30)), n_bubbles=nb, rmin=0.02,
                             rmax=0.08, centred=False, gas_rho=1.0, name=f"batch{q}_{n}"))
    return out


def bubbles_1024(n: int = 1024, seed: int = 2, length: float = 1.0, dt: float = 1e-7) -> Problem:
    """2D n x n grid with 16 seeded bubbles, radii uniform in [0.02, 0.08] of the domain."""
    return bubble_2d(n=n, seed=seed, n_bubbles=16, rmin=0.02, rmax=0.08, centred=False, length=length, dt=dt,
                     name=f"bubbles16_{n}x{n}")


def composite_bubble(n: int = 64, box=None, seed: int = 9, n_bubbles: int = 2, rmin: float = 0.06,
                     rmax: float = 0.12, length: float = 1.0, dt: float = 1e-7, bc=None, bcT=None, bcp=None,
                     name: str = "", centres=None, radii=None):
    """A refined-patch (adaptive) grid around bubbles: (base, patch, box).

    base: the n x n grid of spacing length / n over the whole domain, its
    coefficients and right-hand side assembled at that spacing; box = ((i0,
    i1), (j0, j1)) the base cells refined 2:1 (by default the bubbles'
    bounding box, one base cell wider); patch: the fine cells of the box,
    cut from the same field assembled on the 2n x 2n grid of the whole domain
    (its grid's origin at the box's corner).  The bubbles stay inside the box,
    so the base cells outside it are pure liquid, as on a grid coarsened away
    from the bubble.  centres, radii (fractions of the domain): given bubbles
    instead of seeded ones."""
    rng = np.random.default_rng(seed)
    bc = bc or _walls(2)
    bcT = bcT or ((0.0, 0.0),) * 3
    bcp = bcp or ((0.0, 0.0),) * 3
    H = length / n
    gb = Grid(dim=2, axisym=0, n=(n, n, 1), h=H, bc=bc, bcT=bcT, bcp=bcp)
    gf = Grid(dim=2, axisym=0, n=(2 * n, 2 * n, 1), h=H / 2, bc=bc, bcT=bcT, bcp=bcp)
    if centres is None:
        centres, radii = _place_bubbles(rng, n_bubbles, rmin * length, rmax * length, 2, (length, length))
    else:
        centres = [[c[0] * length, c[1] * length] for c in centres]
        radii = [r * length for r in radii]
    if box is None:
        lo = [min(c[a] - r for c, r in zip(centres, radii)) for a in range(2)]
        hi = [max(c[a] + r for c, r in zip(centres, radii)) for a in range(2)]
        box = tuple((max(0, int(math.floor(lo[a] / H)) - 1), min(n, int(math.ceil(hi[a] / H)) + 1)) for a in range(2))
    base = assemble(name or f"composite_base_{n}", gb, volume_fraction(gb, centres, radii), liquid(), gas(), dt, rng)
    full = assemble(f"composite_fine_{2 * n}", gf, volume_fraction(gf, centres, radii), liquid(), gas(), dt, rng)
    (i0, i1), (j0, j1) = box
    m0, m1 = 2 * (i1 - i0), 2 * (j1 - j0)
    pbc = [list(s) for s in bc]
    pT = [list(s) for s in bcT]
    pP = [list(s) for s in bcp]
    for a, (lo_, hi_) in enumerate(box):
        if lo_ > 0:
            pbc[a][0], pT[a][0], pP[a][0] = BC_WALL, 0.0, 0.0
        if hi_ < n:
            pbc[a][1], pT[a][1], pP[a][1] = BC_WALL, 0.0, 0.0
    gp = Grid(dim=2, axisym=0, n=(m0, m1, 1), h=H / 2, origin=(i0 * H, j0 * H, 0.0),
              bc=tuple(map(tuple, pbc)), bcT=tuple(map(tuple, pT)), bcp=tuple(map(tuple, pP)))
    cells = lambda arr, k: arr.reshape(2 * n, 2 * n, k)[2 * j0: 2 * j1, 2 * i0: 2 * i1].reshape(-1, k)
    fa = [full.fa[0].reshape(2 * n, 2 * n + 1)[2 * j0: 2 * j1, 2 * i0: 2 * i1 + 1].reshape(-1),
          full.fa[1].reshape(2 * n + 1, 2 * n)[2 * j0: 2 * j1 + 1, 2 * i0: 2 * i1].reshape(-1)]
    fk = [full.fk[0].reshape(2 * n, 2 * n + 1)[2 * j0: 2 * j1, 2 * i0: 2 * i1 + 1].reshape(-1),
          full.fk[1].reshape(2 * n + 1, 2 * n)[2 * j0: 2 * j1 + 1, 2 * i0: 2 * i1].reshape(-1)]
    patch = Problem(name=f"composite_patch_{m0}x{m1}", grid=gp, lam=np.ascontiguousarray(cells(full.lam, 4)),
                    fa=[np.ascontiguousarray(f) for f in fa], fk=[np.ascontiguousarray(f) for f in fk],
                    b=np.ascontiguousarray(cells(full.b, 2)), x0=np.ascontiguousarray(cells(full.x0, 2)),
                    meta=dict(dt=dt))
    return base, patch, box


def random_coeff_problem(g: Grid, seed: int, jump: float = 1000.0, dt: float = 1e-7,
                         couple: bool = True) -> Problem:
    """Small problem with random bubble placement on an arbitrary grid (tests)."""
    rng = np.random.default_rng(seed)
    L = [g.n[a] * g.h for a in range(g.dim)]
    X0 = [g.origin[a] for a in range(g.dim)]
    if g.axisym:
        X0[0] = g.r0
    c = [X0[a] + rng.uniform(0.3, 0.7) * L[a] for a in range(g.dim)]
    R = 0.25 * min(L)
    Cc = volume_fraction(g, [c], [R])
    p = assemble(f"random{seed}", g, Cc, liquid(), gas(rho=1000.0 / jump), dt, rng)
    if not couple:
        p.lam[:, 1] = 0.0
        p.lam[:, 3] = 0.0
    # random initial guess around the background
    p.x0 = p.x0 * (1.0 + 1e-3 * rng.standard_normal(p.x0.shape))
    return p


# ---------------------------------------------------------------------------
# Advected state of one time step (the input of the coefficient assembly).
# The fields are built from chosen temperature, pressure and velocity fields
# through the NASG equations of state: the phase density from the thermal
# relation rho_i (c_p,i - c_v,i) T = (p + Pi_i)(1 - rho_i b_i) (the one-phase
# form of Eq. 23) and the internal energy from Eq. 9.  Liquid water of Table 1
# and air as an ideal gas (Gamma = gamma = 1.4, Pi = b = q = 0, Sec. 2).
# ---------------------------------------------------------------------------
NASG_AIR = dict(Gamma=1.4, Pi=0.0, b=0.0, q=0.0, cp=1005.0, cv=717.857142857)


@dataclasses.dataclass
class NasgPhase:
    Gamma: float
    Pi: float
    b: float
    q: float
    cp: float
    cv: float
    k: float
    mu: float = 0.0               # dynamic viscosity (Eq. 3), for the energy update of Eq. 39


def water_phase(k: float = 0.6, mu: float = 8.5e-4) -> NasgPhase:
    return NasgPhase(k=k, mu=mu, **NASG_WATER)


def air_phase(k: float = 0.026, mu: float = 1.85e-5) -> NasgPhase:
    return NasgPhase(k=k, mu=mu, **NASG_AIR)


@dataclasses.dataclass
class AdvectedState:
    name: str
    grid: Grid
    ph1: NasgPhase                # phase 1 (C = 1), the liquid
    ph2: NasgPhase
    dt: float
    C: np.ndarray                 # (n2, n1, n0) volume fraction of phase 1
    m1: np.ndarray                # C rho_1
    m2: np.ndarray                # (1 - C) rho_2
    E: np.ndarray                 # averaged total energy per volume
    mom: List[np.ndarray]         # averaged momentum per axis
    uf: List[np.ndarray]          # face-normal velocity u* per axis, shape grid.face_shape(a)
    kappa: np.ndarray             # interface curvature (for Eqs. 37-38)
    sigma: float
    T: np.ndarray                 # the fields the state was built from
    p: np.ndarray


def phase_density(T, p, ph: NasgPhase):
    """rho from rho (c_p - c_v) T = (p + Pi)(1 - rho b)."""
    return (p + ph.Pi) / ((ph.cp - ph.cv) * T + ph.b * (p + ph.Pi))


def phase_energy(p, rho, ph: NasgPhase):
    """rho e from Eq. 9."""
    return (p + ph.Gamma * ph.Pi) / (ph.Gamma - 1.0) * (1.0 - rho * ph.b) + rho * ph.q


def advected_state(g: Grid, Cc: np.ndarray, seed: int, dt: float = 1e-7, dT: float = 4.0, dp: float = 3e3,
                   u0: float = 0.5, sigma: float = 0.072, name: str = "") -> AdvectedState:
    """Smooth seeded T, p, velocity fields (a few modes plus 1e-3 noise) on a
    volume-fraction field; face velocities u* are the cell velocity's face means
    plus noise, zero on walls and the axis."""
    rng = np.random.default_rng(seed)
    shape = (g.n[2], g.n[1], g.n[0])
    X = [(np.arange(g.n[a], dtype=np.float64) + 0.5) / g.n[a] for a in range(3)]
    grid3 = np.meshgrid(X[2], X[1], X[0], indexing="ij")
    xs = [grid3[2], grid3[1], grid3[0]]

    def smooth(amp: float) -> np.ndarray:
        f = np.zeros(shape)
        for _ in range(3):
            k = rng.integers(1, 4, size=3)
            ph = rng.uniform(0, 2 * np.pi, size=3)
            term = np.ones(shape)
            for a in range(g.dim):
                term = term * np.cos(np.pi * k[a] * xs[a] + ph[a])
            f = f + term * rng.uniform(0.3, 1.0)
        return amp * f / 3.0 * (1.0 + 1e-3 * rng.standard_normal(shape))

    T = T_INF + smooth(dT)
    p = P_INF + smooth(dp)
    u = [smooth(u0) for _ in range(g.dim)]
    ph1, ph2 = water_phase(), air_phase()
    C = np.clip(np.asarray(Cc, dtype=np.float64).reshape(shape), 0.0, 1.0)
    r1, r2 = phase_density(T, p, ph1), phase_density(T, p, ph2)
    m1, m2 = C * r1, (1.0 - C) * r2
    rho = m1 + m2
    E = C * phase_energy(p, r1, ph1) + (1.0 - C) * phase_energy(p, r2, ph2) + 0.5 * rho * sum(v * v for v in u)
    mom = [rho * v for v in u]
    uf = []
    for a in range(g.dim):
        fs = list(shape)
        fs[2 - a] += 1
        f = np.zeros(fs)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[2 - a] = slice(0, -1)
        hi[2 - a] = slice(1, None)
        inner = [slice(None)] * 3
        inner[2 - a] = slice(1, -1)
        f[tuple(inner)] = 0.5 * (u[a][tuple(lo)] + u[a][tuple(hi)])
        f = f + 1e-3 * u0 * rng.standard_normal(fs)
        for side in (0, 1):
            if g.bc[a][side] != BC_DIRICHLET:
                edge = [slice(None)] * 3
                edge[2 - a] = slice(0, 1) if side == 0 else slice(-1, None)
                f[tuple(edge)] = 0.0
        uf.append(f)
    kappa = rng.uniform(-50.0, 50.0, size=shape)
    return AdvectedState(name=name or f"state{seed}", grid=g, ph1=ph1, ph2=ph2, dt=dt, C=C, m1=m1, m2=m2, E=E,
                         mom=mom, uf=uf, kappa=kappa, sigma=sigma, T=T, p=p)


def bubbles_state_1024(n: int = 1024, seed: int = 2) -> AdvectedState:
    """The advected state on the 16-bubble 1024^2 grid of bubbles_1024."""
    g = Grid(dim=2, axisym=0, n=(n, n, 1), h=1.0 / n, bc=_walls(2))
    rng = np.random.default_rng(seed)
    centres, radii = _place_bubbles(rng, 16, 0.02, 0.08, 2, (1.0, 1.0))
    Cc = volume_fraction(g, centres, radii)
    return advected_state(g, Cc, seed + 100, name=f"bubbles16_{n}x{n}_state")
