"""Pins of the assembly / correction oracle (oracle/assembly.py) against what
the paper and thermodynamics fix, independent of the oracle's own formulas:

- round trip: p and T built from chosen fields through Eq. 9 and the thermal
  relation are recovered by Eqs. 20 and 23 (pure and mixed cells, moving fluid);
- Eq. 10 at Table 1's water, 300 K, 1e5 Pa (hand-evaluated golden value), and
  against a finite difference of the density at constant pressure;
- Eq. 11 against the isentropic derivative of Eq. 9 by finite differences;
- the bracket of Eq. 8 equals the isentropic compressibility 1/(rho c^2) for a
  thermodynamically consistent phase (c_p = Gamma c_v), so lambda_3 of a pure
  cell is -1/(rho c^2 dt^2);
- mixed cells at fixed (p, T): every lambda is the volume-fraction average of
  the two pure-phase values;
- lambda_T and lambda_p rearrange Eqs. 18-19 (divided by dt);
- the discrete divergence is exact on linear velocity fields (Cartesian and
  axisymmetric);
- after the correction, div u^{n+1} = div u* - dt L_alpha p with L_alpha built by
  the independent sparse assembly of tests/fv_matrix.py; Eqs. 37-38 average back
  to p and differ by sigma kappa.
"""
import json
import os

import numpy as np
import pytest

from oracle import assembly as A
from paper_2206_11294_gb300 import inputs as I

from fv_matrix import laplacian

HERE = os.path.dirname(os.path.abspath(__file__))
W, D, AX = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS


def _state(grid, seed=7, **kw):
    X = I._centres(grid)
    c = [X[a].mean() for a in range(grid.dim)]
    R = 0.3 * min(grid.n[a] * grid.h for a in range(grid.dim))
    Cc = I.volume_fraction(grid, [c], [R])
    return I.advected_state(grid, Cc, seed, **kw)


GRIDS = {
    "2d": I.Grid(dim=2, axisym=0, n=(40, 24, 1), h=1e-3, bc=((W, W), (W, W), (0, 0))),
    "2d_dir": I.Grid(dim=2, axisym=0, n=(32, 20, 1), h=1e-3, bc=((D, W), (W, D), (0, 0)),
                     bcT=((300.0, 0.0), (0.0, 305.0), (0, 0)), bcp=((1.02e5, 0.0), (0.0, 0.99e5), (0, 0))),
    "axi": I.Grid(dim=2, axisym=1, n=(24, 40, 1), h=1e-3, r0=0.0, bc=((AX, W), (W, D), (0, 0)),
                  bcp=((0, 0), (0.0, 1.01e5), (0, 0))),
    "3d": I.Grid(dim=3, axisym=0, n=(12, 10, 8), h=1e-3, bc=((W, D), (W, W), (D, W)),
                 bcp=((0.0, 1e5), (0, 0), (1.01e5, 0.0))),
}


@pytest.mark.parametrize("name", list(GRIDS))
def test_round_trip_p_T(name):
    g = GRIDS[name]
    s = _state(g)
    p, T = A.mixture_pT(s.C, s.m1, s.m2, s.E, s.mom, s.ph1, s.ph2)
    # p is a difference of terms of order Gamma Pi / (Gamma - 1) ~ 4e9 J/m^3: a few ulps of those
    scale = s.ph1.Gamma * s.ph1.Pi / (s.ph1.Gamma - 1.0)
    assert np.max(np.abs(p - s.p)) <= 64 * np.finfo(float).eps * scale
    np.testing.assert_allclose(T, s.T, rtol=1e-12, atol=0)
    # pure cells of either phase
    for Cv in (0.0, 1.0):
        C = np.full_like(s.C, Cv)
        r1, r2 = I.phase_density(s.T, s.p, s.ph1), I.phase_density(s.T, s.p, s.ph2)
        m1, m2 = C * r1, (1 - C) * r2
        E = C * I.phase_energy(s.p, r1, s.ph1) + (1 - C) * I.phase_energy(s.p, r2, s.ph2)
        p2, T2 = A.mixture_pT(C, m1, m2, E, [np.zeros_like(C)] * g.dim, s.ph1, s.ph2)
        assert np.max(np.abs(p2 - s.p)) <= 64 * np.finfo(float).eps * (scale if Cv else 2.5 * s.p.max())
        np.testing.assert_allclose(T2, s.T, rtol=1e-12, atol=0)


def test_eq10_golden_water():
    with open(os.path.join(HERE, "golden", "nasg_water_table1.json")) as f:
        gold = json.load(f)
    w = gold["table1"]
    b = A.phase_beta(300.0, 1e5, dict(w))
    assert abs(b - gold["beta_300K_1e5Pa"]) <= 1e-12 * gold["beta_300K_1e5Pa"]


def _consistent(Gamma=1.19, Pi=7028e5, b=6.61e-4, q=-1177788.0, cv=3610.0, k=0.6):
    return I.NasgPhase(Gamma=Gamma, Pi=Pi, b=b, q=q, cp=Gamma * cv, cv=cv, k=k)


@pytest.mark.parametrize("ph", [_consistent(), _consistent(Gamma=1.4, Pi=0.0, b=0.0, q=0.0, cv=717.86, k=0.026)])
@pytest.mark.parametrize("T,p", [(300.0, 1e5), (350.0, 3e6), (290.0, 5e4)])
def test_eq10_finite_difference(ph, T, p):
    """beta = -(1/rho) (d rho / d T)_p of the thermal relation, by central differences."""
    dT = 1e-5 * T
    rho = I.phase_density(T, p, ph)
    fd = -(I.phase_density(T + dT, p, ph) - I.phase_density(T - dT, p, ph)) / (2 * dT) / rho
    assert abs(A.phase_beta(T, p, ph) - fd) <= 1e-8 * abs(fd)


@pytest.mark.parametrize("ph", [I.water_phase(), I.air_phase()])
@pytest.mark.parametrize("T,p", [(300.0, 1e5), (400.0, 2e6)])
def test_eq11_isentropic_derivative(ph, T, p):
    """c^2 = (dp/drho)_s = (p/rho^2 - (de/drho)_p) / (de/dp)_rho for e of Eq. 9."""
    rho = I.phase_density(T, p, ph)
    e = lambda pp, rr: I.phase_energy(pp, rr, ph) / rr
    dr, dp = 1e-5 * rho, 1e-5 * (p + ph.Pi)
    de_dr = (e(p, rho + dr) - e(p, rho - dr)) / (2 * dr)
    de_dp = (e(p + dp, rho) - e(p - dp, rho)) / (2 * dp)
    c2 = (p / rho ** 2 - de_dr) / de_dp
    assert abs(A.phase_c2(p, rho, ph) - c2) <= 1e-6 * c2


def _uniform_state(g, C, T=310.0, p=2e5, ph1=None, ph2=None):
    ph1 = ph1 or I.water_phase()
    ph2 = ph2 or I.air_phase()
    shape = (g.n[2], g.n[1], g.n[0])
    C = np.full(shape, C)
    Tf, pf = np.full(shape, T), np.full(shape, p)
    r1, r2 = I.phase_density(Tf, pf, ph1), I.phase_density(Tf, pf, ph2)
    m1, m2 = C * r1, (1 - C) * r2
    E = C * I.phase_energy(pf, r1, ph1) + (1 - C) * I.phase_energy(pf, r2, ph2)
    uf = [np.zeros(g.face_shape(a)) for a in range(g.dim)]
    return ph1, ph2, C, m1, m2, E, [np.zeros(shape)] * g.dim, uf


def test_pure_consistent_phase_lambda3_is_isentropic():
    g = GRIDS["2d"]
    ph = _consistent()
    dt = 1e-6
    ph1, ph2, C, m1, m2, E, mom, uf = _uniform_state(g, 1.0, ph1=ph, ph2=I.air_phase())
    out = A.assemble(g, ph1, ph2, dt, C, m1, m2, E, mom, uf)
    T, p = out["T"].reshape(-1), out["p"].reshape(-1)
    rho = I.phase_density(T, p, ph)
    # isentropic compressibility from the finite-difference sound speed of Eq. 9 (independent of Eq. 11)
    e = lambda pp, rr: I.phase_energy(pp, rr, ph) / rr
    dr, dp = 1e-5 * rho, 1e-5 * (p + ph.Pi)
    c2 = (p / rho ** 2 - (e(p, rho + dr) - e(p, rho - dr)) / (2 * dr)) / ((e(p + dp, rho) - e(p - dp, rho)) / (2 * dp))
    np.testing.assert_allclose(out["lam"][:, 2], -1.0 / (rho * c2 * dt * dt), rtol=1e-6)
    np.testing.assert_allclose(out["lam"][:, 0], -rho * ph.cp / dt, rtol=1e-13)
    # beta read back from lambda_2 = beta T / dt against the finite-difference dilation of the thermal relation
    dT = 1e-5 * T
    beta_fd = -(I.phase_density(T + dT, p, ph) - I.phase_density(T - dT, p, ph)) / (2 * dT) / rho
    np.testing.assert_allclose(out["lam"][:, 1] * dt / T, beta_fd, rtol=1e-8)
    # one phase: beta / (rho c_p) = -lambda_2 / (lambda_1 T); lambda_4 carries the restored 1/dt
    l1, l2, l4 = out["lam"][:, 0], out["lam"][:, 1], out["lam"][:, 3]
    np.testing.assert_allclose(l4, -l2 / (l1 * T * dt), rtol=1e-13)
    printed = A.assemble(g, ph1, ph2, dt, C, m1, m2, E, mom, uf, lambda4="printed")
    np.testing.assert_allclose(printed["lam"][:, 3], -l2 / (l1 * T), rtol=1e-13)


@pytest.mark.parametrize("Cmix", [0.25, 0.5, 0.9])
def test_mixed_cells_average_pure_values(Cmix):
    g = GRIDS["2d"]
    dt = 1e-7
    res = {}
    for Cv in (0.0, 1.0, Cmix):
        ph1, ph2, C, m1, m2, E, mom, uf = _uniform_state(g, Cv)
        res[Cv] = A.assemble(g, ph1, ph2, dt, C, m1, m2, E, mom, uf)
    mix = Cmix * res[1.0]["lam"] + (1 - Cmix) * res[0.0]["lam"]
    # the bracket of lambda_3 cancels two terms of similar size: rounding grows to ~1e-12
    np.testing.assert_allclose(res[Cmix]["lam"], mix, rtol=1e-10)
    np.testing.assert_allclose(res[Cmix]["b"], Cmix * res[1.0]["b"] + (1 - Cmix) * res[0.0]["b"], rtol=1e-10)


@pytest.mark.parametrize("name", ["2d", "axi", "3d"])
def test_lambda_T_p_rearrange_eqs_18_19(name):
    """With LT = div(k grad T), Lp = div((1/rho) grad p) and D = div u* as free
    numbers, L(x) - b of Eqs. 27-28 equals minus Eq. 18 and minus Eq. 19 / dt."""
    g = GRIDS[name]
    s = _state(g, seed=11)
    out = A.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    rng = np.random.default_rng(3)
    N = g.N
    Tn = out["x0"][:, 0] + rng.normal(0, 2.0, N)
    pn = out["x0"][:, 1] + rng.normal(0, 500.0, N)
    LT = rng.normal(0, 1e6, N)
    Lp = rng.normal(0, 1e8, N)
    l1, l2, l3, l4 = out["lam"].T
    lT, lp = out["b"].T
    Ta, pa = out["x0"].T
    dt = s.dt
    Dv = out["div"].reshape(-1)
    # mixture coefficients read back from lambda_1..lambda_4 (Eqs. 29-32)
    rho_cp, beta, bracket, b_over = -l1 * dt, l2 * dt / Ta, -l3 * dt * dt, l4 * dt
    eq18 = rho_cp * (Tn - Ta) / dt - beta * Ta * (pn - pa) / dt - LT
    eq19 = bracket * (pn - pa) / dt / dt - b_over * LT / dt + Dv / dt - Lp
    np.testing.assert_allclose(LT + l1 * Tn + l2 * pn - lT, -eq18, rtol=1e-9, atol=1e-9 * np.abs(l1 * Tn).max())
    np.testing.assert_allclose(Lp + l3 * pn + l4 * LT - lp, -eq19, rtol=1e-9, atol=1e-9 * np.abs(l3 * pn).max())


def test_divergence_exact_on_linear_fields():
    for name, g in GRIDS.items():
        uf = []
        for a in range(g.dim):
            s = list(g.face_shape(a))
            xf = np.arange(s[2 - a], dtype=float) * g.h + (g.r0 if (g.axisym and a == 0) else 0.0)
            shape = [1, 1, 1]
            shape[2 - a] = s[2 - a]
            uf.append(np.broadcast_to((0.7 + a) * xf.reshape(shape), s).copy())
        div = A.div_faces(g, uf)
        expect = sum(0.7 + a for a in range(g.dim)) + (0.7 if g.axisym else 0.0)   # axisymmetric: (1/r) d(r a r)/dr = 2a
        np.testing.assert_allclose(div, expect, rtol=1e-12)


@pytest.mark.parametrize("name", list(GRIDS))
def test_correction_divergence_and_phase_pressures(name):
    g = GRIDS[name]
    s = _state(g, seed=13)
    out = A.assemble(g, s.ph1, s.ph2, s.dt, s.C, s.m1, s.m2, s.E, s.mom, s.uf)
    rng = np.random.default_rng(5)
    x = out["x0"] + rng.normal(0, 1.0, out["x0"].shape) * np.array([1.0, 300.0])
    cor = A.correct(g, s.dt, s.sigma, x, s.C, s.kappa, out["fa"], s.uf)
    La, ba = laplacian(g, [f.reshape(-1) for f in out["fa"]])
    p = x[:, 1]
    Lp = La @ p
    for a in range(g.dim):
        for side in range(2):
            Lp = Lp + ba[a][side] * g.bcp[a][side]
    lhs = A.div_faces(g, cor["uf"]).reshape(-1)
    rhs = A.div_faces(g, s.uf).reshape(-1) - s.dt * Lp
    np.testing.assert_allclose(lhs, rhs, rtol=1e-9, atol=1e-9 * np.abs(rhs).max())
    pc = p.reshape(s.C.shape)
    np.testing.assert_allclose(s.C * cor["p1"] + (1 - s.C) * cor["p2"], pc, rtol=1e-14)
    np.testing.assert_allclose(cor["p1"] - cor["p2"], s.sigma * s.kappa, rtol=1e-9, atol=1e-9)


# ----------------------------------------------------------------------------
# Planted mistakes: each one is written into a copy of the oracle's source and
# must make at least one pin above fail.
# ----------------------------------------------------------------------------
import types

_SRC = open(os.path.join(os.path.dirname(HERE), "oracle", "assembly.py")).read()


def _mutant(old, new):
    assert _SRC.count(old) >= 1, old
    m = types.ModuleType("assembly_mutant")
    exec(compile(_SRC.replace(old, new, 1), "assembly_mutant", "exec"), m.__dict__)
    return m


MUTATIONS = [
    ("kinetic energy dropped (Eq. 20)", "p = (E - kinetic - shift) / denom", "p = (E - shift) / denom",
     lambda: test_round_trip_p_T("2d")),
    ("c_v instead of c_p - c_v (Eq. 23)", 'heat = heat + mi * (ph["cp"] - ph["cv"])', 'heat = heat + mi * ph["cv"]',
     lambda: test_round_trip_p_T("2d")),
    ("b p instead of b (p + Pi) (Eq. 10)", 'g1cv * T + ph["b"] * (p + ph["Pi"])', 'g1cv * T + ph["b"] * p',
     test_eq10_golden_water),
    ("sign of the bracket's second term (Eq. 31)", "gamma_i / (rho_i * c2) - bi * bi * T", "gamma_i / (rho_i * c2) + bi * bi * T",
     test_pure_consistent_phase_lambda3_is_isentropic),
    ("lambda_4 without 1/dt", 'l4 = b_over / dt if lambda4 == "restored" else b_over', "l4 = b_over",
     test_pure_consistent_phase_lambda3_is_isentropic),
    ("phase fractions C instead of m in rho c_p", 'rho_cp = rho_cp + mi * ph["cp"]', 'rho_cp = rho_cp + Ci * ph["cp"]',
     test_pure_consistent_phase_lambda3_is_isentropic),
    ("Dirichlet face gradient without the half-cell factor", "2.0 * (pc - gval) / h if side == 0", "(pc - gval) / h if side == 0",
     lambda: test_correction_divergence_and_phase_pressures("2d_dir")),
    ("axisymmetric divergence without r weights", "out = out + (rhi * u[hi] - rlo * u[lo]) / (ri * h)",
     "out = out + (u[hi] - u[lo]) / h", test_divergence_exact_on_linear_fields),
    ("lambda_p without div u*", "lp = l3 * p + div / dt", "lp = l3 * p",
     lambda: test_lambda_T_p_rearrange_eqs_18_19("2d")),
]


@pytest.mark.parametrize("label,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(monkeypatch, label, old, new, pin):
    monkeypatch.setitem(globals(), "A", _mutant(old, new))
    with pytest.raises(AssertionError):
        pin()


def test_harmonic_face_k_is_series_conduction():
    """Steady conduction through two half cells of conductivities k_L and k_R in
    series: the flux is (T_R - T_L) / (h/(2 k_L) + h/(2 k_R)), so the face
    coefficient of the difference (T_R - T_L)/h is 1 / (1/(2 k_L) + 1/(2 k_R))."""
    g = I.Grid(dim=2, axisym=0, n=(8, 4, 1), h=1e-3, bc=((W, W), (W, W), (0, 0)))
    ph1, ph2, C, m1, m2, E, mom, uf = _uniform_state(g, 0.0)
    C = np.zeros_like(C)
    C[:, :, :4] = 1.0                                  # liquid left, gas right: the interface at face i = 4
    r1, r2 = I.phase_density(310.0, 2e5, ph1), I.phase_density(310.0, 2e5, ph2)
    m1, m2 = C * r1, (1 - C) * r2
    E = C * I.phase_energy(2e5, r1, ph1) + (1 - C) * I.phase_energy(2e5, r2, ph2)
    out = A.assemble(g, ph1, ph2, 1e-7, C, m1, m2, E, mom, uf, face_k="harmonic")
    kL, kR = ph1.k, ph2.k
    series = 1.0 / (g.h / (2 * kL) / g.h + g.h / (2 * kR) / g.h)
    np.testing.assert_allclose(out["fk"][0][:, :, 4], series, rtol=1e-14)
    np.testing.assert_allclose(out["fk"][0][:, :, 2], kL, rtol=1e-14)     # inside one phase: its own k
    np.testing.assert_allclose(out["fk"][0][:, :, 6], kR, rtol=1e-14)
    arith = A.assemble(g, ph1, ph2, 1e-7, C, m1, m2, E, mom, uf)
    np.testing.assert_allclose(arith["fk"][0][:, :, 4], 0.5 * (kL + kR), rtol=1e-14)


# ----------------------------------------------------------------------------
# Eq. 39: the phase energies at the end of the step
# ----------------------------------------------------------------------------
def _faces_from(g, f):
    """Face arrays of each axis from a function f(a, X) of the face-centre coordinates."""
    out = []
    for a in range(g.dim):
        s = g.face_shape(a)
        X = []
        for b in range(3):
            n = s[2 - b]
            off = (g.r0 if (g.axisym and b == 0) else 0.0)
            x = (np.arange(n, dtype=float) + (0.0 if b == a else 0.5)) * g.h + off
            shape = [1, 1, 1]
            shape[2 - b] = n
            X.append(np.broadcast_to(x.reshape(shape), s))
        out.append(np.array(f(a, X), dtype=float) * np.ones(s))
    return out


def _energy_inputs(g, C=1.0, p=1e5, T=300.0, mu=0.0, k=0.0, uf=None):
    shape = (g.n[2], g.n[1], g.n[0])
    ph = I.NasgPhase(Gamma=1.4, Pi=0.0, b=0.0, q=0.0, cp=1005.0, cv=717.86, k=k, mu=mu)
    Cc = np.full(shape, C) if np.isscalar(C) else C
    pf = np.full(shape, p) if np.isscalar(p) else p
    Tf = np.full(shape, T) if np.isscalar(T) else T
    uf = uf if uf is not None else [np.zeros(g.face_shape(a)) for a in range(g.dim)]
    E = np.full(shape, 2.5e5)
    return ph, Cc, pf, Tf, uf, E


G2 = I.Grid(dim=2, axisym=0, n=(16, 12, 1), h=1e-3, bc=((W, W), (W, W), (0, 0)))


def _dE_close(dE, expect, E):
    """The change is read off E (~2.5e5): a few ulps of E, not of the change."""
    np.testing.assert_allclose(dE, expect, rtol=1e-9, atol=8 * np.finfo(float).eps * np.abs(E).max())
GAXI = I.Grid(dim=2, axisym=1, n=(12, 16, 1), h=1e-3, r0=0.0, bc=((AX, W), (W, W), (0, 0)))


def test_energy_at_rest_unchanged():
    ph, C, p, T, uf, E = _energy_inputs(G2, mu=1e-3, k=0.6)
    out = A.energy(G2, ph, ph, 1e-6, C, p, p, T, uf, E, E)
    assert np.array_equal(out["E1"], E) and np.array_equal(out["E2"], E)


def test_energy_couette_viscous_heating():
    """u_x = gamma y, u_y = 0: (S . u)_y = mu gamma^2 y, whose divergence is the
    viscous heating mu gamma^2 (rows whose two y-faces are inside)."""
    g, gam, mu, dt = G2, 300.0, 2e-3, 1e-6
    uf = _faces_from(g, lambda a, X: gam * X[1] if a == 0 else 0.0 * X[1])
    ph, C, p, T, _, E = _energy_inputs(g, p=0.0, mu=mu, uf=uf)
    out = A.energy(g, ph, ph, dt, C, p, p, T, uf, E, E)
    _dE_close((out["E1"] - E)[:, 1:-1, :], dt * mu * gam ** 2, E)


def test_energy_heat_conduction_of_a_quadratic():
    """No flow, T = T0 + a x^2: div(k grad T) = 2 a k exactly inside; C_i weights each phase."""
    g, a_, k, dt = G2, 4e4, 0.6, 1e-6
    x = (np.arange(g.n[0]) + 0.5) * g.h
    T = 300.0 + a_ * np.broadcast_to(x ** 2, (g.n[2], g.n[1], g.n[0]))
    ph, C, p, _, uf, E = _energy_inputs(g, C=0.3, k=k)
    out = A.energy(g, ph, ph, dt, C, p, p, T, uf, E, E)
    _dE_close((out["E1"] - E)[:, :, 1:-1], dt * 0.3 * 2 * a_ * k, E)
    _dE_close((out["E2"] - E)[:, :, 1:-1], dt * 0.7 * 2 * a_ * k, E)


@pytest.mark.parametrize("g", [G2, GAXI], ids=["2d", "axi"])
def test_energy_pressure_work_of_a_linear_flow(g):
    """Uniform p, u_a = c_a x_a: -div(p u) = -p (c_0 + c_1) (axisymmetric: u_r = c r has div = 2c)."""
    cs = (250.0, -120.0)
    uf = _faces_from(g, lambda a, X: cs[a] * X[a])
    ph, C, p, T, _, E = _energy_inputs(g, p=2e5, uf=uf)
    out = A.energy(g, ph, ph, 1e-6, C, p, p, T, uf, E, E)
    divu = (2 * cs[0] if g.axisym else cs[0]) + cs[1]
    _dE_close((out["E1"] - E)[:, 1:-1, 1:-1], -1e-6 * 2e5 * divu, E)


@pytest.mark.parametrize("g", [G2, GAXI, I.Grid(dim=3, axisym=0, n=(8, 6, 10), h=1e-3,
                                                bc=((W, W), (W, W), (W, W)))], ids=["2d", "axi", "3d"])
def test_energy_conserved_with_walls(g):
    """One phase everywhere, walls: every flux crosses between two cells and the
    boundary carries none, so the volume-weighted sum of the change vanishes."""
    rng = np.random.default_rng(8)
    shape = (g.n[2], g.n[1], g.n[0])
    uf = [rng.normal(0, 0.3, g.face_shape(a)) for a in range(g.dim)]
    for a in range(g.dim):
        uf[a][tuple(slice(0, 1) if ax == 2 - a else slice(None) for ax in range(3))] = 0.0
        uf[a][tuple(slice(-1, None) if ax == 2 - a else slice(None) for ax in range(3))] = 0.0
    ph, C, _, _, _, E = _energy_inputs(g, mu=1e-3, k=0.6)
    p = 1e5 + rng.normal(0, 300.0, shape)
    T = 300.0 + rng.normal(0, 2.0, shape)
    out = A.energy(g, ph, ph, 1e-6, C, p, p, T, uf, E, E)
    V = np.ones(shape) if not g.axisym else (g.r0 + (np.arange(g.n[0]) + 0.5) * g.h) * np.ones(shape)
    change = np.sum(V * (out["E1"] - E))
    scale = np.sum(V * np.abs(out["E1"] - E))
    assert abs(change) <= 1e-12 * scale


def test_energy_phases_add_to_one_phase():
    """Equal properties and pressures: the two phase updates sum to the one-phase update."""
    g = G2
    rng = np.random.default_rng(9)
    shape = (g.n[2], g.n[1], g.n[0])
    uf = [rng.normal(0, 0.3, g.face_shape(a)) for a in range(g.dim)]
    C = rng.uniform(0, 1, shape)
    ph, _, _, _, _, E = _energy_inputs(g, mu=1e-3, k=0.6)
    p = 1e5 + rng.normal(0, 300.0, shape)
    T = 300.0 + rng.normal(0, 2.0, shape)
    two = A.energy(g, ph, ph, 1e-6, C, p, p, T, uf, E, E)
    one = A.energy(g, ph, ph, 1e-6, np.ones(shape), p, p, T, uf, E, E)
    np.testing.assert_allclose(two["E1"] + two["E2"] - 2 * E, one["E1"] - E, rtol=1e-9, atol=1e-9 * np.abs(one["E1"] - E).max())


def _viscous_linear_pin():
    """Pure straining u_a = c_a x_a with p = 0: (S . u)_a = 2 c_a^2 x_a, whose divergence is 2 (c_0^2 + c_1^2)."""
    g, mu, dt = G2, 1e-3, 1e-6
    cs = (250.0, -120.0)
    uf = _faces_from(g, lambda a, X: cs[a] * X[a])
    ph, C, p, T, _, E = _energy_inputs(g, p=0.0, mu=mu, uf=uf)
    out = A.energy(g, ph, ph, dt, C, p, p, T, uf, E, E)
    _dE_close((out["E1"] - E)[:, 2:-2, 2:-2], dt * mu * 2 * (cs[0] ** 2 + cs[1] ** 2), E)


def test_energy_pure_straining_viscous_work():
    _viscous_linear_pin()


def test_energy_pressure_work_quadratic_pressure():
    """Uniform u_x = U, p = a x^2: -div(p u) = -U p'(x) = -2 a U x exactly with
    the two-cell face mean of p (central difference of a quadratic)."""
    g, U, a_, dt = G2, 3.0, 2e8, 1e-6
    uf = _faces_from(g, lambda a, X: U + 0.0 * X[0] if a == 0 else 0.0 * X[0])
    x = (np.arange(g.n[0]) + 0.5) * g.h
    shape = (g.n[2], g.n[1], g.n[0])
    p = 1e5 + a_ * np.broadcast_to(x ** 2, shape)
    ph, C, _, T, _, E = _energy_inputs(g, uf=uf)
    out = A.energy(g, ph, ph, dt, C, p, p, T, uf, E, E)
    _dE_close((out["E1"] - E)[:, :, 1:-1], np.broadcast_to(-dt * 2 * a_ * U * x, shape)[:, :, 1:-1], E)


def _taylor_green_error(n):
    """Viscous work of u = U (sin pi x cos pi y, -cos pi x sin pi y) on the unit
    square: div(mu S . u) = 2 mu U^2 pi^2 (cos 2 pi x cos^2 pi y + cos^2 pi x cos 2 pi y)
    (S_xy = 0 for this flow).  Max error over cells two or more from the walls."""
    g = I.Grid(dim=2, axisym=0, n=(n, n, 1), h=1.0 / n, bc=((W, W), (W, W), (0, 0)))
    U, mu, dt = 2.0, 1e-3, 1.0
    pi = np.pi
    uf = _faces_from(g, lambda a, X: U * np.sin(pi * X[0]) * np.cos(pi * X[1]) if a == 0
                     else -U * np.cos(pi * X[0]) * np.sin(pi * X[1]))
    ph, C, p, T, _, E = _energy_inputs(g, p=0.0, mu=mu, uf=uf)
    E = np.zeros_like(E)
    out = A.energy(g, ph, ph, dt, C, p, p, T, uf, E, E)
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc, indexing="xy")
    exact = 2 * mu * U ** 2 * pi ** 2 * (np.cos(2 * pi * X) * np.cos(pi * Y) ** 2 + np.cos(pi * X) ** 2 * np.cos(2 * pi * Y))
    return np.max(np.abs(out["E1"][0] - exact)[2:-2, 2:-2])


def test_energy_viscous_work_second_order():
    e1, e2 = _taylor_green_error(32), _taylor_green_error(64)
    assert e2 < e1 and e1 / e2 > 3.5, (e1, e2)


ENERGY_MUTATIONS = [
    ("normal strain without its factor 2", "s_ab = 2.0 * (ucell[a][hi] - ucell[a][lo]) / h",
     "s_ab = (ucell[a][hi] - ucell[a][lo]) / h", _viscous_linear_pin),
    ("heat flux with the wrong sign", "F[inner] = -pf * u_f[inner] + mu * visc + k * dTdn",
     "F[inner] = -pf * u_f[inner] + mu * visc - k * dTdn", test_energy_heat_conduction_of_a_quadratic),
    ("pressure-work face value from one cell", "pf = 0.5 * (pi[lo] + pi[hi])", "pf = pi[lo]",
     test_energy_pressure_work_quadratic_pressure),
    ("axisymmetric energy flux without r weights",
     "div = div + ((ri + 0.5 * h) * F[hi] - (ri - 0.5 * h) * F[lo]) / (ri * h)", "div = div + (F[hi] - F[lo]) / h",
     lambda: test_energy_pressure_work_of_a_linear_flow(GAXI)),
    ("tangential derivative from one cell", "s_ab = 0.5 * (dcell[a][b][lo] + dcell[a][b][hi]) + (ucell[b][hi] - ucell[b][lo]) / h",
     "s_ab = dcell[a][b][lo] + (ucell[b][hi] - ucell[b][lo]) / h", test_energy_viscous_work_second_order),
]


@pytest.mark.parametrize("label,old,new,pin", ENERGY_MUTATIONS, ids=[m[0] for m in ENERGY_MUTATIONS])
def test_planted_energy_mistake_is_caught(monkeypatch, label, old, new, pin):
    monkeypatch.setitem(globals(), "A", _mutant(old, new))
    with pytest.raises(AssertionError):
        pin()
