"""Pins of the momentum-predictor oracle (oracle/momentum.py) against what the
mathematics fixes, independently of the oracle itself:

- quadratic velocities with a linear viscosity: the scheme's face fluxes are
  exact there, so away from the boundaries A(u) equals (rho/dt) u minus the
  closed-form div(mu (grad u + grad u^T)), in 2D and 3D;
- axisymmetric closed forms: a uniform radial expansion u_r = a r (its stress
  divergence and the hoop term cancel, down to the cell on the axis), u_z = b r^2
  and the shear u_r = c z;
- the wall rules on uniform flows (free slip, no slip, flow into a wall) and
  the pressure boundaries;
- the direct solve recovers a manufactured solution, and the sparse matrix
  reproduces apply().
Each planted mistake in the oracle's source must fail one of these.
"""
import os
import types

import numpy as np
import pytest

from paper_2206_11294_gb300 import inputs as I

W, D, AX = I.BC_WALL, I.BC_DIRICHLET, I.BC_AXIS
EPS = np.finfo(float).eps
_SRC = open(os.path.join(os.path.dirname(__file__), "..", "oracle", "momentum.py")).read()

import oracle.momentum as M  # noqa: E402


def _centres(g):
    """Cell-centre coordinates (x_0, x_1, x_2) broadcast to (n2, n1, n0)."""
    out = []
    for a in range(3):
        shape = [1, 1, 1]
        shape[2 - a] = g.n[a]
        base = g.r0 if (g.axisym and a == 0) else 0.0
        out.append(np.broadcast_to((base + (np.arange(g.n[a]) + 0.5) * g.h).reshape(shape),
                                   (g.n[2], g.n[1], g.n[0])))
    return out


def _interior(g, k=2):
    s = [slice(None)] * 3
    for a in range(g.dim):
        s[2 - a] = slice(k, g.n[a] - k)
    return tuple(s)


def _quadratic_case(g, seed):
    """u_c = B_c . x + x^T Q_c x, mu = m0 + m . x, and the closed-form div(mu (grad u + grad u^T))."""
    rng = np.random.default_rng(seed)
    d = g.dim
    X = _centres(g)[:d]
    B = rng.normal(size=(d, d))
    Q = rng.normal(size=(d, d, d))
    Q = 0.5 * (Q + Q.transpose(0, 2, 1))
    m0, m = 2.0, rng.uniform(-0.5, 0.5, d)
    u = [sum(B[c, a] * X[a] for a in range(d)) + sum(Q[c, a, b] * X[a] * X[b] for a in range(d) for b in range(d))
         for c in range(d)]
    mu = m0 + sum(m[a] * X[a] for a in range(d))
    grad = lambda c, a: B[c, a] + 2 * sum(Q[c, a, b] * X[b] for b in range(d))        # du_c/dx_a
    div = []
    for c in range(d):
        t = 0.0
        for a in range(d):
            t = t + m[a] * (grad(c, a) + grad(a, c)) + mu * (2 * Q[c, a, a] + 2 * Q[a, a, c])
        div.append(t)
    return u, mu, div


@pytest.mark.parametrize("dim", [2, 3])
def test_quadratic_velocity_linear_viscosity_exact(dim):
    n = (12, 10, 1) if dim == 2 else (9, 8, 7)
    bc = ((W, D), (D, W), (W, W)) if dim == 3 else ((W, D), (D, W), (0, 0))
    g = I.Grid(dim=dim, axisym=0, n=n, h=0.1, bc=bc)
    u, mu, div = _quadratic_case(g, 3 + dim)
    rho, dt = np.full(mu.shape, 3.0), 0.25
    Au = M.apply(g, rho, mu, dt, u)
    s = _interior(g)
    for c in range(dim):
        expect = rho / dt * u[c] - div[c]
        scale = np.abs(rho / dt * u[c]) + np.abs(div[c]) + 1.0
        np.testing.assert_allclose(Au[c][s] / scale[s], expect[s] / scale[s], rtol=0, atol=1e-12)


def _axi(n=(10, 12, 1)):
    return I.Grid(dim=2, axisym=1, n=n, h=0.05, r0=0.0, bc=((AX, D), (D, D), (0, 0)))


def test_axisymmetric_uniform_expansion_has_no_viscous_force():
    """u_r = a r: (1/r) d(r 2 mu a)/dr = 2 mu a / r is cancelled by the hoop term, in every cell whose r-faces carry
    the radial stress (the first cell's low face is the axis, r_f = 0)."""
    g = _axi()
    r = _centres(g)[0]
    a, mu0, rho, dt = 0.7, 1.3, 2.0, 0.1
    u = [a * r, np.zeros_like(r)]
    Au = M.apply(g, np.full(r.shape, rho), np.full(r.shape, mu0), dt, u)
    s = (slice(None), slice(None), slice(0, -1))            # all but the last column (its outer face has no stress)
    np.testing.assert_allclose(Au[0][s], (rho / dt * a * r)[s], rtol=1e-13)
    np.testing.assert_allclose(Au[1], 0.0, atol=1e-12)


def test_axisymmetric_quadratic_axial_velocity():
    """u_z = b r^2: (1/r) d(r mu 2 b r)/dr = 4 mu b, exact including the cell on the axis."""
    g = _axi()
    r = _centres(g)[0]
    b, mu0, rho, dt = 0.9, 0.6, 1.5, 0.2
    u = [np.zeros_like(r), b * r * r]
    Au = M.apply(g, np.full(r.shape, rho), np.full(r.shape, mu0), dt, u)
    s = (slice(None), slice(2, -2), slice(0, -1))
    np.testing.assert_allclose(Au[1][s], (rho / dt * b * r * r - 4 * mu0 * b)[s], rtol=1e-12)
    np.testing.assert_allclose(Au[0][s], 0.0, atol=1e-11)


def test_axisymmetric_shear_cross_term():
    """u_r = c z: tau_rz = mu c, so the z-row gets -(1/r) d(r mu c)/dr = -mu c / r and the r-row the hoop term
    2 mu c z / r^2 (no r-stress divergence, d(mu c)/dz = 0)."""
    g = _axi()
    X = _centres(g)
    r, z = X[0], X[1]
    c, mu0, rho, dt = 1.1, 0.8, 1.0, 0.5
    u = [c * z, np.zeros_like(r)]
    Au = M.apply(g, np.full(r.shape, rho), np.full(r.shape, mu0), dt, u)
    s = (slice(None), slice(2, -2), slice(0, -1))
    np.testing.assert_allclose(Au[1][s], (-mu0 * c / r)[s], rtol=1e-12)
    np.testing.assert_allclose(Au[0][s], (rho / dt * c * z + 2 * mu0 * c * z / r ** 2)[s], rtol=1e-12)


GW = I.Grid(dim=2, axisym=0, n=(8, 6, 1), h=0.1, bc=((D, D), (W, W), (0, 0)))


@pytest.mark.parametrize("no_slip", [False, True])
def test_wall_tangential_uniform_flow(no_slip):
    """u_x = c along the y-walls: free slip leaves (rho/dt) u; no slip adds the shear mu 2c/h / h in the wall rows."""
    g = GW
    shape = (1, g.n[1], g.n[0])
    cval, mu0, rho, dt, h = 2.0, 0.3, 1.2, 0.1, g.h
    u = [np.full(shape, cval), np.zeros(shape)]
    Au = M.apply(g, np.full(shape, rho), np.full(shape, mu0), dt, u, no_slip=no_slip)
    expect = np.full(shape, rho / dt * cval)
    if no_slip:
        expect[:, 0, :] += 2 * mu0 * cval / h ** 2
        expect[:, -1, :] += 2 * mu0 * cval / h ** 2
    np.testing.assert_allclose(Au[0], expect, rtol=1e-14)
    np.testing.assert_allclose(Au[1], 0.0, atol=1e-13)


def test_wall_normal_uniform_flow_and_pressure_boundary():
    """u_y = c into the y-walls: the normal stress 2 mu 2c/h adds 4 mu c / h^2 in the wall rows whatever the slip
    condition; u_x = c through the pressure (x) boundaries meets no stress there."""
    g = GW
    shape = (1, g.n[1], g.n[0])
    cval, mu0, rho, dt, h = 1.5, 0.4, 0.8, 0.2, g.h
    for no_slip in (False, True):
        u = [np.zeros(shape), np.full(shape, cval)]
        Au = M.apply(g, np.full(shape, rho), np.full(shape, mu0), dt, u, no_slip=no_slip)
        expect = np.full(shape, rho / dt * cval)
        expect[:, 0, :] += 4 * mu0 * cval / h ** 2
        expect[:, -1, :] += 4 * mu0 * cval / h ** 2
        np.testing.assert_allclose(Au[1], expect, rtol=1e-14)
        np.testing.assert_allclose(Au[0], 0.0, atol=1e-13)
    u = [np.full(shape, cval), np.zeros(shape)]
    Au = M.apply(g, np.full(shape, rho), np.full(shape, mu0), dt, u)
    np.testing.assert_allclose(Au[0], rho / dt * cval, rtol=1e-14)


@pytest.mark.parametrize("kind", ["2d", "axi", "3d"])
def test_solve_recovers_manufactured_velocity(kind):
    if kind == "2d":
        g = I.Grid(dim=2, axisym=0, n=(10, 8, 1), h=0.1, bc=((W, D), (W, W), (0, 0)))
    elif kind == "axi":
        g = _axi((8, 10, 1))
    else:
        g = I.Grid(dim=3, axisym=0, n=(6, 5, 4), h=0.1, bc=((W, D), (W, W), (D, W)))
    rng = np.random.default_rng(11)
    shape = (g.n[2], g.n[1], g.n[0])
    rho = rng.uniform(1.0, 1000.0, shape)
    mu = rng.uniform(1e-3, 1.0, shape)
    dt = 0.05
    u = [rng.normal(size=shape) for _ in range(g.dim)]
    for no_slip in (False, True):
        R = M.apply(g, rho, mu, dt, u, no_slip=no_slip)
        A = M.matrix(g, rho, mu, dt, no_slip=no_slip)
        np.testing.assert_allclose(A @ np.concatenate([v.reshape(-1) for v in u]),
                                   np.concatenate([v.reshape(-1) for v in R]), rtol=1e-13, atol=1e-10)
        got = M.solve(g, rho, mu, dt, R, no_slip=no_slip)
        for c in range(g.dim):
            np.testing.assert_allclose(got[c], u[c], rtol=1e-9, atol=1e-9)


GD = I.Grid(dim=2, axisym=0, n=(10, 8, 1), h=0.1, bc=((D, W), (W, D), (0, 0)),
            bcp=((0.0, 0.0), (0.0, 0.0), (0.0, 0.0)))


def _linear(g, a0, grad):
    X = _centres(g)
    return a0 + sum(grad[a] * X[a] for a in range(g.dim))


def _dirichlet_of_linear(g, a0, grad):
    """Boundary values of the linear field on each face plane (they vary along it only through other axes: the
    pins below use fields that vary along one axis, so each boundary value is one number)."""
    vals = []
    for a in range(3):
        lo = a0 + (grad[a] * 0.0 if a < g.dim else 0.0)
        hi = a0 + (grad[a] * g.n[a] * g.h if a < g.dim else 0.0)
        vals.append((lo, hi))
    return vals


@pytest.mark.parametrize("axis", [0, 1])
def test_cell_gradient_of_a_linear_field(axis):
    """Inside: the slope.  At a Dirichlet face with the field's own boundary value: the slope too.  At a wall
    (zero face gradient) the boundary cell gets half the slope; without boundary values every boundary cell does."""
    slope = [0.0, 0.0]
    slope[axis] = 3.0
    bc = [(W, W), (W, W), (0, 0)]
    bc[axis] = (D, W)                                  # boundary values only where the field is one number per plane
    g = I.Grid(dim=2, axisym=0, n=(10, 8, 1), h=0.1, bc=tuple(bc))
    s = _linear(g, 2.0, slope)
    gd = M.cell_gradient(g, s, _dirichlet_of_linear(g, 2.0, slope))
    expect = np.full(s.shape, 3.0)
    lo, hi = _sl_cells(axis, 0), _sl_cells(axis, -1)
    if g.bc[axis][0] != D:
        expect[lo] = 1.5
    if g.bc[axis][1] != D:
        expect[hi] = 1.5
    np.testing.assert_allclose(gd[axis], expect, rtol=1e-12)
    np.testing.assert_allclose(gd[1 - axis], 0.0, atol=1e-12)
    g0 = M.cell_gradient(g, s)
    expect = np.full(s.shape, 3.0)
    expect[lo] = expect[hi] = 1.5
    np.testing.assert_allclose(g0[axis], expect, rtol=1e-12)


def _sl_cells(a, i):
    s = [slice(None)] * 3
    s[2 - a] = slice(i, i + 1) if i >= 0 else slice(i, None)
    return tuple(s)


def test_rhs_closed_form():
    """R = mom/dt - grad p + sigma kappa grad C for linear p and C, uniform kappa, inside."""
    g = GD
    rng = np.random.default_rng(3)
    shape = (1, g.n[1], g.n[0])
    mom = [rng.normal(size=shape) for _ in range(2)]
    gp, gC = (2e3, -5e2), (4.0, 7.0)
    p, C = _linear(g, 1e5, gp), _linear(g, 0.3, gC)
    dt, sigma, kap = 1e-4, 0.07, 50.0
    R = M.rhs(g, dt, sigma, mom, p, np.full(shape, kap), C)
    s = _interior(g, 1)
    for c in range(2):
        np.testing.assert_allclose(R[c][s], (mom[c] / dt - gp[c] + sigma * kap * gC[c])[s], rtol=1e-12)


def test_provisional_faces_of_a_linear_velocity():
    """u_pred,x = U + S x, p uniform: inside, u*_f is the field at the face; walls carry 0; a pressure boundary its
    cell's value."""
    g = I.Grid(dim=2, axisym=0, n=(10, 8, 1), h=0.1, bc=((D, W), (W, D), (0, 0)),
               bcp=((1e5, 0.0), (0.0, 1e5), (0.0, 0.0)))
    X = _centres(g)
    U, S = 0.4, 2.0
    shape = (1, g.n[1], g.n[0])
    u = [U + S * X[0], np.zeros(shape)]
    uf = M.provisional_faces(g, 1e-3, np.full(shape, 2.0), np.full(shape, 1e5), u)
    xf = np.arange(g.n[0] + 1) * g.h
    expect = np.broadcast_to(U + S * xf, g.face_shape(0)).copy()
    expect[:, :, 0] = U + S * 0.5 * g.h               # axis 0, low side: pressure boundary -> the cell's value
    expect[:, :, -1] = 0.0                            # high side: wall
    np.testing.assert_allclose(uf[0], expect, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(uf[1], 0.0, atol=1e-15)


def test_pressure_only_step_leaves_no_provisional_velocity():
    """No momentum, viscosity or surface tension: the predictor gives u_pred = -(dt/rho) grad p^n, and Eq. provel
    removes exactly that, so u* vanishes on every face (the projection then carries the whole pressure gradient)."""
    g = GD
    rng = np.random.default_rng(5)
    shape = (1, g.n[1], g.n[0])
    rho = rng.uniform(1.0, 1000.0, shape)
    p = 1e5 + rng.normal(0.0, 1e3, shape)
    dt = 1e-3
    R = M.rhs(g, dt, 0.0, [np.zeros(shape)] * 2, p, np.zeros(shape), np.zeros(shape))
    u_pred = M.solve(g, rho, np.zeros(shape), dt, R)
    uf = M.provisional_faces(g, dt, rho, p, u_pred)
    scale = max(np.abs(dt / rho * gp).max() for gp in M.cell_gradient(g, p, g.bcp))
    for a in range(2):
        np.testing.assert_allclose(uf[a], 0.0, atol=1e-12 * scale)


def _mutant(old, new):
    assert _SRC.count(old) >= 1, old
    m = types.ModuleType("momentum_mutant")
    exec(compile(_SRC.replace(old, new, 1), "momentum_mutant", "exec"), m.__dict__)
    return m


MUTATIONS = [
    ("hoop term dropped", "Au = Au + 2.0 * mu * u[0] / _r_cells(grid) ** 2", "Au = Au",
     test_axisymmetric_uniform_expansion_has_no_viscous_force),
    ("normal stress without its factor 2", "F[inner] = muf[inner] * (normal + normal)", "F[inner] = muf[inner] * normal",
     lambda: test_quadratic_velocity_linear_viscosity_exact(2)),
    ("transposed cross derivative", "dc = _cell_derivative(u[a], c, h)", "dc = _cell_derivative(u[c], a, h)",
     lambda: test_quadratic_velocity_linear_viscosity_exact(2)),
    ("face viscosity from one cell",
     "0.5 * (mu[_sl(a, slice(0, -1))] + mu[_sl(a, slice(1, None))])", "mu[_sl(a, slice(0, -1))]",
     lambda: test_quadratic_velocity_linear_viscosity_exact(3)),
    ("wall ghost at h instead of h/2", "d = 2.0 * ub / h if side == 0 else -2.0 * ub / h",
     "d = ub / h if side == 0 else -ub / h", test_wall_normal_uniform_flow_and_pressure_boundary),
    ("axisymmetric fluxes without r weights",
     "div = div + ((ri + 0.5 * h) * F[hi] - (ri - 0.5 * h) * F[lo]) / (ri * h)", "div = div + (F[hi] - F[lo]) / h",
     test_axisymmetric_quadratic_axial_velocity),
    ("free slip treated as no slip", "if c != a and not no_slip:", "if False:",
     lambda: test_wall_tangential_uniform_flow(False)),
    ("tangential derivative from one cell", "F[inner] = muf[inner] * (normal + 0.5 * (dc[lo] + dc[hi]))",
     "F[inner] = muf[inner] * (normal + dc[lo])", lambda: test_quadratic_velocity_linear_viscosity_exact(2)),
    ("Eq. provel with the wrong sign", "ua = np.asarray(u_pred[a], dtype=np.float64) + dt / rho * gp[a]",
     "ua = np.asarray(u_pred[a], dtype=np.float64) - dt / rho * gp[a]",
     test_pressure_only_step_leaves_no_provisional_velocity),
    ("face velocity from one cell",
     "f[_sl(a, slice(1, -1))] = 0.5 * (ua[_sl(a, slice(0, -1))] + ua[_sl(a, slice(1, None))])",
     "f[_sl(a, slice(1, -1))] = ua[_sl(a, slice(0, -1))]", test_provisional_faces_of_a_linear_velocity),
    ("Dirichlet face gradient at h", "g[cell] = 2.0 * (s[cell] - gv) / h if side == 0 else 2.0 * (gv - s[cell]) / h",
     "g[cell] = (s[cell] - gv) / h if side == 0 else (gv - s[cell]) / h", lambda: test_cell_gradient_of_a_linear_field(0)),
    ("surface-tension force with the wrong sign", "- gp[c] + sigma * kap * gC[c]", "- gp[c] - sigma * kap * gC[c]",
     test_rhs_closed_form),
]


@pytest.mark.parametrize("label,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_momentum_mistake_is_caught(monkeypatch, label, old, new, pin):
    monkeypatch.setitem(globals(), "M", _mutant(old, new))
    with pytest.raises(AssertionError):
        pin()
