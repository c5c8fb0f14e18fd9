"""FP64 CPU oracle of the implicit momentum predictor (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may
import this module.  The CUDA library never calls it and shares no code with
it.  Plain numpy and scipy, float64, in the paper's notation.

The predicted velocity of a time step (Sec. 3, the equation before Eq. unp1)
solves, per cell and component c,

    (rho/dt) u_c - [div(mu (grad u + grad u^T))]_c = R_c,

R = (rho u)^(adv)/dt - grad p^n + sigma kappa grad C, given.  rho and mu are the
cells' averaged density and viscosity.
- ``face_viscosity``  mu on the faces;
- ``stress_flux``     tau_{ca} = mu_f ((du_c/dx_a)_f + (du_a/dx_c)_f) on the
                      faces of axis a;
- ``apply``           the left-hand side A(u), face flux by face flux;
- ``matrix``          A as a sparse matrix, column by column from ``apply``;
- ``solve``           the exact solution of A u = R by a sparse direct solve
                      (small grids);
- ``cell_gradient``   the gradient of a cell field at the cells: the mean of
                      the cell's two face gradients along each axis;
- ``rhs``             R = (rho u)^(adv)/dt - grad p^n + sigma kappa grad C;
- ``provisional_faces`` Eq. provel, u* = u_pred + (dt/rho) grad p^n at the
                      cells, then the faces' normal components for the
                      projection (Eq. unp1).

Readings where the paper is silent:
- mu_f is the mean of the two cells' mu; a boundary face takes its cell's;
- on a face the normal derivative is the difference across the face; the
  tangential derivative (du_a/dx_c, c != a) the mean of the two cells' central
  differences, one-sided in the first and last cell (as for Eq. 39);
- walls: the normal component is zero on the wall (ghost value -u), so the
  normal stress is 2 mu 2 u / h towards it; the tangential components slip
  freely (no shear stress), or with ``no_slip`` are zero on the wall (shear
  mu 2 u / h); the tangential derivative of the normal component is zero along
  a wall;
- Dirichlet (pressure) boundaries and the axis: zero velocity gradient, no
  stress through the face;
- axisymmetric (axis 0 = r, axis 1 = z): r-face fluxes weighted by r_f / r_i,
  and the hoop stress adds 2 mu u_r / r_i^2 to the r-row (the hoop component
  of the stress is 2 mu u_r / r; it adds nothing to the z-row);
- no bulk viscosity (Stokes' hypothesis, Sec. 2);
- cell gradients are the means of the face gradients of the projection's
  operator: (s_R - s_L)/h inside; for p, 2 (g - p)/h towards a Dirichlet value
  and 0 at walls and the axis; for C, 0 at every boundary (no value given);
- the face velocity u*_f is the mean of the two cells' normal components of
  u*; walls and the axis carry 0, a pressure boundary its cell's value.
"""
from __future__ import annotations

from typing import List, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BC_WALL, BC_DIRICHLET, BC_AXIS = 0, 1, 2


def _sl(a: int, s) -> tuple:
    out = [slice(None)] * 3
    out[2 - a] = s
    return tuple(out)


def _r_cells(grid) -> np.ndarray:
    """Radius of the cell centres, broadcast to (n2, n1, n0)."""
    return (grid.r0 + (np.arange(grid.n[0], dtype=np.float64) + 0.5) * grid.h).reshape(1, 1, -1)


def _cell_derivative(v: np.ndarray, b: int, h: float) -> np.ndarray:
    """d v / d x_b at the cells: central differences inside, one-sided in the first and last cell."""
    n = v.shape[2 - b]
    if n == 1:
        return np.zeros_like(v)
    d = np.empty_like(v)
    d[_sl(b, slice(1, -1))] = (v[_sl(b, slice(2, None))] - v[_sl(b, slice(0, -2))]) / (2.0 * h)
    d[_sl(b, slice(0, 1))] = (v[_sl(b, slice(1, 2))] - v[_sl(b, slice(0, 1))]) / h
    d[_sl(b, slice(-1, None))] = (v[_sl(b, slice(-1, None))] - v[_sl(b, slice(-2, -1))]) / h
    return d


def face_viscosity(grid, mu) -> List[np.ndarray]:
    mu = np.asarray(mu, dtype=np.float64)
    out = []
    for a in range(grid.dim):
        f = np.empty(grid.face_shape(a), dtype=np.float64)
        f[_sl(a, slice(1, -1))] = 0.5 * (mu[_sl(a, slice(0, -1))] + mu[_sl(a, slice(1, None))])
        f[_sl(a, slice(0, 1))] = mu[_sl(a, slice(0, 1))]
        f[_sl(a, slice(-1, None))] = mu[_sl(a, slice(-1, None))]
        out.append(f)
    return out


def stress_flux(grid, mu, u: Sequence[np.ndarray], c: int, a: int, no_slip: bool = False) -> np.ndarray:
    """tau_{ca} on the faces of axis a (shape grid.face_shape(a))."""
    h = grid.h
    muf = face_viscosity(grid, mu)[a]
    F = np.zeros(grid.face_shape(a), dtype=np.float64)
    lo, hi = _sl(a, slice(0, -1)), _sl(a, slice(1, None))
    inner = _sl(a, slice(1, -1))
    normal = (u[c][hi] - u[c][lo]) / h                     # du_c/dx_a across the face
    if c == a:
        F[inner] = muf[inner] * (normal + normal)
    else:
        dc = _cell_derivative(u[a], c, h)                   # du_a/dx_c at the cells
        F[inner] = muf[inner] * (normal + 0.5 * (dc[lo] + dc[hi]))
    for side in (0, 1):
        if grid.bc[a][side] != BC_WALL:
            continue                                        # pressure boundary or axis: no stress
        if c != a and not no_slip:
            continue                                        # free slip: no shear on the wall
        cell = _sl(a, slice(0, 1) if side == 0 else slice(-1, None))
        ub = u[c][cell]
        d = 2.0 * ub / h if side == 0 else -2.0 * ub / h     # towards the wall value 0
        F[cell] = (2.0 if c == a else 1.0) * muf[cell] * d
    return F


def apply(grid, rho, mu, dt: float, u: Sequence[np.ndarray], no_slip: bool = False) -> List[np.ndarray]:
    """A(u) = (rho/dt) u - div(mu (grad u + grad u^T)) (+ 2 mu u_r / r^2 in the r-row, axisymmetric)."""
    h = grid.h
    rho = np.asarray(rho, dtype=np.float64)
    mu = np.asarray(mu, dtype=np.float64)
    u = [np.asarray(v, dtype=np.float64) for v in u]
    out = []
    for c in range(grid.dim):
        div = np.zeros_like(rho)
        for a in range(grid.dim):
            F = stress_flux(grid, mu, u, c, a, no_slip)
            lo, hi = _sl(a, slice(0, -1)), _sl(a, slice(1, None))
            if grid.axisym and a == 0:
                ri = _r_cells(grid)
                div = div + ((ri + 0.5 * h) * F[hi] - (ri - 0.5 * h) * F[lo]) / (ri * h)
            else:
                div = div + (F[hi] - F[lo]) / h
        Au = rho / dt * u[c] - div
        if grid.axisym and c == 0:
            Au = Au + 2.0 * mu * u[0] / _r_cells(grid) ** 2
        out.append(Au)
    return out


def matrix(grid, rho, mu, dt: float, no_slip: bool = False) -> sp.csc_matrix:
    """A as a sparse (dim N) x (dim N) matrix, unknown c * N + cell (cells in C order of (n2, n1, n0))."""
    N, dim = grid.N, grid.dim
    shape = (grid.n[2], grid.n[1], grid.n[0])
    cols = []
    for c in range(dim):
        for i in range(N):
            e = [np.zeros(shape) for _ in range(dim)]
            e[c].reshape(-1)[i] = 1.0
            col = np.concatenate([v.reshape(-1) for v in apply(grid, rho, mu, dt, e, no_slip)])
            cols.append(sp.csc_matrix(col.reshape(-1, 1)))
    return sp.hstack(cols).tocsc()


def solve(grid, rho, mu, dt: float, R: Sequence[np.ndarray], no_slip: bool = False) -> List[np.ndarray]:
    """The exact solution of A u = R (sparse LU)."""
    A = matrix(grid, rho, mu, dt, no_slip)
    b = np.concatenate([np.asarray(r, dtype=np.float64).reshape(-1) for r in R])
    x = spla.spsolve(A, b)
    shape = (grid.n[2], grid.n[1], grid.n[0])
    return [x[c * grid.N:(c + 1) * grid.N].reshape(shape) for c in range(grid.dim)]


def cell_gradient(grid, s, dirichlet=None) -> List[np.ndarray]:
    """d s / d x_a at the cells, a < dim: the mean of the low and high face gradients.  dirichlet: None (zero
    gradient at every boundary) or per-axis, per-side boundary values used where grid.bc is BC_DIRICHLET."""
    h = grid.h
    s = np.asarray(s, dtype=np.float64)
    out = []
    for a in range(grid.dim):
        g = np.zeros(grid.face_shape(a), dtype=np.float64)
        g[_sl(a, slice(1, -1))] = (s[_sl(a, slice(1, None))] - s[_sl(a, slice(0, -1))]) / h
        if dirichlet is not None:
            for side in (0, 1):
                if grid.bc[a][side] != BC_DIRICHLET:
                    continue
                cell = _sl(a, slice(0, 1) if side == 0 else slice(-1, None))
                gv = dirichlet[a][side]
                g[cell] = 2.0 * (s[cell] - gv) / h if side == 0 else 2.0 * (gv - s[cell]) / h
        out.append(0.5 * (g[_sl(a, slice(0, -1))] + g[_sl(a, slice(1, None))]))
    return out


def rhs(grid, dt: float, sigma: float, mom: Sequence[np.ndarray], p, kappa, C) -> List[np.ndarray]:
    """R_c = (rho u)_c^(adv) / dt - (dp^n/dx_c) + sigma kappa (dC/dx_c), per cell."""
    gp = cell_gradient(grid, p, grid.bcp)
    gC = cell_gradient(grid, C)
    kap = np.asarray(kappa, dtype=np.float64)
    return [np.asarray(mom[c], dtype=np.float64) / dt - gp[c] + sigma * kap * gC[c] for c in range(grid.dim)]


def provisional_faces(grid, dt: float, rho, p, u_pred: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Eq. provel at the cells, u* = u_pred + (dt/rho) grad p^n, then per axis a the face-normal component: the mean
    of the two cells' u*_a inside, 0 at walls and the axis, the cell's value at a pressure boundary."""
    gp = cell_gradient(grid, p, grid.bcp)
    rho = np.asarray(rho, dtype=np.float64)
    out = []
    for a in range(grid.dim):
        ua = np.asarray(u_pred[a], dtype=np.float64) + dt / rho * gp[a]
        f = np.zeros(grid.face_shape(a), dtype=np.float64)
        f[_sl(a, slice(1, -1))] = 0.5 * (ua[_sl(a, slice(0, -1))] + ua[_sl(a, slice(1, None))])
        for side in (0, 1):
            if grid.bc[a][side] == BC_DIRICHLET:
                cell = _sl(a, slice(0, 1) if side == 0 else slice(-1, None))
                f[cell] = ua[cell]
        out.append(f)
    return out
