"""FP64 CPU oracle of the steps on either side of the solve (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU leg of ``bench.py`` may
import this module.  The CUDA library never calls it and shares no code with
it.  Plain numpy, float64, element by element in the paper's notation.

Before the solve (Sec. 3, from the advected state of Eq. Yadv):
- ``mixture_pT``   p^(adv) from the averaged total energy (Eq. 20), then
                   T^(adv) from p^(adv) (Eq. 23), both by the mixture's NASG EOS;
- ``phase_beta``   thermal dilation of a phase at (T, p) (Eq. 10);
- ``phase_c2``     squared speed of sound of a phase (Eq. 11);
- ``div_faces``    the cell divergence of a face-normal velocity field;
- ``assemble``     lambda_1..lambda_4, lambda_T, lambda_p (Eqs. 29-34), the face
                   coefficients 1/rho and k, and the initial guess
                   (T^(adv), p^(adv)).
After it:
- ``correct``      the velocity at the faces, u^{n+1} = u* - dt/rho grad p^{n+1}
                   (Eq. unp1), and the phase pressures of Eqs. 37-38;
- ``energy``       the phase total energies at the end of the step (Eq. 39):
                   pressure work, viscous work and heat conduction as face
                   fluxes, each face flux one value shared by its two cells.

Readings where the paper is silent:
- overlines are volume-fraction averages of the phase expressions; with the
  partial densities m_i = C_i rho_i they read C_i (1 - rho_i b_i) = C_i - m_i b_i
  and C_i rho_i q_i = m_i q_i, so no phase density is needed for p and T;
- the bracket gamma/(rho c^2) - beta^2 T/(rho c_p), beta, beta/(rho c_p) and
  rho c_p are averaged by C_i phase by phase; a phase with C_i = 0 adds nothing;
- lambda_4 = beta/(rho c_p dt) (Eq. 32 as printed lacks the 1/dt that dividing
  Eq. 19 by dt gives); ``lambda4="printed"`` gives the printed form;
- faces: 1/rho_f with rho_f the mean of the two cells' mixture densities, k_f =
  C_f k_1 + (1 - C_f) k_2 with C_f the mean of the two cells' C; a boundary face
  takes its cell's values; ``face_k="harmonic"`` instead takes the series mean
  2 k_L k_R / (k_L + k_R) of the cells' mixture conductivities k = C k_1 +
  (1 - C) k_2 (heat crossing two half cells);
- div u* and grad p are the finite-volume differences of the solve's operator
  (axisymmetric: r_f / r_i weights on the r-faces), so that the divergence of
  the corrected velocity is div u* - dt times the operator's p-Laplacian;
- Eq. 39: cell velocities are the means of the two face velocities; on a face
  the normal velocity is the face's own, the tangential velocities and p_i the
  means of the two cells, normal derivatives the difference across the face and
  tangential derivatives the mean of the two cells' central differences
  (one-sided in the first and last cell); walls and the axis carry no energy
  flux, a Dirichlet face carries -g_p u_f + k_i 2 (g_T - T)/h and no viscous
  flux; the divergence is multiplied by C_i (the phase's share).
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

BC_WALL, BC_DIRICHLET, BC_AXIS = 0, 1, 2


def _phase(ph) -> dict:
    return ph if isinstance(ph, dict) else dict(ph.__dict__)


def phase_beta(T, p, ph):
    """Eq. 10: beta_i = (Gamma_i - 1) c_v,i / ((Gamma_i - 1) c_v,i T + b_i (p + Pi_i))."""
    ph = _phase(ph)
    g1cv = (ph["Gamma"] - 1.0) * ph["cv"]
    return g1cv / (g1cv * T + ph["b"] * (p + ph["Pi"]))


def phase_c2(p, rho_i, ph):
    """Eq. 11: c_i^2 = Gamma_i (p + Pi_i) / (rho_i (1 - rho_i b_i))."""
    ph = _phase(ph)
    return ph["Gamma"] * (p + ph["Pi"]) / (rho_i * (1.0 - rho_i * ph["b"]))


def mixture_pT(C, m1, m2, E, mom: Sequence[np.ndarray], ph1, ph2):
    """Eq. 20 then Eq. 23 on the averaged state (C = C_1, C_2 = 1 - C)."""
    ph1, ph2 = _phase(ph1), _phase(ph2)
    Cs, ms = (C, 1.0 - C), (m1, m2)
    rho = m1 + m2
    kinetic = 0.5 * sum(mo * mo for mo in mom) / rho           # (1/2) rho |u|^2 with u = (rho u) / rho
    shift = 0.0
    denom = 0.0
    for Ci, mi, ph in zip(Cs, ms, (ph1, ph2)):
        free = Ci - mi * ph["b"]                                  # C_i (1 - rho_i b_i)
        shift = shift + ph["Gamma"] * ph["Pi"] / (ph["Gamma"] - 1.0) * free + mi * ph["q"]
        denom = denom + free / (ph["Gamma"] - 1.0)
    p = (E - kinetic - shift) / denom
    num = 0.0
    heat = 0.0
    for Ci, mi, ph in zip(Cs, ms, (ph1, ph2)):
        free = Ci - mi * ph["b"]
        num = num + free * p + ph["Pi"] * free                    # (1 - rho b) p + Pi (1 - rho b), averaged
        heat = heat + mi * (ph["cp"] - ph["cv"])                  # rho (c_p - c_v), averaged
    T = num / heat
    return p, T


def _cell_xyz(grid, a: int) -> np.ndarray:
    """Cell-centre coordinate index i_a + 1/2 along axis a, broadcast to (n2, n1, n0)."""
    n = grid.n
    shape = [1, 1, 1]
    shape[2 - a] = n[a]
    return (np.arange(n[a], dtype=np.float64) + 0.5).reshape(shape)


def _face_slices(a: int):
    lo = [slice(None)] * 3
    hi = [slice(None)] * 3
    lo[2 - a] = slice(0, -1)
    hi[2 - a] = slice(1, None)
    return tuple(lo), tuple(hi)


def div_faces(grid, uf: Sequence[np.ndarray]) -> np.ndarray:
    """Sum over axes of (flux through the high face - flux through the low face) / (cell size); face arrays
    shaped grid.face_shape(a).  Axisymmetric grids weight the r-faces (axis 0) by r_f / r_i."""
    h = grid.h
    out = np.zeros((grid.n[2], grid.n[1], grid.n[0]), dtype=np.float64)
    for a in range(grid.dim):
        lo, hi = _face_slices(a)
        u = np.asarray(uf[a], dtype=np.float64)
        if grid.axisym and a == 0:
            ri = grid.r0 + _cell_xyz(grid, 0) * h
            rlo, rhi = ri - 0.5 * h, ri + 0.5 * h
            out = out + (rhi * u[hi] - rlo * u[lo]) / (ri * h)
        else:
            out = out + (u[hi] - u[lo]) / h
    return out


def _neighbour_mean(v: np.ndarray, a: int) -> np.ndarray:
    """Face values of a cell field along axis a: the mean of the two cells, the cell's own at the boundary."""
    s = list(v.shape)
    s[2 - a] += 1
    f = np.empty(s, dtype=np.float64)
    lo, hi = _face_slices(a)
    inner = [slice(None)] * 3
    inner[2 - a] = slice(1, -1)
    first = [slice(None)] * 3
    first[2 - a] = slice(0, 1)
    last = [slice(None)] * 3
    last[2 - a] = slice(-1, None)
    f[tuple(inner)] = 0.5 * (v[lo] + v[hi])
    f[tuple(first)] = v[tuple(first)]
    f[tuple(last)] = v[tuple(last)]
    return f


def _harmonic_faces(v: np.ndarray, a: int) -> np.ndarray:
    """Face values 2 v_L v_R / (v_L + v_R) along axis a; the cell's own at the boundary."""
    f = _neighbour_mean(v, a)              # boundary faces: the cell's value
    lo, hi = _face_slices(a)
    inner = [slice(None)] * 3
    inner[2 - a] = slice(1, -1)
    f[tuple(inner)] = 2.0 * v[lo] * v[hi] / (v[lo] + v[hi])
    return f


def assemble(grid, ph1, ph2, dt: float, C, m1, m2, E, mom: Sequence[np.ndarray], uf: Sequence[np.ndarray],
             lambda4: str = "restored", face_k: str = "arithmetic") -> Dict[str, np.ndarray]:
    """The inputs of the solve from the advected state.  Cell arrays shaped
    (n2, n1, n0), face arrays grid.face_shape(a).  Returns lam (N x 4), b
    (N x 2), x0 (N x 2), fa / fk (per axis), and p, T, div."""
    ph1, ph2 = _phase(ph1), _phase(ph2)
    p, T = mixture_pT(C, m1, m2, E, mom, ph1, ph2)
    Cs, ms = (C, 1.0 - C), (m1, m2)
    rho_cp = 0.0
    beta = 0.0
    b_over = 0.0
    bracket = 0.0
    for Ci, mi, ph in zip(Cs, ms, (ph1, ph2)):
        bi = phase_beta(T, p, ph)
        present = Ci > 0.0
        rho_i = np.where(present, mi / np.where(present, Ci, 1.0), 1.0)   # phase density where the phase is present
        c2 = phase_c2(p, rho_i, ph)
        gamma_i = ph["cp"] / ph["cv"]
        rho_cp = rho_cp + mi * ph["cp"]
        beta = beta + Ci * bi
        b_over = b_over + np.where(present, Ci * bi / (rho_i * ph["cp"]), 0.0)
        bracket = bracket + np.where(present, Ci * (gamma_i / (rho_i * c2) - bi * bi * T / (rho_i * ph["cp"])), 0.0)
    div = div_faces(grid, uf)
    l1 = -rho_cp / dt                                            # Eq. 29
    l2 = beta * T / dt                                           # Eq. 30
    l3 = -bracket / (dt * dt)                                    # Eq. 31
    l4 = b_over / dt if lambda4 == "restored" else b_over        # Eq. 32 (1/dt restored)
    lT = l1 * T + l2 * p                                         # Eq. 33
    lp = l3 * p + div / dt                                       # Eq. 34
    rho = m1 + m2
    fa: List[np.ndarray] = []
    fk: List[np.ndarray] = []
    for a in range(grid.dim):
        fa.append(1.0 / _neighbour_mean(rho, a))
        if face_k == "harmonic":
            fk.append(_harmonic_faces(C * ph1["k"] + (1.0 - C) * ph2["k"], a))
        else:
            Cf = _neighbour_mean(C, a)
            fk.append(Cf * ph1["k"] + (1.0 - Cf) * ph2["k"])
    flat = lambda v: np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    lam = np.stack([flat(l1), flat(l2), flat(l3), flat(l4)], axis=1)
    return dict(lam=lam, b=np.stack([flat(lT), flat(lp)], axis=1), x0=np.stack([flat(T), flat(p)], axis=1),
                fa=fa, fk=fk, p=p, T=T, div=div)


def correct(grid, dt: float, sigma: float, x: np.ndarray, C, kappa, fa: Sequence[np.ndarray],
            uf: Sequence[np.ndarray]) -> Dict[str, object]:
    """Eq. unp1 at the faces: u^{n+1} = u* - dt (1/rho)_f (grad p^{n+1})_f, with
    the operator's face gradients: (p_R - p_L)/h inside, 2 (g - p_cell)/h
    towards a Dirichlet value g, zero at walls and the axis.  Then Eqs. 37-38:
    p_1 = p + (1 - C) sigma kappa, p_2 = p - C sigma kappa."""
    n = grid.n
    p = np.asarray(x, dtype=np.float64).reshape(n[2], n[1], n[0], 2)[..., 1]
    h = grid.h
    out = []
    for a in range(grid.dim):
        lo, hi = _face_slices(a)
        g = np.zeros(grid.face_shape(a), dtype=np.float64)
        inner = [slice(None)] * 3
        inner[2 - a] = slice(1, -1)
        g[tuple(inner)] = (p[hi] - p[lo]) / h
        for side in (0, 1):
            if grid.bc[a][side] != BC_DIRICHLET:
                continue
            gval = grid.bcp[a][side]
            face = [slice(None)] * 3
            cell = [slice(None)] * 3
            face[2 - a] = slice(0, 1) if side == 0 else slice(-1, None)
            cell[2 - a] = slice(0, 1) if side == 0 else slice(-1, None)
            pc = p[tuple(cell)]
            g[tuple(face)] = 2.0 * (pc - gval) / h if side == 0 else 2.0 * (gval - pc) / h
        out.append(np.asarray(uf[a], dtype=np.float64) - dt * np.asarray(fa[a], dtype=np.float64) * g)
    sk = sigma * np.asarray(kappa, dtype=np.float64)
    Cc = np.asarray(C, dtype=np.float64)
    return dict(uf=out, p1=p + (1.0 - Cc) * sk, p2=p - Cc * sk)


# ---------------------------------------------------------------------------
# Eq. 39: the phase total energies at the end of the step.
# ---------------------------------------------------------------------------
def cell_velocity(grid, uf: Sequence[np.ndarray]) -> List[np.ndarray]:
    """Cell-centre velocity components: the mean of the two face velocities along each axis (Algorithm 1)."""
    out = []
    for a in range(grid.dim):
        lo, hi = _face_slices(a)
        u = np.asarray(uf[a], dtype=np.float64)
        out.append(0.5 * (u[lo] + u[hi]))
    return out


def _cell_derivative(v: np.ndarray, b: int, h: float) -> np.ndarray:
    """d v / d x_b at the cells: central differences inside, one-sided at the first and last cell."""
    d = np.empty_like(v)
    n = v.shape[2 - b]
    sl = lambda s: tuple(s if ax == 2 - b else slice(None) for ax in range(3))
    if n == 1:
        return np.zeros_like(v)
    d[sl(slice(1, -1))] = (v[sl(slice(2, None))] - v[sl(slice(0, -2))]) / (2.0 * h)
    d[sl(slice(0, 1))] = (v[sl(slice(1, 2))] - v[sl(slice(0, 1))]) / h
    d[sl(slice(-1, None))] = (v[sl(slice(-1, None))] - v[sl(slice(-2, -1))]) / h
    return d


def energy(grid, ph1, ph2, dt: float, C, p1, p2, T, uf: Sequence[np.ndarray], E1, E2) -> Dict[str, np.ndarray]:
    """Eq. 39 for both phases: (C_i rho_i e_T,i)^{n+1} = (C_i rho_i e_T,i)^(adv) +
    dt C_i div F_i with the face fluxes of axis a
        F_i = -p_i,f u_f + mu_i (S . u)_{a,f} + k_i (dT/dx_a)_f,
    S = grad u + grad u^T.  u_f: the face velocity (u^{n+1} of Eq. unp1); cell
    velocities: means of the two face velocities; p_i,f, u_b,f (b != a): means of
    the two cells; normal derivatives across the face, tangential ones the mean
    of the two cells' (central, one-sided at the edge).  Boundary faces: walls and
    the axis carry no flux; a Dirichlet face carries -g_p u_f + k_i 2 (g_T - T)/h
    towards the boundary value (no viscous flux).  Both phases share T (thermal
    equilibrium).  The divergence uses the solve's finite volumes (r_f / r_i on
    axisymmetric r-faces)."""
    ph1, ph2 = _phase(ph1), _phase(ph2)
    h = grid.h
    dim = grid.dim
    ucell = cell_velocity(grid, uf)
    dcell = [[_cell_derivative(ucell[a], b, h) for b in range(dim)] for a in range(dim)]   # dcell[a][b] = du_a/dx_b
    Tc = np.asarray(T, dtype=np.float64)
    out = {}
    for name, ph, pi, Ci, Ei in (("E1", ph1, p1, C, E1), ("E2", ph2, p2, 1.0 - np.asarray(C), E2)):
        mu, k = ph.get("mu", 0.0), ph["k"]
        div = np.zeros_like(Tc)
        for a in range(dim):
            lo, hi = _face_slices(a)
            u_f = np.asarray(uf[a], dtype=np.float64)
            F = np.zeros(grid.face_shape(a), dtype=np.float64)
            inner = [slice(None)] * 3
            inner[2 - a] = slice(1, -1)
            inner = tuple(inner)
            # pressure work and heat flux on interior faces
            pf = 0.5 * (pi[lo] + pi[hi])
            dTdn = (Tc[hi] - Tc[lo]) / h
            visc = 0.0
            for b in range(dim):
                if b == a:
                    s_ab = 2.0 * (ucell[a][hi] - ucell[a][lo]) / h
                    ub = u_f[inner]
                else:
                    s_ab = 0.5 * (dcell[a][b][lo] + dcell[a][b][hi]) + (ucell[b][hi] - ucell[b][lo]) / h
                    ub = 0.5 * (ucell[b][lo] + ucell[b][hi])
                visc = visc + s_ab * ub
            F[inner] = -pf * u_f[inner] + mu * visc + k * dTdn
            for side in (0, 1):
                if grid.bc[a][side] != BC_DIRICHLET:
                    continue
                face = [slice(None)] * 3
                cell = [slice(None)] * 3
                face[2 - a] = slice(0, 1) if side == 0 else slice(-1, None)
                cell[2 - a] = slice(0, 1) if side == 0 else slice(-1, None)
                Tb = Tc[tuple(cell)]
                gT, gp = grid.bcT[a][side], grid.bcp[a][side]
                dT = 2.0 * (Tb - gT) / h if side == 0 else 2.0 * (gT - Tb) / h
                F[tuple(face)] = -gp * u_f[tuple(face)] + k * dT
            if grid.axisym and a == 0:
                ri = grid.r0 + _cell_xyz(grid, 0) * h
                div = div + ((ri + 0.5 * h) * F[hi] - (ri - 0.5 * h) * F[lo]) / (ri * h)
            else:
                div = div + (F[hi] - F[lo]) / h
        out[name] = np.asarray(Ei, dtype=np.float64) + dt * np.asarray(Ci, dtype=np.float64) * div
    return out
