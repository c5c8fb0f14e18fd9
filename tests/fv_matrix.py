"""Independent sparse assembly of the paper's operator (test helper).

Builds L of Eqs. 27-28 as matrices from one-dimensional gradient operators
(Kronecker products), face-area and cell-volume diagonals:

    div(c grad u) = V^-1  sum_a  Gt_a  diag(A_a c_a)  G_a u   (+ boundary part)

with G_a the face gradient along axis a (interior faces (u_R - u_L)/h,
Dirichlet faces (g - u)/(h/2) on the low side's outward normal convention
folded in, walls and the axis zero) and Gt_a the signed face-to-cell sum.
This is a different construction from the oracle's per-cell stencil loop, so
agreement pins the oracle's geometry, face indexing and boundary handling.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

WALL, DIRICHLET, AXIS = 0, 1, 2


def _grid_get(g):
    return (lambda k: g[k]) if isinstance(g, dict) else (lambda k: getattr(g, k))


def _grad_1d(n: int, h: float, lo: int, hi: int):
    """(n+1) x n face gradient along one axis and the (n+1) vector of
    coefficients multiplying the boundary value g (so grad = G u + gb * g)."""
    G = sp.lil_matrix((n + 1, n))
    glo = np.zeros(n + 1)
    ghi = np.zeros(n + 1)
    for f in range(1, n):
        G[f, f - 1] = -1.0 / h
        G[f, f] = 1.0 / h
    if lo == DIRICHLET:          # gradient at face 0 = (u_0 - g) / (h/2)
        G[0, 0] = 2.0 / h
        glo[0] = -2.0 / h
    if hi == DIRICHLET:          # gradient at face n = (g - u_{n-1}) / (h/2)
        G[n, n - 1] = -2.0 / h
        ghi[n] = 2.0 / h
    return G.tocsr(), glo, ghi


def _div_1d(n: int):
    """n x (n+1): cell sum of (flux at high face - flux at low face)."""
    D = sp.lil_matrix((n, n + 1))
    for i in range(n):
        D[i, i] = -1.0
        D[i, i + 1] = 1.0
    return D.tocsr()


def _expand(M1, a: int, n):
    """Lift a 1D operator on axis a to the full grid (x fastest)."""
    ops = []
    for b in (2, 1, 0):                 # kron order: slowest axis first
        if b >= len(n):
            continue
        ops.append(M1 if b == a else sp.identity(n[b], format="csr"))
    out = ops[0]
    for o in ops[1:]:
        out = sp.kron(out, o, format="csr")
    return out


def laplacian(g, coef):
    """(Lc, c_bnd) with div(c grad u) = Lc u + sum_{a,side} c_bnd[a][side] * g_value."""
    get = _grid_get(g)
    dim, axisym, h, r0 = get("dim"), get("axisym"), get("h"), get("r0")
    n = list(get("n"))[:dim]
    bc = get("bc")
    N = int(np.prod(n))
    # cell volumes, face areas
    ic = [np.arange(n[a]) for a in range(dim)]
    mesh = np.meshgrid(*[ic[a] for a in reversed(range(dim))], indexing="ij")
    idx = [m.reshape(-1) for m in reversed(mesh)]        # idx[a][cell] (x fastest)
    if axisym:
        rc = r0 + (idx[0] + 0.5) * h
        V = rc * h * h
    else:
        V = np.full(N, h ** dim)
    Vinv = sp.diags(1.0 / V)
    L = sp.csr_matrix((N, N))
    bnd = []
    for a in range(dim):
        G1, glo1, ghi1 = _grad_1d(n[a], h, bc[a][0], bc[a][1])
        D1 = _div_1d(n[a])
        G = _expand(G1, a, n)
        Dv = _expand(D1, a, n)
        nf = [n[b] + 1 if b == a else n[b] for b in range(dim)]
        fmesh = np.meshgrid(*[np.arange(nf[b]) for b in reversed(range(dim))], indexing="ij")
        fidx = [m.reshape(-1) for m in reversed(fmesh)]
        if axisym:
            Af = (r0 + fidx[0] * h) * h if a == 0 else (r0 + (fidx[0] + 0.5) * h) * h
        else:
            Af = np.full(fidx[0].shape, h ** (dim - 1))
        c = np.asarray(coef[a], dtype=float)
        W = sp.diags(Af * c)
        L = L + Vinv @ Dv @ W @ G
        # boundary value columns
        sides = []
        for gb in (glo1, ghi1):
            ones = np.ones(1)
            gvec_1d = gb
            lifted = _expand(sp.csr_matrix(gvec_1d.reshape(-1, 1)), a, n) @ np.ones(
                int(np.prod([n[b] for b in range(dim) if b != a])))
            sides.append(Vinv @ Dv @ (Af * c * lifted))
        bnd.append(sides)
    return L.tocsr(), bnd


def paper_operator(g, lam, fa, fk):
    """(M, affine) with L(x) = M x + affine, unknowns interleaved (T, p) per cell."""
    get = _grid_get(g)
    dim = get("dim")
    bcT, bcp = get("bcT"), get("bcp")
    Lk, bk = laplacian(g, fk)
    La, ba = laplacian(g, fa)
    lam = np.asarray(lam).reshape(-1, 4)
    l1, l2, l3, l4 = (sp.diags(lam[:, q]) for q in range(4))
    top = sp.hstack([Lk + l1, l2])
    bot = sp.hstack([l4 @ Lk, La + l3])
    M = sp.vstack([top, bot]).tocsr()
    N = lam.shape[0]
    perm = np.empty(2 * N, dtype=int)
    perm[0::2] = np.arange(N)
    perm[1::2] = N + np.arange(N)
    M = M[perm][:, perm]
    aT = np.zeros(N)
    ap = np.zeros(N)
    for a in range(dim):
        for side in range(2):
            aT += bk[a][side] * bcT[a][side]
            ap += ba[a][side] * bcp[a][side]
    affine = np.empty(2 * N)
    affine[0::2] = aT
    affine[1::2] = ap + lam[:, 3] * aT
    return M, affine
