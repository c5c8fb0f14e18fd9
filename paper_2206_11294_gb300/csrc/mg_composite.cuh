// Kernels of the coupled p-T solve on a refined-patch (adaptive) grid: a
// uniform base grid of spacing H over the domain and one box of base cells
// refined 2:1 into a patch of spacing h = H / 2 (2D Cartesian, FP64).  The
// paper's production grids are coarsened away from the bubble (Sec. 5.2);
// this is the two-level, block-structured form of that.
//
// Unknowns: the patch's cells and the base cells outside the box.  Every
// valid cell carries Eqs. 27-28 with its finite-volume divergence:
//   - between two cells of one level: the uniform-grid flux (physical
//     coefficients c on the faces, no row scaling);
//   - domain boundary: wall (no flux) or Dirichlet (value h/2 away);
//   - coarse-fine interface, fine side: c_f (u~ - u_f) / (1.5 h), with
//     u~ = u_C + s (u_{C+t} - u_{C-t}) / 8 the coarse field at the fine cell's
//     tangential position, 1.5 h from its centre;
//   - coarse-fine interface, base side: the sum of its two fine faces' fluxes
//     (conservative).
// The solve (mg_composite_solve) is defect correction with FAC cycles: patch
// colour sweeps on the composite rows, the patch residual restricted under
// the box and the base residual corrected for the patch's interface fluxes,
// one V-cycle of the base grid's hierarchy, the correction prolonged onto the
// patch, patch sweeps again.
//
// Cells are x-fastest; base faces of axis 0 are (n0 + 1) per row, of axis 1
// n0 per row over n1 + 1 rows; the patch's likewise with m0, m1.
#pragma once
#include "mg_types.cuh"

namespace cmg {

struct CfGeom {
    int n0, n1;            // base cells per axis
    int b0[2], b1[2];      // the box: base cells [b0[a], b1[a]) per axis
    int m0, m1;            // patch cells per axis
    double H, h;           // spacings
    int dir[2][2];         // Dirichlet side (1) or wall (0), per axis and side
    double gT[2][2], gp[2][2];   // Dirichlet values (zero for the correction problems)
    int iface[2][2];       // patch side inside the domain (1): a coarse-fine interface
    // the flux factors, as reciprocals (the kernels multiply; FP64 division
    // is a long instruction sequence on this GPU): patch faces between two
    // patch cells 1/h^2, at the interface 1/(1.5 h^2), at a Dirichlet side
    // 1/(0.5 h^2); base faces 1/H^2, 1/(0.5 H^2), and the base side of the
    // interface 1/(1.5 H^2) (two fine faces of length h over the area H^2)
    double rh2, rif, rdf, rH2, rdb, rbif;
};

struct CfCoef {            // physical coefficients of both levels
    const double *lamb, *fab[2], *fkb[2];
    const double *lamf, *faf[2], *fkf[2];
};

__device__ __forceinline__ bool cf_covered(const CfGeom &g, int I, int J) {
    return I >= g.b0[0] && I < g.b1[0] && J >= g.b0[1] && J < g.b1[1];
}

__device__ __forceinline__ long long cf_bface(const CfGeom &g, int a, int I, int J) {
    return a == 0 ? (long long)I + (long long)(g.n0 + 1) * J : (long long)I + (long long)g.n0 * J;
}

__device__ __forceinline__ long long cf_fface(const CfGeom &g, int a, int i, int j) {
    return a == 0 ? (long long)i + (long long)(g.m0 + 1) * j : (long long)i + (long long)g.m0 * j;
}

// (T, p) of base cell (I, J), or across the domain boundary its ghost: the
// mirror at a wall, 2 g - u at a Dirichlet side, each side's rule in turn
// (x first) at a corner.
__device__ __forceinline__ double2 cf_base_value(const CfGeom &g, const double2 *__restrict__ xb, int I, int J) {
    int out[2] = {-1, -1};
    int ci = I, cj = J;
    if (I < 0) { ci = 0; out[0] = 0; }
    if (I >= g.n0) { ci = g.n0 - 1; out[0] = 1; }
    if (J < 0) { cj = 0; out[1] = 0; }
    if (J >= g.n1) { cj = g.n1 - 1; out[1] = 1; }
    double2 u = xb[ci + (long long)g.n0 * cj];
#pragma unroll
    for (int ax = 0; ax < 2; ax++) {
        const int s = out[ax];
        if (s < 0 || !g.dir[ax][s]) continue;
        u = make_double2(2.0 * g.gT[ax][s] - u.x, 2.0 * g.gp[ax][s] - u.y);
    }
    return u;
}

// u~ of patch cell (fi, fj) across its interface side (a, s).
__device__ __forceinline__ double2 cf_ghost(const CfGeom &g, const double2 *__restrict__ xb, int a, int s, int fi,
                                            int fj) {
    const int t = 1 - a;
    const int f[2] = {fi, fj};
    int C[2];
    C[a] = s == 0 ? g.b0[a] - 1 : g.b1[a];
    C[t] = g.b0[t] + f[t] / 2;
    const double sgn = (f[t] & 1) ? 1.0 : -1.0;
    int Cp[2] = {C[0], C[1]}, Cm[2] = {C[0], C[1]};
    Cp[t] += 1;
    Cm[t] -= 1;
    const double2 uc = cf_base_value(g, xb, C[0], C[1]);
    const double2 up = cf_base_value(g, xb, Cp[0], Cp[1]);
    const double2 um = cf_base_value(g, xb, Cm[0], Cm[1]);
    return make_double2(uc.x + sgn * (up.x - um.x) * 0.125, uc.y + sgn * (up.y - um.y) * 0.125);
}

// div(k grad T), div((1/rho) grad p) of valid base cell (I, J).
__device__ __forceinline__ void cf_base_div(const CfGeom &g, const CfCoef &k, const double2 *__restrict__ xb,
                                            const double2 *__restrict__ xf, int I, int J, double &lapT, double &lapp) {
    const double2 u = xb[I + (long long)g.n0 * J];
    lapT = 0.0;
    lapp = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            int nb[2] = {I, J};
            nb[a] += s ? 1 : -1;
            const int na = a == 0 ? g.n0 : g.n1;
            const bool inside = nb[a] >= 0 && nb[a] < na;
            if (inside && cf_covered(g, nb[0], nb[1])) {
                const int t = 1 - a, side = s ? 0 : 1;
                const int fin = side == 0 ? 0 : (a == 0 ? g.m0 : g.m1) - 1;
                const int ct = t == 0 ? I : J;
#pragma unroll
                for (int q = 0; q < 2; q++) {
                    int ff[2];
                    ff[a] = fin;
                    ff[t] = 2 * (ct - g.b0[t]) + q;
                    int fface[2] = {ff[0], ff[1]};
                    fface[a] += side;
                    const long long fid = cf_fface(g, a, fface[0], fface[1]);
                    const double2 uf = xf[ff[0] + (long long)g.m0 * ff[1]];
                    const double2 gu = cf_ghost(g, xb, a, side, ff[0], ff[1]);
                    lapT += k.fkf[a][fid] * (uf.x - gu.x) * g.rbif;
                    lapp += k.faf[a][fid] * (uf.y - gu.y) * g.rbif;
                }
            } else if (inside) {
                const long long fid = cf_bface(g, a, I + (a == 0 ? s : 0), J + (a == 1 ? s : 0));
                const double2 un = xb[nb[0] + (long long)g.n0 * nb[1]];
                lapT += k.fkb[a][fid] * (un.x - u.x) * g.rH2;
                lapp += k.fab[a][fid] * (un.y - u.y) * g.rH2;
            } else if (g.dir[a][s]) {
                const long long fid = cf_bface(g, a, I + (a == 0 ? s : 0), J + (a == 1 ? s : 0));
                lapT += k.fkb[a][fid] * (g.gT[a][s] - u.x) * g.rdb;
                lapp += k.fab[a][fid] * (g.gp[a][s] - u.y) * g.rdb;
            }
        }
}

// div(k grad T), div((1/rho) grad p) of patch cell (i, j), and the diagonal
// terms sigma_k, sigma_a (minus the coefficients of its own T and p).
__device__ __forceinline__ void cf_fine_div(const CfGeom &g, const CfCoef &k, const double2 *__restrict__ xb,
                                            const double2 *__restrict__ xf, int i, int j, double &lapT, double &lapp,
                                            double &sk, double &sa) {
    const double2 u = xf[i + (long long)g.m0 * j];
    lapT = lapp = sk = sa = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            int nb[2] = {i, j};
            nb[a] += s ? 1 : -1;
            const int ma = a == 0 ? g.m0 : g.m1;
            const long long fid = cf_fface(g, a, i + (a == 0 ? s : 0), j + (a == 1 ? s : 0));
            const double ck = k.fkf[a][fid], ca = k.faf[a][fid];
            if (nb[a] >= 0 && nb[a] < ma) {
                const double2 un = xf[nb[0] + (long long)g.m0 * nb[1]];
                lapT += ck * (un.x - u.x) * g.rh2;
                lapp += ca * (un.y - u.y) * g.rh2;
                sk += ck * g.rh2;
                sa += ca * g.rh2;
            } else if (g.iface[a][s]) {
                const double2 gu = cf_ghost(g, xb, a, s, i, j);
                lapT += ck * (gu.x - u.x) * g.rif;
                lapp += ca * (gu.y - u.y) * g.rif;
                sk += ck * g.rif;
                sa += ca * g.rif;
            } else if (g.dir[a][s]) {
                lapT += ck * (g.gT[a][s] - u.x) * g.rdf;
                lapp += ca * (g.gp[a][s] - u.y) * g.rdf;
                sk += ck * g.rdf;
                sa += ca * g.rdf;
            }
        }
}

// Composite rows: y = L(x) on the valid base cells (covered cells 0) or, with
// b, r = b - L(x).
__global__ void __launch_bounds__(256) k_cf_rows_base(CfGeom g, CfCoef k, const double2 *__restrict__ xb,
                                                      const double2 *__restrict__ xf, const double2 *__restrict__ b,
                                                      double2 *__restrict__ out) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= g.n0 || J >= g.n1) return;
    const long long c = I + (long long)g.n0 * J;
    if (cf_covered(g, I, J)) {
        out[c] = make_double2(0.0, 0.0);
        return;
    }
    double lapT, lapp;
    cf_base_div(g, k, xb, xf, I, J, lapT, lapp);
    const double *l = k.lamb + 4 * c;
    const double2 u = xb[c];
    const double yT = lapT + l[0] * u.x + l[1] * u.y;
    const double yp = lapp + l[2] * u.y + l[3] * lapT;
    out[c] = b ? make_double2(b[c].x - yT, b[c].y - yp) : make_double2(yT, yp);
}

__global__ void __launch_bounds__(256) k_cf_rows_fine(CfGeom g, CfCoef k, const double2 *__restrict__ xb,
                                                      const double2 *__restrict__ xf, const double2 *__restrict__ b,
                                                      double2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.m0 || j >= g.m1) return;
    const long long c = i + (long long)g.m0 * j;
    double lapT, lapp, sk, sa;
    cf_fine_div(g, k, xb, xf, i, j, lapT, lapp, sk, sa);
    const double *l = k.lamf + 4 * c;
    const double2 u = xf[c];
    const double yT = lapT + l[0] * u.x + l[1] * u.y;
    const double yp = lapp + l[2] * u.y + l[3] * lapT;
    out[c] = b ? make_double2(b[c].x - yT, b[c].y - yp) : make_double2(yT, yp);
}

// One colour of a red-black block Gauss-Seidel sweep on the patch rows of the
// correction problem (homogeneous: g has zero Dirichlet values and the base
// values xb0 are zero; a nonzero base correction enters through rhs).
__global__ void __launch_bounds__(256) k_cf_rbgs_fine(CfGeom g, CfCoef k, const double2 *__restrict__ xb0,
                                                      const double2 *__restrict__ rhs, double2 *__restrict__ xf,
                                                      int colour) {
    const int ii = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = 2 * ii + ((j + colour) & 1);
    if (i >= g.m0 || j >= g.m1) return;
    const long long c = i + (long long)g.m0 * j;
    double lapT, lapp, sk, sa;
    cf_fine_div(g, k, xb0, xf, i, j, lapT, lapp, sk, sa);
    const double *l = k.lamf + 4 * c;
    const double2 u = xf[c];
    const double e0 = lapT + l[0] * u.x + l[1] * u.y;
    const double e1 = lapp + l[2] * u.y + l[3] * lapT;
    const double D0 = l[0] - sk, D1 = l[1], D2 = -l[3] * sk, D3 = l[2] - sa;
    const double s0 = rhs[c].x - (e0 - (D0 * u.x + D1 * u.y));
    const double s1 = rhs[c].y - (e1 - (D2 * u.x + D3 * u.y));
    const double rdet = 1.0 / (D0 * D3 - D1 * D2);
    xf[c] = make_double2((D3 * s0 - D1 * s1) * rdet, (D0 * s1 - D2 * s0) * rdet);
}

// The base correction problem's right-hand side: valid cells the composite
// residual rb minus what the patch correction df adds to their rows through
// the interface (zero base values); covered cells the mean of their four
// children's patch residual sf.
__global__ void __launch_bounds__(256) k_cf_base_rhs(CfGeom g, CfCoef k, const double2 *__restrict__ rb,
                                                     const double2 *__restrict__ df, const double2 *__restrict__ sf,
                                                     double2 *__restrict__ sb) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I >= g.n0 || J >= g.n1) return;
    const long long c = I + (long long)g.n0 * J;
    if (cf_covered(g, I, J)) {
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const long long f = (2 * (I - g.b0[0]) + (q & 1)) + (long long)g.m0 * (2 * (J - g.b0[1]) + (q >> 1));
            s0 += sf[f].x;
            s1 += sf[f].y;
        }
        sb[c] = make_double2(s0 * 0.25, s1 * 0.25);
        return;
    }
    double tT = 0.0, tp = 0.0;
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            int nb[2] = {I, J};
            nb[a] += s ? 1 : -1;
            const int na = a == 0 ? g.n0 : g.n1;
            if (!(nb[a] >= 0 && nb[a] < na && cf_covered(g, nb[0], nb[1]))) continue;
            const int t = 1 - a, side = s ? 0 : 1;
            const int fin = side == 0 ? 0 : (a == 0 ? g.m0 : g.m1) - 1;
            const int ct = t == 0 ? I : J;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                int ff[2];
                ff[a] = fin;
                ff[t] = 2 * (ct - g.b0[t]) + q;
                int fface[2] = {ff[0], ff[1]};
                fface[a] += side;
                const long long fid = cf_fface(g, a, fface[0], fface[1]);
                const double2 d = df[ff[0] + (long long)g.m0 * ff[1]];
                tT += k.fkf[a][fid] * d.x * g.rbif;
                tp += k.faf[a][fid] * d.y * g.rbif;
            }
        }
    const double oT = tT, op = tp + k.lamb[4 * c + 3] * tT;
    sb[c] = make_double2(rb[c].x - oT, rb[c].y - op);
}

// After the base correction db: the patch correction df += its bilinear
// prolongation (the fine cells' positions in the whole domain; homogeneous
// ghosts outside it), and out = rf minus what db adds to the patch rows
// through the interface ghosts (the p-row's l4 div(k grad T) included).
__global__ void __launch_bounds__(256) k_cf_prolong_ghost(CfGeom g, CfCoef k, const double2 *__restrict__ db,
                                                          const double2 *__restrict__ rf, double2 *__restrict__ df,
                                                          double2 *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.m0 || j >= g.m1) return;
    const long long c = i + (long long)g.m0 * j;
    const int gi = 2 * g.b0[0] + i, gj = 2 * g.b0[1] + j;
    const int P[2] = {gi / 2, gj / 2};
    const int sg[2] = {(gi & 1) ? 1 : -1, (gj & 1) ? 1 : -1};
    double aT = 0.0, ap = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        double w = 1.0;
        int Q[2] = {P[0], P[1]};
#pragma unroll
        for (int a = 0; a < 2; a++) {
            if ((q >> a) & 1) {
                w *= 0.25;
                Q[a] += sg[a];
            } else {
                w *= 0.75;
            }
        }
        const double2 v = cf_base_value(g, db, Q[0], Q[1]);
        aT += w * v.x;
        ap += w * v.y;
    }
    df[c] = make_double2(df[c].x + aT, df[c].y + ap);
    double gT = 0.0, gp = 0.0;
    const int pos[2] = {i, j};
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            if (!g.iface[a][s]) continue;
            const int ma = a == 0 ? g.m0 : g.m1;
            if ((s == 0 && pos[a] != 0) || (s == 1 && pos[a] != ma - 1)) continue;
            const long long fid = cf_fface(g, a, i + (a == 0 ? s : 0), j + (a == 1 ? s : 0));
            const double2 gu = cf_ghost(g, db, a, s, i, j);
            gT += k.fkf[a][fid] * gu.x * g.rif;
            gp += k.faf[a][fid] * gu.y * g.rif;
        }
    out[c] = make_double2(rf[c].x - gT, rf[c].y - (gp + k.lamf[4 * c + 3] * gT));
}

// x += correction on the valid base cells and the patch.
__global__ void __launch_bounds__(256) k_cf_update(CfGeom g, double2 *__restrict__ xb, double2 *__restrict__ xf,
                                                   const double2 *__restrict__ db, const double2 *__restrict__ df) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x, J = blockIdx.y * blockDim.y + threadIdx.y;
    if (I < g.n0 && J < g.n1 && !cf_covered(g, I, J)) {
        const long long c = I + (long long)g.n0 * J;
        xb[c] = make_double2(xb[c].x + db[c].x, xb[c].y + db[c].y);
    }
    if (I < g.m0 && J < g.m1) {
        const long long c = I + (long long)g.m0 * J;
        xf[c] = make_double2(xf[c].x + df[c].x, xf[c].y + df[c].y);
    }
}

// Covered base cells of xb: the mean of their four children in xf.
__global__ void __launch_bounds__(256) k_cf_covered_mean(CfGeom g, double2 *__restrict__ xb,
                                                         const double2 *__restrict__ xf) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x + g.b0[0], J = blockIdx.y * blockDim.y + threadIdx.y + g.b0[1];
    if (I >= g.b1[0] || J >= g.b1[1]) return;
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const long long f = (2 * (I - g.b0[0]) + (q & 1)) + (long long)g.m0 * (2 * (J - g.b0[1]) + (q >> 1));
        s0 += xf[f].x;
        s1 += xf[f].y;
    }
    xb[I + (long long)g.n0 * J] = make_double2(s0 * 0.25, s1 * 0.25);
}

// The base hierarchy's coefficients: the caller's base arrays, with the
// covered cells' l1..l4 the mean of their four children's and every face of
// a covered cell the mean of its two fine faces (in, out: base arrays; out
// starts as a copy of in).
__global__ void __launch_bounds__(256) k_cf_cover(CfGeom g, CfCoef k, double *__restrict__ lam,
                                                  double *__restrict__ fa0, double *__restrict__ fa1,
                                                  double *__restrict__ fk0, double *__restrict__ fk1) {
    const int I = blockIdx.x * blockDim.x + threadIdx.x + g.b0[0], J = blockIdx.y * blockDim.y + threadIdx.y + g.b0[1];
    if (I >= g.b1[0] || J >= g.b1[1]) return;
    const long long c = I + (long long)g.n0 * J;
#pragma unroll
    for (int t = 0; t < 4; t++) {
        double acc = 0.0;
#pragma unroll
        for (int q = 0; q < 4; q++) {
            const long long f = (2 * (I - g.b0[0]) + (q & 1)) + (long long)g.m0 * (2 * (J - g.b0[1]) + (q >> 1));
            acc += k.lamf[4 * f + t];
        }
        lam[4 * c + t] = acc * 0.25;
    }
    double *fa[2] = {fa0, fa1}, *fk[2] = {fk0, fk1};
#pragma unroll
    for (int a = 0; a < 2; a++)
#pragma unroll
        for (int s = 0; s < 2; s++) {
            const int F0 = I + (a == 0 ? s : 0), F1 = J + (a == 1 ? s : 0);
            double sa = 0.0, sk = 0.0;
#pragma unroll
            for (int q = 0; q < 2; q++) {
                int f[2] = {2 * (F0 - g.b0[0]), 2 * (F1 - g.b0[1])};
                f[1 - a] += q;
                const long long fid = cf_fface(g, a, f[0], f[1]);
                sa += k.faf[a][fid];
                sk += k.fkf[a][fid];
            }
            const long long bid = cf_bface(g, a, F0, F1);
            fa[a][bid] = sa * 0.5;
            fk[a][bid] = sk * 0.5;
        }
}

// Per-block sums of squares of (T, p) of the valid base cells' residual and
// the patch's; the last block to finish sums the partials in block order into
// out[0..3] (L2 norms) and re-arms the ticket.
__global__ void __launch_bounds__(256) k_cf_norms(CfGeom g, const double2 *__restrict__ rb,
                                                  const double2 *__restrict__ rf, long long nb, long long nf,
                                                  double *__restrict__ partial, unsigned int *__restrict__ ticket,
                                                  double *__restrict__ out) {
    __shared__ double sm[4][256];
    __shared__ bool last;
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nb; q += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(q % g.n0), J = (int)(q / g.n0);
        if (cf_covered(g, I, J)) continue;
        a[0] += rb[q].x * rb[q].x;
        a[1] += rb[q].y * rb[q].y;
    }
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < nf; q += (long long)gridDim.x * blockDim.x) {
        a[2] += rf[q].x * rf[q].x;
        a[3] += rf[q].y * rf[q].y;
    }
#pragma unroll
    for (int v = 0; v < 4; v++) sm[v][threadIdx.x] = a[v];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o)
#pragma unroll
            for (int v = 0; v < 4; v++) sm[v][threadIdx.x] += sm[v][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
#pragma unroll
        for (int v = 0; v < 4; v++) partial[4 * blockIdx.x + v] = sm[v][0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double s[4] = {0.0, 0.0, 0.0, 0.0};
        for (unsigned q = 0; q < gridDim.x; q++)
#pragma unroll
            for (int v = 0; v < 4; v++) s[v] += __ldcg(partial + 4 * q + v);
#pragma unroll
        for (int v = 0; v < 4; v++) out[v] = sqrt(s[v]);
        *ticket = 0u;
    }
}

}  // namespace cmg
