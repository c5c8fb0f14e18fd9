// The implicit momentum predictor (Sec. 3, the equation before Eq. unp1):
//   (rho/dt) u - div(mu (grad u + grad u^T)) = R
// per cell and component, with rho, mu the cells' averaged density and
// viscosity.  Solved by defect correction: the full residual r = R - A(u)
// (k_mom_residual) drives a correction solve with the component-diagonal part
// of A - (rho/dt) u_c - div(mu_c,a grad u_c), mu_c,a = 2 mu on the faces
// normal to component c and mu on the others - on the pair multigrid of the
// pressure-temperature solve (two components per hierarchy, coupling
// coefficients lambda_2 = lambda_4 = 0).  The cross terms div(mu grad u^T)
// off the diagonal are the difference the outer loop removes.  When the
// set-up's row bound 2 (off-diagonal sum) / diagonal is small (the mass term
// dominates), the corrections are point-Jacobi steps instead (k_mom_jacobi);
// optionally the loop is restarted GMRES right-preconditioned by the
// multigrid correction (the k_kry_* kernels).
//
// Boundary faces: walls hold the normal component at zero (a Dirichlet face
// of the inner grid with coefficient 2 mu) and let the tangential ones slip
// (coefficient 0: no shear) or, with no-slip, hold them at zero too
// (coefficient mu); pressure boundaries and the axis pass no stress.  On
// axisymmetric grids the r-row has the hoop term 2 mu u_r / r^2.
// Tangential derivatives on a face are the mean of the two cells' central
// differences (one-sided in the first and last cell).
#pragma once
#include "mg_assemble.cuh"

namespace cmg {

struct MomCoeffArgs {
    int n[3];
    int wall[3][2];          // wall faces (normal component held at zero)
    int no_slip;
    double r0, h, dt, inv_dt, inv_h2;
    const double *rho, *mu;  // the caller's (k_mom_diag)
    double *rho_dt, *wgt;    // owned: rho / dt (mass term) and dt / rho (stopping weight)
    double *mu_o;            // owned copy of mu
    double *inv_diag[3];     // per component: 1 / the diagonal of the component-diagonal operator
    double *partial;         // per block: the largest Jacobi bound 2 off / diag of its cells and components
    double2 *lamA, *lamB;    // [N][2 pairs] of the correction hierarchies (B: 3D, component z)
    double *fA[2][3];        // face coefficients of components 0 and 1 (the hierarchies' T and p slots)
    double *fB[3];           // component 2 (3D)
};

__device__ __forceinline__ long long axis_stride(const int n[3], int a) {
    return a == 0 ? 1LL : a == 1 ? (long long)n[0] : (long long)n[0] * n[1];
}

// Per cell: the owned copies, the inverse diagonals of the component-diagonal operator and the row bound
// 2 (off-diagonal sum) / diagonal; per block, the largest bound.  A face's coefficient for component q is 2 mu_f on
// faces normal to q and mu_f on the others, mu_f the mean of the two cells' mu; on a boundary face mu of the cell at
// walls (normal component, or every component with no-slip, ghost factor 2) and 0 elsewhere.
template <int DIM, bool AXI>
__global__ void __launch_bounds__(256) k_mom_diag(const __grid_constant__ MomCoeffArgs A) {
    __shared__ double red[8];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    double nu = 0.0;
    if (i < A.n[0] && j < A.n[1]) {
        const long long c = (long long)i + (long long)A.n[0] * ((long long)j + (long long)A.n[1] * k);
        const double rho = A.rho[c], mu = A.mu[c];
        const double rdt = rho * A.inv_dt;
        A.rho_dt[c] = rdt;
        A.wgt[c] = A.dt / rho;
        A.mu_o[c] = mu;
        const int pos[3] = {i, j, k};
        double ri = 0.0;
        if (AXI) ri = A.r0 + (i + 0.5) * A.h;
        double off[DIM];
#pragma unroll
        for (int q = 0; q < DIM; q++) off[q] = 0.0;
#pragma unroll
        for (int a = 0; a < DIM; a++) {
#pragma unroll
            for (int sd = 0; sd < 2; sd++) {
                const int fpos = pos[a] + sd;
                const double w = ((AXI && a == 0) ? (ri + (sd ? 0.5 : -0.5) * A.h) / ri : 1.0) * A.inv_h2;
                if (fpos == 0 || fpos == A.n[a]) {
                    if (A.wall[a][sd]) {
#pragma unroll
                        for (int q = 0; q < DIM; q++)
                            if (q == a || A.no_slip) off[q] += w * 2.0 * (q == a ? 2.0 * mu : mu);
                    }
                } else {
                    const long long st = axis_stride(A.n, a);
                    const double mf = 0.5 * (mu + A.mu[sd ? c + st : c - st]);
#pragma unroll
                    for (int q = 0; q < DIM; q++) off[q] += w * (q == a ? 2.0 * mf : mf);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < DIM; q++) {
            const double diag = rdt + off[q] + ((AXI && q == 0) ? 2.0 * mu / (ri * ri) : 0.0);
            const double inv = 1.0 / diag;
            A.inv_diag[q][c] = inv;
            const double b = 2.0 * off[q] * inv;
            nu = (b > nu || b != b) ? b : nu;
        }
    }
    const int tid = threadIdx.x + blockDim.x * threadIdx.y;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, nu, o);
        nu = (y > nu || y != y) ? y : nu;
    }
    if ((tid & 31) == 0) red[tid >> 5] = nu;
    __syncthreads();
    if (tid == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x * blockDim.y) / 32; w++) t = (red[w] > t || red[w] != red[w]) ? red[w] : t;
        A.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * (long long)blockIdx.z)] = t;
    }
}

// Coefficients of the correction hierarchies (multigrid corrections only): lambda_1 = lambda_3 = -rho/dt
// (- 2 mu / r^2 for u_r), lambda_2 = lambda_4 = 0, and the face coefficients of each cell's low faces (and high
// faces on the high boundary).  Reads the owned rho/dt and mu written by k_mom_diag.
template <int DIM, bool AXI>
__global__ void __launch_bounds__(256) k_mom_hier(const __grid_constant__ MomCoeffArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const int n0 = A.n[0], n1 = A.n[1];
    const long long c = (long long)i + (long long)n0 * ((long long)j + (long long)n1 * k);
    const double mu = A.mu_o[c];
    const double m = -A.rho_dt[c];
    double l0 = m;
    if (AXI) {
        const double ri = A.r0 + (i + 0.5) * A.h;
        l0 = m - 2.0 * mu / (ri * ri);                      // hoop term of the r-row
    }
    A.lamA[2 * c] = make_double2(l0, 0.0);
    A.lamA[2 * c + 1] = make_double2(m, 0.0);
    if (DIM == 3) {
        A.lamB[2 * c] = make_double2(m, 0.0);
        A.lamB[2 * c + 1] = make_double2(m, 0.0);           // unused slot: p = 0 for a zero right-hand side
    }
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const int pos[3] = {i, j, k};
#pragma unroll
        for (int sd = 0; sd < 2; sd++) {
            const int fpos = pos[a] + sd;
            if (sd == 1 && fpos != A.n[a]) continue;
            const bool edge = fpos == 0 || fpos == A.n[a];
            double base[3];
            if (edge) {
                const int side = fpos == 0 ? 0 : 1;
                const bool w = A.wall[a][side] != 0;
#pragma unroll
                for (int q = 0; q < DIM; q++) base[q] = w && (q == a || A.no_slip) ? mu : 0.0;
            } else {
                const double mf = 0.5 * (mu + A.mu_o[c - axis_stride(A.n, a)]);
#pragma unroll
                for (int q = 0; q < DIM; q++) base[q] = mf;
            }
            const long long f = face_index(A.n, a, pos[0] + (a == 0 ? sd : 0), pos[1] + (a == 1 ? sd : 0),
                                           pos[2] + (a == 2 ? sd : 0));
            A.fA[0][a][f] = a == 0 ? 2.0 * base[0] : base[0];
            A.fA[1][a][f] = a == 1 ? 2.0 * base[1] : base[1];
            if (DIM == 3) A.fB[a][f] = a == 2 ? 2.0 * base[2] : base[2];
        }
    }
}

struct MomArgs {
    int n[3];
    int wall[3][2];
    int no_slip;
    double r0, h, inv_h, half_inv_h, two_inv_h, inv_dt, dt;
    const double *rho_dt, *wgt, *mu;   // rho / dt, dt / rho, mu per cell
    const double *u[3];
    const double *R[3];       // residual mode: the right-hand side
    double2 *rA, *rB;         // residual mode: -r as the inner right-hand sides (B: 3D, (-r_z, 0))
    double *partial;          // residual mode: per block sum of (dt r / rho)^2 over its cells and components
    double *r_out[3];         // residual mode, optional: r itself
    double *y[3];             // apply mode: A(u)
};

__device__ __forceinline__ long long cell_of(const int n[3], int i, int j, int k) {
    return (long long)i + (long long)n[0] * ((long long)j + (long long)n[1] * k);
}

// d u_q / d x_b at a cell: central inside, one-sided in the first and last cell.
__device__ __forceinline__ double mom_du(const MomArgs &A, int q, int b, const int pos[3]) {
    const int nb = A.n[b];
    if (nb < 2) return 0.0;
    int up[3] = {pos[0], pos[1], pos[2]}, dn[3] = {pos[0], pos[1], pos[2]};
    up[b] = pos[b] + 1 < nb ? pos[b] + 1 : pos[b];
    dn[b] = pos[b] > 0 ? pos[b] - 1 : pos[b];
    const double d = A.u[q][cell_of(A.n, up[0], up[1], up[2])] - A.u[q][cell_of(A.n, dn[0], dn[1], dn[2])];
    return d * (up[b] - dn[b] == 2 ? A.half_inv_h : A.inv_h);
}

// tau_{c a} for every component c on the face of axis a at face position f.
template <int DIM>
__device__ __forceinline__ void mom_face_stress(const MomArgs &A, int a, const int f[3], double tau[DIM]) {
    const int fa = f[a];
    if (fa == 0 || fa == A.n[a]) {
        const int side = fa == 0 ? 0 : 1;
        int cpos[3] = {f[0], f[1], f[2]};
        if (side) cpos[a] = fa - 1;
        const long long cc = cell_of(A.n, cpos[0], cpos[1], cpos[2]);
        const bool w = A.wall[a][side] != 0;
        const double mu = A.mu[cc];
#pragma unroll
        for (int q = 0; q < DIM; q++) {
            if (w && (q == a || A.no_slip)) {
                const double ub = A.u[q][cc];
                const double d = (side == 0 ? ub : -ub) * A.two_inv_h;     // towards the wall value 0
                tau[q] = (q == a ? 2.0 * mu : mu) * d;
            } else {
                tau[q] = 0.0;
            }
        }
        return;
    }
    int L[3] = {f[0], f[1], f[2]};
    L[a] = fa - 1;
    const long long cl = cell_of(A.n, L[0], L[1], L[2]), cr = cell_of(A.n, f[0], f[1], f[2]);
    const double mf = 0.5 * (A.mu[cl] + A.mu[cr]);
#pragma unroll
    for (int q = 0; q < DIM; q++) {
        const double normal = (A.u[q][cr] - A.u[q][cl]) * A.inv_h;
        if (q == a) {
            tau[q] = mf * (normal + normal);
        } else {
            const double tang = 0.5 * (mom_du(A, a, q, L) + mom_du(A, a, q, f));
            tau[q] = mf * (normal + tang);
        }
    }
}

template <int DIM, bool AXI, bool APPLY, int TX, int TY>
__global__ void __launch_bounds__(TX * TY) k_mom_residual(const __grid_constant__ MomArgs A) {
    constexpr int NX = (TX + 1) * TY, NY = TX * (TY + 1), NZ = DIM == 3 ? 2 * TX * TY : 0, NF = NX + NY + NZ;
    __shared__ double F[DIM][NF];
    __shared__ double red[TX * TY / 32];
    const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k = DIM == 3 ? (int)blockIdx.z : 0;
    const int tid = threadIdx.x + TX * threadIdx.y;
    for (int t = tid; t < NF; t += TX * TY) {
        int a, f[3];
        if (t < NX) {
            a = 0;
            f[0] = i0 + t % (TX + 1);
            f[1] = j0 + t / (TX + 1);
            f[2] = k;
        } else if (t < NX + NY) {
            const int v = t - NX;
            a = 1;
            f[0] = i0 + v % TX;
            f[1] = j0 + v / TX;
            f[2] = k;
        } else {
            const int v = t - NX - NY;
            a = 2;
            f[0] = i0 + v % TX;
            f[1] = j0 + (v / TX) % TY;
            f[2] = k + v / (TX * TY);
        }
        bool in = true;
#pragma unroll
        for (int b = 0; b < 3; b++) in = in && f[b] < A.n[b] + (b == a);
        double tau[DIM];
        if (in) {
            mom_face_stress<DIM>(A, a, f, tau);
        } else {
#pragma unroll
            for (int q = 0; q < DIM; q++) tau[q] = 0.0;
        }
#pragma unroll
        for (int q = 0; q < DIM; q++) F[q][t] = tau[q];
    }
    __syncthreads();
    const int li = threadIdx.x, lj = threadIdx.y, i = i0 + li, j = j0 + lj;
    double s = 0.0;
    if (i < A.n[0] && j < A.n[1]) {
        const long long c = cell_of(A.n, i, j, k);
        const double rdt = A.rho_dt[c];
        const int ilo[3] = {lj * (TX + 1) + li, NX + lj * TX + li, NX + NY + lj * TX + li};
        const int ihi[3] = {lj * (TX + 1) + li + 1, NX + (lj + 1) * TX + li, NX + NY + TX * TY + lj * TX + li};
        double ri = 0.0, wl = 0.0, wh = 0.0, inv_rh = 0.0;
        if (AXI) {
            ri = A.r0 + (i + 0.5) * A.h;
            wl = ri - 0.5 * A.h;
            wh = ri + 0.5 * A.h;
            inv_rh = 1.0 / (ri * A.h);
        }
        double Au[DIM];
#pragma unroll
        for (int q = 0; q < DIM; q++) {
            double div = 0.0;
#pragma unroll
            for (int a = 0; a < DIM; a++) {
                const double lo = F[q][ilo[a]], hi = F[q][ihi[a]];
                const double t = (AXI && a == 0) ? (wh * hi - wl * lo) * inv_rh : (hi - lo) * A.inv_h;
                div = a == 0 ? t : div + t;
            }
            const double uq = A.u[q][c];
            double v = rdt * uq - div;
            if (AXI && q == 0) v += 2.0 * A.mu[c] * uq / (ri * ri);
            Au[q] = v;
        }
        if (APPLY) {
#pragma unroll
            for (int q = 0; q < DIM; q++) A.y[q][c] = Au[q];
        } else {
            double r[DIM];
            const double w = A.wgt[c];
#pragma unroll
            for (int q = 0; q < DIM; q++) {
                r[q] = A.R[q][c] - Au[q];
                s += (w * r[q]) * (w * r[q]);
            }
            A.rA[c] = make_double2(-r[0], -r[1]);
            if (DIM == 3) A.rB[c] = make_double2(-r[DIM - 1], 0.0);
            if (A.r_out[0]) {
#pragma unroll
                for (int q = 0; q < DIM; q++) A.r_out[q][c] = r[q];
            }
        }
    }
    if constexpr (!APPLY) {
        // fixed-order block sum of the stopping norm
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if ((tid & 31) == 0) red[tid >> 5] = s;
        __syncthreads();
        if (tid == 0) {
            double b = 0.0;
            for (int w = 0; w < TX * TY / 32; w++) b += red[w];
            A.partial[blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * (long long)blockIdx.z)] = b;
        }
    }
}

// Largest value of an array (one block); non-finite values propagate as NaN.
__global__ void __launch_bounds__(1024) k_mom_max(const double *v, long long n, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long b = threadIdx.x; b < n; b += blockDim.x) {
        const double x = v[b];
        s = (x > s || x != x) ? x : s;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, s, o);
        s = (y > s || y != y) ? y : s;
    }
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t = (red[w] > t || red[w] != red[w]) ? red[w] : t;
        out[0] = t;
    }
}

// Point-Jacobi correction: delta_q += r_q / diag_q, r read back from the correction right-hand sides (-r).
template <int DIM>
__global__ void __launch_bounds__(256) k_mom_jacobi(long long N, const double2 *rA, const double2 *rB,
                                                    const double *i0, const double *i1, const double *i2, double *d0,
                                                    double *d1, double *d2) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double2 r = rA[c];
        d0[c] -= r.x * i0[c];
        d1[c] -= r.y * i1[c];
        if (DIM == 3) d2[c] -= rB[c].x * i2[c];
    }
}

// Sum of the per-block partials in a fixed order (one block).
__global__ void __launch_bounds__(1024) k_mom_norm(const double *partial, long long nblocks, double *out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long b = threadIdx.x; b < nblocks; b += blockDim.x) s += partial[b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w];
        out[0] = t;
    }
}

// u += delta, per component.
template <int DIM>
__global__ void __launch_bounds__(256) k_mom_add(long long N, const double *d0, const double *d1, const double *d2,
                                                 double *u0, double *u1, double *u2) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        u0[c] += d0[c];
        u1[c] += d1[c];
        if (DIM == 3) u2[c] += d2[c];
    }
}

// delta += the correction solves' solutions (A = (u_0, u_1), B = (u_2, unused)).
template <int DIM>
__global__ void __launch_bounds__(256) k_mom_update(long long N, const double2 *xA, const double2 *xB, double *u0,
                                                    double *u1, double *u2) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double2 d = xA[c];
        u0[c] += d.x;
        u1[c] += d.y;
        if (DIM == 3) u2[c] += xB[c].x;
    }
}

// ---------------------------------------------------------------- Krylov acceleration (restarted GMRES)
// Vectors hold all components, component q at offset q N.  The inner product is weighted like the stopping norm:
// <x, y> = sum over cells and components of (dt / rho)^2 x y.
constexpr int kKryM = 16;                 // restart length
constexpr int kKryBlocks = 152 * 4;       // grid of the reduction kernels (grid-stride)

struct KryCoef {
    double c[kKryM + 1];
};

// partial[d * gridDim.x + block] = block's share of <V_d, w>, d < nd (V_d at V + d * stride).
__global__ void __launch_bounds__(256) k_kry_dots(long long N, int dim, const double *wgt, const double *V,
                                                  long long stride, int nd, const double *w, double *partial) {
    __shared__ double red[8][kKryM + 1];
    double s[kKryM + 1];
#pragma unroll
    for (int d = 0; d <= kKryM; d++) s[d] = 0.0;
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double g = wgt[c] * wgt[c];
        for (int q = 0; q < dim; q++) {
            const double wv = g * w[q * N + c];
#pragma unroll
            for (int d = 0; d <= kKryM; d++)
                if (d < nd) s[d] += wv * V[d * stride + q * N + c];
        }
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int d = 0; d <= kKryM; d++) {
        if (d >= nd) break;
        double v = s[d];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) red[wid][d] = v;
    }
    __syncthreads();
    if ((int)threadIdx.x < nd) {
        double t = 0.0;
        for (int q = 0; q < (int)(blockDim.x >> 5); q++) t += red[q][threadIdx.x];
        partial[(long long)threadIdx.x * gridDim.x + blockIdx.x] = t;
    }
}

// out[d] = sum of the nblocks partials of dot d, in a fixed order (one block, one warp per dot).
__global__ void __launch_bounds__(1024) k_kry_reduce(const double *partial, int nblocks, int nd, double *out) {
    const int lane = threadIdx.x & 31, d = threadIdx.x >> 5;
    if (d >= nd) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(long long)d * nblocks + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) out[d] = s;
}

// w = scale * (w - sum_d h_d V_d), d < nd (scale 1: plain orthogonalisation).
__global__ void __launch_bounds__(256) k_kry_orth(long long M, const double *V, long long stride, int nd,
                                                  const __grid_constant__ KryCoef h, double scale, double *w) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
        double v = w[e];
        for (int d = 0; d < nd; d++) v -= h.c[d] * V[d * stride + e];
        w[e] = scale * v;
    }
}

// out = sum_d y_d V_d, d < nd.
__global__ void __launch_bounds__(256) k_kry_combine(long long M, const double *V, long long stride, int nd,
                                                     const __grid_constant__ KryCoef y, double *out) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < M; e += (long long)gridDim.x * blockDim.x) {
        double v = 0.0;
        for (int d = 0; d < nd; d++) v += y.c[d] * V[d * stride + e];
        out[e] = v;
    }
}

// The correction right-hand sides for M^-1 v: -v in the pair layouts (A = (v_0, v_1), B = (v_2, 0)).
template <int DIM>
__global__ void __launch_bounds__(256) k_kry_pack(long long N, const double *v, double2 *rA, double2 *rB) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        rA[c] = make_double2(-v[c], -v[N + c]);
        if (DIM == 3) rB[c] = make_double2(-v[2 * N + c], 0.0);
    }
}

// z = the correction solves' solutions, per component (add: z += instead).
template <int DIM, bool ADD>
__global__ void __launch_bounds__(256) k_kry_unpack(long long N, const double2 *xA, const double2 *xB, double *z0,
                                                    double *z1, double *z2) {
    for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N; c += (long long)gridDim.x * blockDim.x) {
        const double2 a = xA[c];
        if (ADD) {
            z0[c] += a.x;
            z1[c] += a.y;
            if (DIM == 3) z2[c] += xB[c].x;
        } else {
            z0[c] = a.x;
            z1[c] = a.y;
            if (DIM == 3) z2[c] = xB[c].x;
        }
    }
}

// ---------------------------------------------------------------- either side of the predictor
// Cell gradients are the means of a cell's two face gradients along each axis,
// the face gradients being those of the projection: (s_R - s_L)/h inside; for
// p, 2 (g - p)/h towards a Dirichlet value and 0 at walls and the axis; for C,
// 0 at every boundary.
struct MomSideArgs {
    int n[3];
    int dir[3][2];            // Dirichlet faces of p
    double gp[3][2];          // their values
    double inv_h, two_inv_h, half_inv_h, dt, inv_dt, sigma;
    const double *p, *C, *kappa, *rho;
    const double *mom[3], *u[3];
    double *R[3], *uf[3];
};

__device__ __forceinline__ double face_grad(const MomSideArgs &A, const double *s, bool dirichlet, int a,
                                            const int pos[3], int fpos, long long c, long long stride) {
    if (fpos == 0) return dirichlet && A.dir[a][0] ? (s[c] - A.gp[a][0]) * A.two_inv_h : 0.0;
    if (fpos == A.n[a]) return dirichlet && A.dir[a][1] ? (A.gp[a][1] - s[c]) * A.two_inv_h : 0.0;
    // interior face between the cell at fpos - 1 and the one at fpos (c is the cell at pos[a])
    const long long lo = c + (long long)(fpos - 1 - pos[a]) * stride, hi = lo + stride;
    return (s[hi] - s[lo]) * A.inv_h;
}

__device__ __forceinline__ double cell_grad(const MomSideArgs &A, const double *s, bool dirichlet, int a,
                                            const int pos[3], long long c) {
    const long long st = a == 0 ? 1LL : a == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1];
    const double lo = face_grad(A, s, dirichlet, a, pos, pos[a], c, st);
    const double hi = face_grad(A, s, dirichlet, a, pos, pos[a] + 1, c, st);
    return 0.5 * (lo + hi);
}

// R = (rho u)^(adv)/dt - grad p^n + sigma kappa grad C per cell.
template <int DIM>
__global__ void __launch_bounds__(256) k_mom_rhs(const __grid_constant__ MomSideArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const long long c = cell_of(A.n, i, j, k);
    const int pos[3] = {i, j, k};
    const double sk = A.sigma * A.kappa[c];
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const double gpa = cell_grad(A, A.p, true, a, pos, c), gCa = cell_grad(A, A.C, false, a, pos, c);
        A.R[a][c] = A.mom[a][c] * A.inv_dt - gpa + sk * gCa;
    }
}

// Eq. provel at the cells, u* = u_pred + (dt/rho) grad p^n, and the face-normal components: the mean of the two
// cells' inside, 0 at walls and the axis, the cell's value at a pressure boundary.  Each cell writes its low face
// of every axis and, in the last cell, the high one.
template <int DIM>
__global__ void __launch_bounds__(256) k_provisional(const __grid_constant__ MomSideArgs A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y * blockDim.y + threadIdx.y;
    const int k = DIM == 3 ? (int)blockIdx.z : 0;
    if (i >= A.n[0] || j >= A.n[1]) return;
    const long long c = cell_of(A.n, i, j, k);
    const int pos[3] = {i, j, k};
#pragma unroll
    for (int a = 0; a < DIM; a++) {
        const long long st = a == 0 ? 1LL : a == 1 ? (long long)A.n[0] : (long long)A.n[0] * A.n[1];
        const double us = A.u[a][c] + A.dt / A.rho[c] * cell_grad(A, A.p, true, a, pos, c);
        // low face
        double v;
        if (pos[a] == 0) {
            v = A.dir[a][0] ? us : 0.0;
        } else {
            int pl[3] = {pos[0], pos[1], pos[2]};
            pl[a] = pos[a] - 1;
            const long long cl = c - st;
            const double ul = A.u[a][cl] + A.dt / A.rho[cl] * cell_grad(A, A.p, true, a, pl, cl);
            v = 0.5 * (ul + us);
        }
        A.uf[a][face_index(A.n, a, i, j, k)] = v;
        if (pos[a] == A.n[a] - 1) {
            A.uf[a][face_index(A.n, a, i + (a == 0), j + (a == 1), k + (a == 2))] = A.dir[a][1] ? us : 0.0;
        }
    }
}

}  // namespace cmg
